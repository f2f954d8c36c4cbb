// fcs_host.cu -- fcs_sketch_cp_host: the CP-route sketch of eq. (FCS_syn)
// from factor matrices in host memory to a sketch in host memory.  The call
// copies the factors (and lambda) into a staging buffer the context owns,
// generates the hash tables from the seed and sketches
// (fcs_sketch_cp_seeded) and copies the D sketches back, all on the
// context's stream; the host output is complete once that stream is
// synchronised.
// Host ranges that lie back to back in memory (factors stored one after
// another, as in one staging block) move in one copy.
#include <vector>

#include "fcs_internal.cuh"

namespace fcs {
namespace {

// Grow the context's host-copy staging buffer to `bytes` (previous contents
// are not kept; stream-ordered, as every context buffer).
int ensure_stage(fcs_ctx *ctx, size_t bytes, void **out) {
  int rc = grow_buffer(ctx, &ctx->stage, &ctx->stage_bytes, bytes, "staging buffer");
  if (rc) return rc;
  *out = ctx->stage;
  return FCS_OK;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace fcs

using namespace fcs;

extern "C" int fcs_sketch_cp_host(fcs_ctx *ctx, int N, const int64_t *host_I,
                                  const int32_t *host_J, int64_t R, int D,
                                  const float *const *host_U, const int64_t *host_ldU,
                                  const float *host_lambda, uint64_t seed, float *host_out) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  Modes m;
  int rc = make_modes(ctx, N, host_I, host_J, 0, &m);
  if (rc) return rc;
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (R < 1) return set_error(ctx, FCS_EINVAL, "R=%lld must be >= 1", (long long)R);
  if (!host_U || !host_ldU || !host_out) return set_error(ctx, FCS_EINVAL, "NULL pointer argument");
  for (int n = 0; n < N; ++n) {
    if (!host_U[n]) return set_error(ctx, FCS_EINVAL, "U[%d] is NULL", n);
    if (host_ldU[n] < R)
      return set_error(ctx, FCS_EINVAL, "ldU[%d]=%lld < R", n, (long long)host_ldU[n]);
  }
  // staging layout: [U_1 .. U_N (I_n x R, dense, back to back) | lambda | h | s | out]
  int64_t totI = 0, ufl = 0;
  for (int n = 0; n < N; ++n) {
    totI += host_I[n];
    ufl += host_I[n] * R;
  }
  const size_t b_u = sizeof(float) * size_t(ufl + (host_lambda ? R : 0));
  const size_t b_h = sizeof(int32_t) * size_t(D) * size_t(totI);
  const size_t b_s = size_t(D) * size_t(totI);
  const size_t b_o = sizeof(float) * size_t(D) * size_t(m.Jt);
  const size_t o_h = up256(b_u), o_s = o_h + up256(b_h), o_o = o_s + up256(b_s);
  DeviceGuard g(ctx->device);
  void *stage = nullptr;
  rc = ensure_stage(ctx, o_o + b_o, &stage);
  if (rc) return rc;
  char *base = static_cast<char *>(stage);
  float *Ud = reinterpret_cast<float *>(base);
  int32_t *hd = reinterpret_cast<int32_t *>(base + o_h);
  int8_t *sd = reinterpret_cast<int8_t *>(base + o_s);
  float *od = reinterpret_cast<float *>(base + o_o);

  // host -> device: dense factor blocks and lambda, merged where the host
  // ranges continue each other
  struct Piece {
    const char *src;
    char *dst;
    size_t bytes;
  };
  std::vector<Piece> pieces;
  std::vector<const float *> Udev(N);
  std::vector<int64_t> ld(N, R);
  float *cur = Ud;
  for (int n = 0; n < N; ++n) {
    Udev[n] = cur;
    const size_t row = sizeof(float) * size_t(R);
    if (host_ldU[n] == R) {
      pieces.push_back({reinterpret_cast<const char *>(host_U[n]), reinterpret_cast<char *>(cur),
                        row * size_t(host_I[n])});
    } else {
      // strided rows: one 2D copy, not merged
      cudaError_t e = cudaMemcpy2DAsync(cur, row, host_U[n], sizeof(float) * size_t(host_ldU[n]),
                                        row, size_t(host_I[n]), cudaMemcpyHostToDevice,
                                        ctx->stream);
      if (e != cudaSuccess) return check_cuda(ctx, e, "cudaMemcpy2DAsync(U)");
    }
    cur += host_I[n] * R;
  }
  const float *lamd = nullptr;
  if (host_lambda) {
    lamd = cur;
    pieces.push_back({reinterpret_cast<const char *>(host_lambda), reinterpret_cast<char *>(cur),
                      sizeof(float) * size_t(R)});
  }
  for (size_t k = 0; k < pieces.size();) {
    Piece p = pieces[k++];
    while (k < pieces.size() && pieces[k].src == p.src + p.bytes &&
           pieces[k].dst == p.dst + p.bytes)
      p.bytes += pieces[k++].bytes;
    cudaError_t e = cudaMemcpyAsync(p.dst, p.src, p.bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return check_cuda(ctx, e, "cudaMemcpyAsync(H2D)");
  }
  rc = fcs_sketch_cp_seeded(ctx, seed, N, host_I, host_J, R, D, Udev.data(), ld.data(), lamd, hd,
                            sd, od);
  if (rc) return rc;
  return check_cuda(ctx, cudaMemcpyAsync(host_out, od, b_o, cudaMemcpyDeviceToHost, ctx->stream),
                    "cudaMemcpyAsync(D2H)");
}
