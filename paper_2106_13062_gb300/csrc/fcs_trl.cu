// fcs_trl.cu -- fcs_sketch_inner: inner products between two sets of
// sketches, the compressed tensor regression layer (TRL subsection, eq.
// net_compress):
//     raw[b][c][d] = < FCS_d(X_b), FCS_d(W_c) >,
//     Y[b][c] = median_d raw[b][c][d] + bias[c],
// i.e. per sketch d the product of the [B][Jt] activation sketches with the
// transposed [C][Jt] weight sketches, then the median over the D sketches.
//
// The product kernel tiles (b, c) by 64 x 64 per CTA (256 threads, 4 x 4
// outputs each), stages 32-bin slices of both operands in shared memory and
// accumulates in FP32 registers, one sketch d per grid z; the median kernel
// then reads the D values of each output.  The sketch is Jt long and B, C
// are batch and class counts, so this is a small dense contraction on the
// FP32 pipe; it is not the hot path.
#include "fcs_internal.cuh"

namespace fcs {
namespace {

constexpr int kTile = 64;
constexpr int kK = 32;

// raw[(b*C + c)*D + d] = sum_j sa[(b*D + d)*Jt + j] * sw[(c*D + d)*Jt + j]
__global__ void __launch_bounds__(256) inner_kernel(const float *__restrict__ sa,
                                                    const float *__restrict__ sw, int64_t B,
                                                    int64_t C, int D, int64_t Jt,
                                                    float *__restrict__ raw) {
  __shared__ float As[kK][kTile + 1];
  __shared__ float Ws[kK][kTile + 1];
  const int d = blockIdx.z;
  const int64_t b0 = int64_t(blockIdx.y) * kTile, c0 = int64_t(blockIdx.x) * kTile;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;    // 16 x 16 threads
  float acc[4][4] = {};
  for (int64_t j0 = 0; j0 < Jt; j0 += kK) {
    // stage sa[b0 .. b0+63][d][j0 .. j0+31] and the same for sw (zeros past the ends)
    for (int e = threadIdx.x; e < kTile * kK; e += 256) {
      const int r = e / kK, k = e % kK;
      const int64_t j = j0 + k;
      const int64_t b = b0 + r, c = c0 + r;
      As[k][r] = (b < B && j < Jt) ? __ldg(sa + (b * D + d) * Jt + j) : 0.f;
      Ws[k][r] = (c < C && j < Jt) ? __ldg(sw + (c * D + d) * Jt + j) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kK; ++k) {
      float a[4], w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[k][ty + 16 * i];
        w[i] = Ws[k][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(a[i], w[q], acc[i][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t b = b0 + ty + 16 * i, c = c0 + tx + 16 * q;
      if (b < B && c < C) raw[(b * C + c) * D + d] = acc[i][q];
    }
}

template <int D>
__global__ void median_bias_kernel(const float *__restrict__ raw, int64_t BC, int64_t C,
                                   const float *__restrict__ bias, float *__restrict__ out) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < BC;
       t += int64_t(gridDim.x) * blockDim.x) {
    float v[D];
#pragma unroll
    for (int d = 0; d < D; ++d) v[d] = raw[t * D + d];
    const float m = median_net<D>(v);
    out[t] = bias ? m + __ldg(bias + t % C) : m;
  }
}

}  // namespace
}  // namespace fcs

using namespace fcs;

extern "C" int fcs_sketch_inner(fcs_ctx *ctx, int D, int64_t Jt, int64_t B, const float *sa,
                                int64_t C, const float *sw, const float *bias, float *out_median,
                                float *out_raw) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (Jt < 1 || B < 1 || C < 1) return set_error(ctx, FCS_EINVAL, "sizes must be >= 1");
  if ((B + kTile - 1) / kTile > 65535)
    return set_error(ctx, FCS_EINVAL, "B=%lld too large", (long long)B);
  if (!sa || !sw || !out_median) return set_error(ctx, FCS_EINVAL, "NULL pointer argument");
  DeviceGuard g(ctx->device);
  float *raw = out_raw;
  if (!raw) {
    int rc = ensure_raw(ctx, sizeof(float) * size_t(B) * size_t(C) * D);
    if (rc) return rc;
    raw = ctx->raw;
  }
  const dim3 grid(unsigned((C + kTile - 1) / kTile), unsigned((B + kTile - 1) / kTile),
                  unsigned(D));
  inner_kernel<<<grid, 256, 0, ctx->stream>>>(sa, sw, B, C, D, Jt, raw);
  int rc = check_cuda(ctx, cudaGetLastError(), "inner_kernel");
  if (rc) return rc;
  const int64_t BC = B * C;
  int blocks = int((BC + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  switch (D) {
#define FCS_MB_CASE(K) \
  case K: median_bias_kernel<K><<<blocks, 256, 0, ctx->stream>>>(raw, BC, C, bias, out_median); break;
    FCS_MB_CASE(1) FCS_MB_CASE(2) FCS_MB_CASE(3) FCS_MB_CASE(4) FCS_MB_CASE(5)
    FCS_MB_CASE(6) FCS_MB_CASE(7) FCS_MB_CASE(8) FCS_MB_CASE(9) FCS_MB_CASE(10)
    FCS_MB_CASE(11) FCS_MB_CASE(12) FCS_MB_CASE(13) FCS_MB_CASE(14) FCS_MB_CASE(15)
    FCS_MB_CASE(16)
#undef FCS_MB_CASE
    default: break;
  }
  return check_cuda(ctx, cudaGetLastError(), "median_bias_kernel");
}
