// fcs_hash.cu -- fcs_make_hashes: the per-mode hash pairs {h_n, s_n} of
// Def. 4 for D independent sketches (the family is in fcs_hash.cuh).
#include "fcs_hash.cuh"

namespace fcs {
namespace {

// One thread per table entry (d, global position e in [0, total)).
__global__ void make_hashes_kernel(HashArgs a, int32_t *__restrict__ h,
                                   int8_t *__restrict__ s) {
  const int d = blockIdx.y;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < a.total;
       e += int64_t(gridDim.x) * blockDim.x)
    hash_entry(a, d, e, h, s);
}

}  // namespace
}  // namespace fcs

using namespace fcs;

extern "C" int fcs_make_hashes(fcs_ctx *ctx, uint64_t seed, int N, const int64_t *host_I,
                               const int32_t *host_J, int D, int32_t *h, int8_t *s) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  Modes m;
  int rc = make_modes(ctx, N, host_I, host_J, 0, &m);
  if (rc) return rc;
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (!h || !s) return set_error(ctx, FCS_EINVAL, "h or s is NULL");
  for (int n = 0; n < N; ++n)
    if (host_I[n] > (int64_t(1) << 32))
      return set_error(ctx, FCS_EINVAL, "I[%d] too large for the hash family", n);
  const HashArgs a = hash_args(seed, N, D, host_I, host_J);
  DeviceGuard g(ctx->device);
  const int threads = 256;
  int64_t blocks = (a.total + threads - 1) / threads;
  if (blocks > 65535) blocks = 65535;
  make_hashes_kernel<<<dim3(unsigned(blocks), unsigned(D)), threads, 0, ctx->stream>>>(a, h, s);
  return check_cuda(ctx, cudaGetLastError(), "make_hashes_kernel");
}
