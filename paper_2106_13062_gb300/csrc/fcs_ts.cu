// fcs_ts.cu -- fcs_fold: Tensor Sketch (Def. 2) from Fast Count Sketch.
//
// With every hash length J_n = J, the TS bin (sum_n h_n(i_n)) mod J is the
// FCS bin sum_n h_n(i_n) reduced mod J, so TS_d[j] = sum_{k = j mod J}
// FCS_d[k]: the mod-J circular convolution of eq. TS is the linear one of
// eq. FCS_syn folded.  One FCS therefore yields the TS with the same hash
// functions (the comparison of Prop. 1).  Each output sums at most
// ceil(Jt / J) inputs; reads and writes are coalesced.
#include "fcs_internal.cuh"

namespace fcs {
namespace {

__global__ void fold_kernel(const float *__restrict__ in, int64_t Jt, int64_t J,
                            float *__restrict__ out) {
  const int64_t row = blockIdx.y;
  const float *x = in + row * Jt;
  float *y = out + row * J;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < J;
       j += int64_t(gridDim.x) * blockDim.x) {
    float acc = 0.f;
    for (int64_t k = j; k < Jt; k += J) acc += __ldg(x + k);
    y[j] = acc;
  }
}

}  // namespace
}  // namespace fcs

using namespace fcs;

extern "C" int fcs_fold(fcs_ctx *ctx, int64_t nrows, int64_t Jt, const float *in, int64_t J,
                        float *out) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  if (nrows < 1 || nrows > 65535)
    return set_error(ctx, FCS_EINVAL, "nrows=%lld outside [1,65535]", (long long)nrows);
  if (Jt < 1 || J < 1) return set_error(ctx, FCS_EINVAL, "lengths must be >= 1");
  if (!in || !out) return set_error(ctx, FCS_EINVAL, "NULL pointer argument");
  DeviceGuard g(ctx->device);
  spec_cache_invalidate(ctx, out, sizeof(float) * size_t(nrows) * size_t(J));
  int64_t blocks = (J + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  fold_kernel<<<dim3(unsigned(blocks), unsigned(nrows)), 256, 0, ctx->stream>>>(in, Jt, J, out);
  return check_cuda(ctx, cudaGetLastError(), "fold_kernel");
}
