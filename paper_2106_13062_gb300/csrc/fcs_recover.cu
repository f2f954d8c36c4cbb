// fcs_recover.cu -- fcs_recover: entry estimates from sketches, the
// decompressing rule of the Kronecker / tensor-contraction compression
// subsections:
//   raw_d[q] = prod_n s_n(i_n) * sketch_d[ sum_n h_n(i_n) ],  out[q] = median_d.
// One thread per sample: N index loads, D table lookups per mode (tables
// staged in shared memory, h and the sign packed into one int32), D gathers
// from the sketches (L1/L2 resident), and the median in registers.
#include "fcs_internal.cuh"

namespace fcs {
namespace {

struct RecoverArgs {
  Modes m;
  const float *sketch;
  const int32_t *h;
  const int8_t *s;
  const int32_t *idx;
  float *out;
  float *raw;
  int64_t M;
  int64_t sbs, ibs, obs;   // batch strides
  int tot;
};

template <int D, bool SMEM>
__global__ void __launch_bounds__(256) recover_kernel(RecoverArgs a) {
  extern __shared__ __align__(16) int32_t tab[];
  const int N = a.m.N, tot = a.tot;
  if (SMEM) {
    for (int e = threadIdx.x; e < D * tot; e += blockDim.x) {
      const int d = e / tot;
      const int64_t g = d * a.m.ldh + (e - d * tot);
      tab[e] = (a.h[g] << 1) | (a.s[g] < 0 ? 1 : 0);
    }
    __syncthreads();
  }
  const int64_t b = blockIdx.y;
  const float *sk = a.sketch + b * a.sbs;
  const int32_t *idx = a.idx + b * a.ibs;
  float *out = a.out + b * a.obs;
  const int64_t Jt = a.m.Jt;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < a.M;
       q += int64_t(gridDim.x) * blockDim.x) {
    int bin[D], neg[D];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < D; ++d) bin[d] = neg[d] = 0;
    for (int n = 0; n < N; ++n) {
      int64_t i = __ldcs(idx + q * N + n);
      if (i < 0 || i >= a.m.I[n]) {      // index outside the tensor: NaN result
        ok = false;
        i = 0;
      }
      const int64_t e = a.m.off[n] + i;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int32_t t =
            SMEM ? tab[d * tot + e]
                 : ((__ldg(a.h + d * a.m.ldh + e) << 1) | (__ldg(a.s + d * a.m.ldh + e) < 0));
        bin[d] += t >> 1;
        neg[d] ^= t & 1;
      }
    }
    float v[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const bool in = ok && unsigned(bin[d]) < unsigned(Jt);
      const float x = in ? __ldg(sk + d * Jt + bin[d]) : __int_as_float(0x7fc00000);
      v[d] = neg[d] ? -x : x;
      if (a.raw) a.raw[d * a.M + q] = v[d];
    }
    __stcs(out + q, median_inplace<D>(v));
  }
}

template <int D>
int launch_recover(fcs_ctx *ctx, RecoverArgs &a, int64_t nbatch) {
  const size_t smem = size_t(D) * a.tot * sizeof(int32_t);
  const bool use_smem = smem <= 96 * 1024;
  auto kern = use_smem ? recover_kernel<D, true> : recover_kernel<D, false>;
  const size_t sm = use_smem ? smem : 0;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(recover)");
  }
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm);
  if (per_sm < 1) per_sm = 1;
  int64_t want = int64_t(ctx->sm_count) * per_sm;
  int64_t per_item = (want + nbatch - 1) / nbatch;
  const int64_t need = (a.M + 255) / 256;
  if (per_item > need) per_item = need;
  if (per_item < 1) per_item = 1;
  kern<<<dim3(unsigned(per_item), unsigned(nbatch)), 256, sm, ctx->stream>>>(a);
  return check_cuda(ctx, cudaGetLastError(), "recover_kernel");
}

}  // namespace
}  // namespace fcs

using namespace fcs;

extern "C" int fcs_recover(fcs_ctx *ctx, int N, const int64_t *host_I, const int32_t *host_J,
                           int D, const float *sketch, const int32_t *h, const int8_t *s,
                           int64_t ldh, int64_t M, const int32_t *idx, float *out,
                           float *out_raw, int64_t nbatch, int64_t sketch_batch_stride,
                           int64_t idx_batch_stride, int64_t out_batch_stride) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  RecoverArgs a{};
  int rc = make_modes(ctx, N, host_I, host_J, ldh, &a.m);
  if (rc) return rc;
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (M < 0) return set_error(ctx, FCS_EINVAL, "M=%lld < 0", (long long)M);
  if (nbatch < 1 || nbatch > 65535)
    return set_error(ctx, FCS_EINVAL, "nbatch=%lld outside [1,65535]", (long long)nbatch);
  if (nbatch > 1 && out_raw)
    return set_error(ctx, FCS_EINVAL, "out_raw must be NULL when nbatch > 1");
  if (M == 0) return FCS_OK;
  if (!sketch || !h || !s || !idx || !out) return set_error(ctx, FCS_EINVAL, "NULL pointer");
  int64_t tot = 0;
  for (int n = 0; n < N; ++n) tot += host_I[n];
  a.tot = int(tot);
  a.sketch = sketch;
  a.h = h;
  a.s = s;
  a.idx = idx;
  a.out = out;
  a.raw = out_raw;
  a.M = M;
  a.sbs = nbatch > 1 ? sketch_batch_stride : 0;
  a.ibs = nbatch > 1 ? idx_batch_stride : 0;
  a.obs = nbatch > 1 ? out_batch_stride : 0;
  DeviceGuard g(ctx->device);
  switch (D) {
#define FCS_REC_CASE(K) \
  case K: return launch_recover<K>(ctx, a, nbatch);
    FCS_REC_CASE(1) FCS_REC_CASE(2) FCS_REC_CASE(3) FCS_REC_CASE(4) FCS_REC_CASE(5)
    FCS_REC_CASE(6) FCS_REC_CASE(7) FCS_REC_CASE(8) FCS_REC_CASE(9) FCS_REC_CASE(10)
    FCS_REC_CASE(11) FCS_REC_CASE(12) FCS_REC_CASE(13) FCS_REC_CASE(14) FCS_REC_CASE(15)
    FCS_REC_CASE(16)
#undef FCS_REC_CASE
    default:
      break;
  }
  return set_error(ctx, FCS_EINVAL, "D=%d outside [1,16]", D);
}
