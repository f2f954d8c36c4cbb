// fcs_outer.cu -- fcs_sketch_outer / fcs_sketch_outer_sum: sketch of an
// outer product from the sketches of its factors (Kronecker product
// compression), and of a contraction over one mode from the sketches of its
// slices (tensor contraction compression):
//   FCS(A o B)          = IFFT_P( FFT_P(FCS A) * FFT_P(FCS B) ),
//   FCS(A (x)_{3,1} B)  = IFFT_P( sum_l FFT_P(FCS A_l) * FFT_P(FCS B_l) ),
// P >= La + Lb - 1, i.e. full linear convolutions; the slice sum stays in the
// frequency domain, so each (batch item, sketch) needs one inverse.  One CTA
// per (batch item, sketch): two real forward FFTs per slice in shared
// memory, the products summed in registers, one inverse real FFT.
#include "fcs_fft.cuh"

namespace fcs {
namespace {

// fa [nbatch][L][D][La], fb [nbatch][L][D][Lb] -> out [nbatch][D][La+Lb-1].
template <int LOG2M, int NT>
__global__ void __launch_bounds__(NT) outer_kernel(const float *__restrict__ fa,
                                                   const float *__restrict__ fb, int64_t La,
                                                   int64_t Lb, int64_t L, int D, int sb,
                                                   float *__restrict__ out,
                                                   const float2 *__restrict__ tw) {
  using LPs = LastPass<LOG2M, NT>;
  using Lay = FftSmem<LOG2M>;
  constexpr int M = 1 << LOG2M;
  constexpr int RL = LPs::RL, EPS = LPs::EPS;
  extern __shared__ __align__(16) unsigned char smem[];
  float2 *B = reinterpret_cast<float2 *>(smem + Lay::kB);
  float2 *tws = reinterpret_cast<float2 *>(smem + Lay::kTw);
  float *A = reinterpret_cast<float *>(smem + Lay::kA);
  const int tid = threadIdx.x;
  const int64_t bi = blockIdx.y;
  const int d = blockIdx.x;
  fill_twiddles<LOG2M, NT>(tws, tw);
  float2 *lps = reinterpret_cast<float2 *>(smem + Lay::kLp);
  LastPassTwShared<LOG2M, NT>::fill(lps, tw);
  const LastPassTwShared<LOG2M, NT> ltw{lps};
  float2 acc[EPS][2][RL], p[EPS][2][RL], X[EPS][2][RL];
#pragma unroll
  for (int e = 0; e < EPS; ++e)
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int r = 0; r < RL; ++r) acc[e][bb][r] = make_float2(0.f, 0.f);
  for (int64_t l = 0; l < L; ++l) {
    const int64_t slice = (bi * L + l) * D + d;
    for (int side = 0; side < 2; ++side) {
      const int64_t len = side == 0 ? La : Lb;
      const float *x = (side == 0 ? fa : fb) + slice * len;
      for (int j = tid; j < sb; j += NT) A[j] = j < len ? __ldg(x + j) : 0.f;
      rfft_to_slots<LOG2M, NT>(A, sb, B, tws, ltw, X);
#pragma unroll
      for (int e = 0; e < EPS; ++e)
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
          for (int r = 0; r < RL; ++r) {
            const bool packed = bb == 0 && r == 0 && tid + e * NT == 0;
            if (side == 0)
              p[e][bb][r] = X[e][bb][r];
            else
              acc[e][bb][r] = cadd(acc[e][bb][r], slot_mul(p[e][bb][r], X[e][bb][r], packed));
          }
    }
  }
  slots_to_conj_packed<LOG2M, NT>(B, acc, tw);
  __syncthreads();
  block_fft<LOG2M, NT>(B, tw);
  const int64_t Lo = La + Lb - 1;
  float *o = out + (bi * D + d) * Lo;
  const float sc = 1.0f / float(M);
  const float *bufr = reinterpret_cast<const float *>(B);
  for (int64_t j = tid; j < Lo; j += NT) {
    const float v = bufr[real_off(int(j))];
    o[j] = (j & 1) ? -v * sc : v * sc;
  }
}

template <int LOG2M>
int launch_outer(fcs_ctx *ctx, int64_t nbatch, int64_t L, int D, int64_t La, int64_t Lb,
                 const float *fa, const float *fb, float *out) {
  constexpr int NT = fft_threads(LOG2M);
  const int sb = int(((La > Lb ? La : Lb) + 3) / 4 * 4);
  const size_t smem = FftSmem<LOG2M>::bytes(sb);
  auto kern = outer_kernel<LOG2M, NT>;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(outer)");
  }
  kern<<<dim3(unsigned(D), unsigned(nbatch)), NT, smem, ctx->stream>>>(fa, fb, La, Lb, L, D, sb,
                                                                       out, ctx->twiddle);
  return check_cuda(ctx, cudaGetLastError(), "outer_kernel");
}

}  // namespace
}  // namespace fcs

using namespace fcs;

namespace fcs {
namespace {

int sketch_outer(fcs_ctx *ctx, int64_t nbatch, int64_t nslices, int D, int64_t La, int64_t Lb,
                 const float *fa, const float *fb, float *out) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (nbatch < 1 || nbatch > 65535)
    return set_error(ctx, FCS_EINVAL, "nbatch=%lld outside [1,65535]", (long long)nbatch);
  if (nslices < 1) return set_error(ctx, FCS_EINVAL, "L=%lld must be >= 1", (long long)nslices);
  if (La < 1 || Lb < 1) return set_error(ctx, FCS_EINVAL, "sketch lengths must be >= 1");
  if (!fa || !fb || !out) return set_error(ctx, FCS_EINVAL, "NULL pointer argument");
  const int64_t Lo = La + Lb - 1;
  const int log2p = ilog2_ceil(Lo) < kMinLog2P ? kMinLog2P : ilog2_ceil(Lo);
  if (log2p > kMaxLog2PBig)
    return set_error(ctx, FCS_EUNSUPPORTED, "output length %lld needs FFT length > %d",
                     (long long)Lo, 1 << kMaxLog2PBig);
  DeviceGuard g(ctx->device);
  spec_cache_invalidate(ctx, out, sizeof(float) * size_t(nbatch) * D * size_t(Lo));
  if (log2p > kMaxLog2P) return big_outer(ctx, nbatch, nslices, D, La, Lb, fa, fb, out, log2p);
  int rc = FCS_EUNSUPPORTED;
  FCS_DISPATCH_LOG2M(log2p - 1, rc = launch_outer<L>(ctx, nbatch, nslices, D, La, Lb, fa, fb, out));
  return rc;
}

}  // namespace
}  // namespace fcs

extern "C" int fcs_sketch_outer(fcs_ctx *ctx, int64_t nbatch, int D, int64_t La, int64_t Lb,
                                const float *fa, const float *fb, float *out) {
  return sketch_outer(ctx, nbatch, 1, D, La, Lb, fa, fb, out);
}

extern "C" int fcs_sketch_outer_sum(fcs_ctx *ctx, int64_t nbatch, int64_t L, int D, int64_t La,
                                    int64_t Lb, const float *fa, const float *fb, float *out) {
  return sketch_outer(ctx, nbatch, L, D, La, Lb, fa, fb, out);
}
