// fcs_outer.cu -- fcs_sketch_outer / fcs_sketch_outer_sum: sketch of an
// outer product from the sketches of its factors (Kronecker product
// compression), and of a contraction over one mode from the sketches of its
// slices (tensor contraction compression):
//   FCS(A o B)          = IFFT_P( FFT_P(FCS A) * FFT_P(FCS B) ),
//   FCS(A (x)_{3,1} B)  = IFFT_P( sum_l FFT_P(FCS A_l) * FFT_P(FCS B_l) ),
// P >= La + Lb - 1, i.e. full linear convolutions; the slice sum stays in the
// frequency domain, so each (batch item, sketch) needs one inverse.  One CTA
// per (batch item, sketch): two real forward FFTs per slice in shared
// memory, the products summed in registers, one inverse real FFT.  The
// block has the slot FFT's M/16 threads, or twice that when
// fcs_outer_autotune found it faster for the problem's shape.
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

#include "fcs_fft.cuh"

namespace fcs {
namespace {

// Shared-memory layout of outer_kernel: as FftSmem, with the last-pass
// twiddle region sized for the block's NT threads (each thread parks its own
// column there).
template <int L, int NT>
struct OuterSmem {
  static constexpr size_t up16(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t kB = 0;
  static constexpr size_t kTw = up16(sizeof(float2) * padded_len(1 << L));
  static constexpr size_t kLp = up16(kTw + sizeof(float2) * plan_twlen(L));
  static constexpr size_t kA = up16(kLp + sizeof(float2) * LastPassTwShared<L, NT>::kLen);
  static size_t bytes(int sb) { return kA + sizeof(float) * size_t(sb); }
};

// fa [nbatch][L][D][La], fb [nbatch][L][D][Lb] -> out [nbatch][D][La+Lb-1].
template <int LOG2M, int NT>
__global__ void __launch_bounds__(NT) outer_kernel(const float *__restrict__ fa,
                                                   const float *__restrict__ fb, int64_t La,
                                                   int64_t Lb, int64_t L, int D, int sb,
                                                   float *__restrict__ out,
                                                   const float2 *__restrict__ tw) {
  using LPs = LastPass<LOG2M, NT>;
  using Lay = OuterSmem<LOG2M, NT>;
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

// Thread multiplier of the block (1: M/16 threads, at least a warp; 2: twice
// that, where it stays within 1024).
constexpr int outer_threads(int log2m, int mult) {
  return mult == 2 && 2 * fft_threads(log2m) <= 1024 ? 2 * fft_threads(log2m) : fft_threads(log2m);
}

template <int LOG2M>
int launch_outer(fcs_ctx *ctx, int64_t nbatch, int64_t L, int D, int64_t La, int64_t Lb,
                 const float *fa, const float *fb, float *out, int mult) {
  const int sb = int(((La > Lb ? La : Lb) + 3) / 4 * 4);
  auto go = [&](auto kern, int nt, size_t smem) -> int {
    if (smem > 48 * 1024) {
      cudaError_t e =
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(outer)");
    }
    kern<<<dim3(unsigned(D), unsigned(nbatch)), nt, smem, ctx->stream>>>(fa, fb, La, Lb, L, D, sb,
                                                                         out, ctx->twiddle);
    return check_cuda(ctx, cudaGetLastError(), "outer_kernel");
  };
  constexpr int NT1 = outer_threads(LOG2M, 1), NT2 = outer_threads(LOG2M, 2);
  if (mult == 2 && NT2 != NT1)
    return go(outer_kernel<LOG2M, NT2>, NT2, OuterSmem<LOG2M, NT2>::bytes(sb));
  return go(outer_kernel<LOG2M, NT1>, NT1, OuterSmem<LOG2M, NT1>::bytes(sb));
}

// Tuned thread multipliers, per (device, nbatch, slices, D, La, Lb); a shape
// not in the table uses multiplier 1.
std::mutex g_outer_mu;
std::map<std::tuple<int, int64_t, int64_t, int, int64_t, int64_t>, int> g_outer_tuned;

int outer_mult(int device, int64_t nbatch, int64_t L, int D, int64_t La, int64_t Lb) {
  std::lock_guard<std::mutex> lk(g_outer_mu);
  auto it = g_outer_tuned.find(std::make_tuple(device, nbatch, L, D, La, Lb));
  return it == g_outer_tuned.end() ? 1 : it->second;
}

}  // namespace
}  // namespace fcs

using namespace fcs;

namespace fcs {
namespace {

// Validate; *log2p = FFT length of the call.
int outer_check(fcs_ctx *ctx, int64_t nbatch, int64_t nslices, int D, int64_t La, int64_t Lb,
                const float *fa, const float *fb, float *out, int *log2p_out) {
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
  *log2p_out = log2p;
  return FCS_OK;
}

int sketch_outer_mult(fcs_ctx *ctx, int64_t nbatch, int64_t nslices, int D, int64_t La,
                      int64_t Lb, const float *fa, const float *fb, float *out, int log2p,
                      int mult) {
  const int64_t Lo = La + Lb - 1;
  DeviceGuard g(ctx->device);
  spec_cache_invalidate(ctx, out, sizeof(float) * size_t(nbatch) * D * size_t(Lo));
  if (log2p > kMaxLog2P) return big_outer(ctx, nbatch, nslices, D, La, Lb, fa, fb, out, log2p);
  int rc = FCS_EUNSUPPORTED;
  FCS_DISPATCH_LOG2M(log2p - 1,
                     rc = launch_outer<L>(ctx, nbatch, nslices, D, La, Lb, fa, fb, out, mult));
  return rc;
}

int sketch_outer(fcs_ctx *ctx, int64_t nbatch, int64_t nslices, int D, int64_t La, int64_t Lb,
                 const float *fa, const float *fb, float *out) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  int log2p = 0;
  int rc = outer_check(ctx, nbatch, nslices, D, La, Lb, fa, fb, out, &log2p);
  if (rc) return rc;
  return sketch_outer_mult(ctx, nbatch, nslices, D, La, Lb, fa, fb, out, log2p,
                           outer_mult(ctx->device, nbatch, nslices, D, La, Lb));
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

extern "C" int fcs_outer_autotune(fcs_ctx *ctx, int64_t nbatch, int64_t L, int D, int64_t La,
                                  int64_t Lb, const float *fa, const float *fb, float *out,
                                  int *host_threads) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  int log2p = 0;
  int rc = outer_check(ctx, nbatch, L, D, La, Lb, fa, fb, out, &log2p);
  if (rc) return rc;
  int best = 1;
  if (log2p <= kMaxLog2P && outer_threads(log2p - 1, 2) != outer_threads(log2p - 1, 1)) {
    DeviceGuard g(ctx->device);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      cudaGetLastError();
      if (e0) cudaEventDestroy(e0);
      return set_error(ctx, FCS_ECUDA, "cudaEventCreate");
    }
    float ms[2] = {0.f, 0.f};
    for (int m = 1; m <= 2 && rc == FCS_OK; ++m) {
      rc = sketch_outer_mult(ctx, nbatch, L, D, La, Lb, fa, fb, out, log2p, m);   // warm-up
      for (int rep = 0; rep < 5 && rc == FCS_OK; ++rep) {
        cudaEventRecord(e0, ctx->stream);
        rc = sketch_outer_mult(ctx, nbatch, L, D, La, Lb, fa, fb, out, log2p, m);
        cudaEventRecord(e1, ctx->stream);
        if (rc == FCS_OK) rc = check_cuda(ctx, cudaEventSynchronize(e1), "cudaEventSynchronize");
        float t = 0.f;
        if (rc == FCS_OK) cudaEventElapsedTime(&t, e0, e1);
        ms[m - 1] += t;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    best = ms[1] < 0.97f * ms[0] ? 2 : 1;   // a clear gain, not timing noise
  } else {
    // one shape only: run it once, so that `out` holds its result
    rc = sketch_outer_mult(ctx, nbatch, L, D, La, Lb, fa, fb, out, log2p, 1);
    if (rc) return rc;
  }
  {
    std::lock_guard<std::mutex> lk(g_outer_mu);
    g_outer_tuned[std::make_tuple(ctx->device, nbatch, L, D, La, Lb)] = best;
  }
  if (host_threads) *host_threads = log2p <= kMaxLog2P ? outer_threads(log2p - 1, best) : 0;
  return FCS_OK;
}
