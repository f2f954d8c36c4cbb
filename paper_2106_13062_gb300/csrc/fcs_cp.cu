// fcs_cp.cu -- fcs_sketch_cp: FCS of a CP tensor by eq. (FCS_syn):
//   FCS(T) = sum_r lambda_r IFFT( prod_n FFT_P( CS_n(U_n(:, r)) ) ),
// with P the smallest power of two >= Jt (any P >= Jt gives the exact linear
// convolution, so out = the first Jt samples).
//
// One fused kernel.  CTA (g, d) owns sketch d and a contiguous group of
// ranks.  For each rank and mode it scatters the signed factor column into a
// zeroed shared-memory buffer (the Count Sketch of Def. 1), runs a block-wide
// real FFT of length P (a complex FFT of length P/2 plus the pair unpack),
// and multiplies the half spectrum into per-thread registers; after the last
// mode it adds lambda_r times the product into a per-thread accumulator.  The
// rank sum therefore stays in the frequency domain (linearity moves the
// paper's sum of inverse transforms inside one inverse transform).  Each CTA
// adds its partial spectrum into a global accumulator with atomics; the last
// CTA to finish for sketch d (ticket counter) runs the single inverse real FFT
// and writes FCS_d.
#include "fcs_internal.cuh"

namespace fcs {
namespace {

struct CpArgs {
  Modes m;
  int D;
  int64_t R;
  int64_t ranks_per_cta;
  const float *U[kMaxN];
  int64_t ldU[kMaxN];
  const float *lambda;
  const int32_t *h;
  const int8_t *s;
  float2 *G;             // [D][M+1] spectrum accumulator, zeroed per call
  unsigned *counter;     // [D] tickets, zero at launch, reset by the last CTA
  float *out;            // [D][Jt]
};

template <int LOG2M, int NT>
__global__ void __launch_bounds__(NT) cp_kernel(CpArgs a, const float2 *__restrict__ tw) {
  constexpr int M = 1 << LOG2M;
  constexpr int HALF = M / 2;
  constexpr int EP = (HALF + NT - 1) / NT;
  extern __shared__ __align__(16) float2 buf[];
  float *bufr = reinterpret_cast<float *>(buf);
  __shared__ int is_last;
  const int tid = threadIdx.x;
  const int d = blockIdx.y;
  const int64_t r0 = blockIdx.x * a.ranks_per_cta;
  const int64_t r1 = min(a.R, r0 + a.ranks_per_cta);

  float2 accA[EP], accB[EP], pA[EP], pB[EP];
#pragma unroll
  for (int e = 0; e < EP; ++e) {
    accA[e] = accB[e] = make_float2(0.f, 0.f);
    pA[e] = pB[e] = make_float2(0.f, 0.f);
  }

  for (int64_t r = r0; r < r1; ++r) {
    for (int n = 0; n < a.m.N; ++n) {
      for (int e = tid; e < padded_len(M); e += NT) buf[e] = make_float2(0.f, 0.f);
      __syncthreads();
      const int32_t *hn = a.h + d * a.m.ldh + a.m.off[n];
      const int8_t *sn = a.s + d * a.m.ldh + a.m.off[n];
      const float *Un = a.U[n];
      const int64_t ld = a.ldU[n];
      for (int64_t i = tid; i < a.m.I[n]; i += NT) {
        float v = __ldg(Un + i * ld + r);
        if (__ldg(sn + i) < 0) v = -v;
        const int p = __ldg(hn + i);
        if (unsigned(p) < unsigned(2 * M)) atomicAdd(bufr + real_off(p), v);
      }
      __syncthreads();
      block_fft<LOG2M, NT>(buf, tw);
#pragma unroll
      for (int e = 0; e < EP; ++e) {
        const int q = tid + e * NT;
        if (q < HALF) {
          float2 A, B;
          unpack_pair<LOG2M>(buf, q, tw, A, B);
          if (n == 0) {
            pA[e] = A;
            pB[e] = B;
          } else {
            pA[e] = slot_mul(pA[e], A, q == 0);
            pB[e] = cmul(pB[e], B);
          }
        }
      }
      __syncthreads();
    }
    const float lam = a.lambda ? __ldg(a.lambda + r) : 1.f;
#pragma unroll
    for (int e = 0; e < EP; ++e) {
      accA[e].x = fmaf(lam, pA[e].x, accA[e].x);
      accA[e].y = fmaf(lam, pA[e].y, accA[e].y);
      accB[e].x = fmaf(lam, pB[e].x, accB[e].x);
      accB[e].y = fmaf(lam, pB[e].y, accB[e].y);
    }
  }

  // publish the partial spectrum
  float2 *Gd = a.G + d * int64_t(M + 1);
#pragma unroll
  for (int e = 0; e < EP; ++e) {
    const int q = tid + e * NT;
    if (q < HALF) {
      if (q == 0) {
        atomicAdd(&Gd[0].x, accA[e].x);
        atomicAdd(&Gd[M].x, accA[e].y);
        atomicAdd(&Gd[HALF].x, accB[e].x);
        atomicAdd(&Gd[HALF].y, accB[e].y);
      } else {
        atomicAdd(&Gd[q].x, accA[e].x);
        atomicAdd(&Gd[q].y, accA[e].y);
        atomicAdd(&Gd[M - q].x, accB[e].x);
        atomicAdd(&Gd[M - q].y, accB[e].y);
      }
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = (atomicAdd(&a.counter[d], 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  // last CTA for sketch d: one inverse real FFT of the summed spectrum
#pragma unroll
  for (int e = 0; e < EP; ++e) {
    const int q = tid + e * NT;
    if (q < HALF) {
      float2 A, B;
      if (q == 0) {
        A = make_float2(__ldcg(&Gd[0].x), __ldcg(&Gd[M].x));
        B = __ldcg(&Gd[HALF]);
      } else {
        A = __ldcg(&Gd[q]);
        B = __ldcg(&Gd[M - q]);
      }
      pack_pair_conj<LOG2M>(buf, q, A, B, tw);
    }
  }
  __syncthreads();
  block_fft<LOG2M, NT>(buf, tw);
  const float sc = 1.0f / float(M);
  float *od = a.out + d * a.m.Jt;
  for (int64_t j = tid; j < a.m.Jt; j += NT) {
    const float v = bufr[real_off(int(j))];
    od[j] = (j & 1) ? -v * sc : v * sc;
  }
  if (tid == 0) a.counter[d] = 0u;
}

template <int LOG2M>
int launch_cp(fcs_ctx *ctx, CpArgs &a, int64_t groups) {
  constexpr int NT = fft_threads(LOG2M);
  const size_t smem = sizeof(float2) * padded_len(1 << LOG2M);
  auto kern = cp_kernel<LOG2M, NT>;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(cp)");
  }
  kern<<<dim3(unsigned(groups), unsigned(a.D)), NT, smem, ctx->stream>>>(a, ctx->twiddle);
  return check_cuda(ctx, cudaGetLastError(), "cp_kernel");
}

}  // namespace
}  // namespace fcs

using namespace fcs;

extern "C" int fcs_sketch_cp(fcs_ctx *ctx, int N, const int64_t *host_I,
                             const int32_t *host_J, int64_t R, int D,
                             const float *const *host_U, const int64_t *host_ldU,
                             const float *lambda, const int32_t *h, const int8_t *s,
                             int64_t ldh, float *out) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  CpArgs a{};
  int rc = make_modes(ctx, N, host_I, host_J, ldh, &a.m);
  if (rc) return rc;
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (R < 1) return set_error(ctx, FCS_EINVAL, "R=%lld must be >= 1", (long long)R);
  if (!host_U || !host_ldU || !h || !s || !out)
    return set_error(ctx, FCS_EINVAL, "NULL pointer argument");
  for (int n = 0; n < N; ++n) {
    if (!host_U[n]) return set_error(ctx, FCS_EINVAL, "U[%d] is NULL", n);
    if (host_ldU[n] < R)
      return set_error(ctx, FCS_EINVAL, "ldU[%d]=%lld < R", n, (long long)host_ldU[n]);
    a.U[n] = host_U[n];
    a.ldU[n] = host_ldU[n];
  }
  const int log2p = ilog2_ceil(a.m.Jt) < kMinLog2P ? kMinLog2P : ilog2_ceil(a.m.Jt);
  if (log2p > kMaxLog2P)
    return set_error(ctx, FCS_EUNSUPPORTED, "Jt=%lld needs FFT length > %d",
                     (long long)a.m.Jt, 1 << kMaxLog2P);
  const int log2m = log2p - 1;
  const int M = 1 << log2m;
  a.D = D;
  a.R = R;
  a.lambda = lambda;
  a.h = h;
  a.s = s;
  a.out = out;
  // rank groups: about one CTA per SM over all sketches
  int64_t groups = (int64_t(ctx->sm_count) + D - 1) / D;
  if (groups < 1) groups = 1;
  if (groups > R) groups = R;
  a.ranks_per_cta = (R + groups - 1) / groups;
  groups = (R + a.ranks_per_cta - 1) / a.ranks_per_cta;

  const size_t gbytes = sizeof(float2) * size_t(D) * size_t(M + 1);
  void *ws = nullptr;
  rc = ensure_workspace(ctx, gbytes + 64 * sizeof(unsigned), &ws);
  if (rc) return rc;
  a.G = static_cast<float2 *>(ws);
  a.counter = reinterpret_cast<unsigned *>(static_cast<char *>(ws) + gbytes);
  DeviceGuard g(ctx->device);
  rc = check_cuda(ctx, cudaMemsetAsync(ws, 0, gbytes + 64 * sizeof(unsigned), ctx->stream),
                  "cudaMemsetAsync(cp workspace)");
  if (rc) return rc;
  rc = FCS_EUNSUPPORTED;
  FCS_DISPATCH_LOG2M(log2m, rc = launch_cp<L>(ctx, a, groups));
  return rc;
}
