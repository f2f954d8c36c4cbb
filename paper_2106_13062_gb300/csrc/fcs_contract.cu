// fcs_contract.cu -- fcs_contract: the sketched contractions of Sec. 4.1.
//
//  ALL  (eq. T_uvw):  e_d = <FCS_d(T), FCS_d(v_1 o ... o v_N)>
//       = (1/P) Re sum_{k<P} conj(F(FCS_d T))[k] prod_n F(CS_n v_n)[k]
//       (Parseval; FCS_d of the rank-1 tensor is the product of the per-mode
//       spectra by eq. FCS_syn with R = 1).
//  FREE (eq. T_Ivw, free mode m; also the ALS columns of Sec. 4.1.2):
//       z_d = IFFT(F(FCS_d T) prod_{n != m} conj F(CS_n v_n)),
//       est_d[i] = s_m(i) z_d[h_m(i)]   (exact for P >= Jt: the circular
//       correlation never wraps at the lags h_m(i) < J_m).
//  Then the median over the D sketches (Sec. 4 opening).
//
// Kernels: (1) the half spectra of the D sketches of T; (2) one CTA per
// (batch item, sketch) that builds each needed Count Sketch in shared memory,
// transforms it and folds it into the per-thread spectrum product, then either
// reduces the Parseval sum or runs the inverse FFT and gathers; (3) the median.
#include "fcs_internal.cuh"

namespace fcs {
namespace {

struct ContractArgs {
  Modes m;
  int D;
  int kind;
  int free_mode;
  int64_t B;
  const float *fcsT;      // [D][Jt]
  const float *vec[kMaxN];
  const int32_t *h;
  const int8_t *s;
  float2 *spec;           // [D][M+1]
  float *raw;             // [B][D] or [B][D][I_m]
  float *out;             // [B] or [B][I_m]
};

// Half spectrum of each of the D sketches of T, natural order [D][M+1].
template <int LOG2M, int NT>
__global__ void __launch_bounds__(NT) spectrum_kernel(const float *__restrict__ x, int64_t len,
                                                      int64_t ld, float2 *__restrict__ spec,
                                                      const float2 *__restrict__ tw) {
  constexpr int M = 1 << LOG2M;
  constexpr int HALF = M / 2;
  constexpr int EP = (HALF + NT - 1) / NT;
  extern __shared__ __align__(16) float2 buf[];
  float *bufr = reinterpret_cast<float *>(buf);
  const int tid = threadIdx.x;
  const float *xd = x + blockIdx.x * ld;
  for (int e = tid; e < padded_len(M); e += NT) buf[e] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int64_t j = tid; j < len; j += NT) bufr[real_off(int(j))] = __ldg(xd + j);
  __syncthreads();
  block_fft<LOG2M, NT>(buf, tw);
  float2 *sd = spec + blockIdx.x * int64_t(M + 1);
#pragma unroll
  for (int e = 0; e < EP; ++e) {
    const int q = tid + e * NT;
    if (q < HALF) {
      float2 A, B;
      unpack_pair<LOG2M>(buf, q, tw, A, B);
      if (q == 0) {
        sd[0] = make_float2(A.x, 0.f);
        sd[M] = make_float2(A.y, 0.f);
        sd[HALF] = B;
      } else {
        sd[q] = A;
        sd[M - q] = B;
      }
    }
  }
}

template <int LOG2M, int NT>
__global__ void __launch_bounds__(NT) contract_kernel(ContractArgs a,
                                                      const float2 *__restrict__ tw) {
  constexpr int M = 1 << LOG2M;
  constexpr int HALF = M / 2;
  constexpr int EP = (HALF + NT - 1) / NT;
  extern __shared__ __align__(16) float2 buf[];
  float *bufr = reinterpret_cast<float *>(buf);
  __shared__ float red[NT / 32];
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x;
  const int d = blockIdx.y;
  const bool all = a.kind == FCS_CONTRACT_ALL;
  const float2 *sd = a.spec + d * int64_t(M + 1);

  // sketch-of-T spectrum slots for this thread's pairs
  float2 FA[EP], FB[EP], pA[EP], pB[EP];
#pragma unroll
  for (int e = 0; e < EP; ++e) {
    const int q = tid + e * NT;
    FA[e] = FB[e] = make_float2(0.f, 0.f);
    if (q < HALF) {
      if (q == 0) {
        FA[e] = make_float2(sd[0].x, sd[M].x);
        FB[e] = sd[HALF];
      } else {
        FA[e] = sd[q];
        FB[e] = sd[M - q];
      }
    }
    // multiplicative identity: slot A of pair 0 packs two reals
    pA[e] = all ? make_float2(1.f, q == 0 ? 1.f : 0.f) : FA[e];
    pB[e] = all ? make_float2(1.f, 0.f) : FB[e];
  }

  for (int n = 0; n < a.m.N; ++n) {
    if (!all && n == a.free_mode) continue;
    for (int e = tid; e < padded_len(M); e += NT) buf[e] = make_float2(0.f, 0.f);
    __syncthreads();
    const int32_t *hn = a.h + d * a.m.ldh + a.m.off[n];
    const int8_t *sn = a.s + d * a.m.ldh + a.m.off[n];
    const float *vn = a.vec[n] + b * a.m.I[n];
    for (int64_t i = tid; i < a.m.I[n]; i += NT) {
      float v = __ldg(vn + i);
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
        float2 A, Bv;
        unpack_pair<LOG2M>(buf, q, tw, A, Bv);
        if (all) {
          pA[e] = slot_mul(pA[e], A, q == 0);
          pB[e] = cmul(pB[e], Bv);
        } else {
          pA[e] = slot_mulconj(pA[e], A, q == 0);
          pB[e] = cmulconj(pB[e], Bv);
        }
      }
    }
    __syncthreads();
  }

  if (all) {
    // sum_{k<P} conj(F_T[k]) Y[k] = F_T[0]Y[0] + F_T[M]Y[M] + 2 sum_{0<k<M} Re(..)
    float part = 0.f;
#pragma unroll
    for (int e = 0; e < EP; ++e) {
      const int q = tid + e * NT;
      if (q < HALF) {
        const float wa = (q == 0) ? 1.f : 2.f;
        part += wa * (FA[e].x * pA[e].x + FA[e].y * pA[e].y);
        part += 2.f * (FB[e].x * pB[e].x + FB[e].y * pB[e].y);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int w = 0; w < NT / 32; ++w) t += red[w];
      a.raw[b * a.D + d] = t / float(2 * M);
    }
    return;
  }

  // FREE: inverse transform of the product, then gather at h_m(i)
#pragma unroll
  for (int e = 0; e < EP; ++e) {
    const int q = tid + e * NT;
    if (q < HALF) pack_pair_conj<LOG2M>(buf, q, pA[e], pB[e], tw);
  }
  __syncthreads();
  block_fft<LOG2M, NT>(buf, tw);
  const int m = a.free_mode;
  const int32_t *hm = a.h + d * a.m.ldh + a.m.off[m];
  const int8_t *sm = a.s + d * a.m.ldh + a.m.off[m];
  const int64_t Im = a.m.I[m];
  float *rawbd = a.raw + (b * a.D + d) * Im;
  const float sc = 1.0f / float(M);
  for (int64_t i = tid; i < Im; i += NT) {
    const int p = __ldg(hm + i);
    const float v = unsigned(p) < unsigned(2 * M) ? bufr[real_off(p)] : __int_as_float(0x7fc00000);
    const float z = (p & 1) ? -v * sc : v * sc;
    rawbd[i] = __ldg(sm + i) < 0 ? -z : z;
  }
}

template <int D>
__global__ void median_kernel(const float *__restrict__ raw, int64_t B, int64_t width,
                              float *__restrict__ out) {
  // raw [B][D][width] -> out [B][width]
  const int64_t total = B * width;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = t / width, i = t - b * width;
    float v[D];
#pragma unroll
    for (int d = 0; d < D; ++d) v[d] = raw[(b * D + d) * width + i];
    out[t] = median_inplace<D>(v);
  }
}

template <int LOG2M>
int launch_contract(fcs_ctx *ctx, ContractArgs &a, int64_t Jt) {
  constexpr int NT = fft_threads(LOG2M);
  const size_t smem = sizeof(float2) * padded_len(1 << LOG2M);
  auto k1 = spectrum_kernel<LOG2M, NT>;
  auto k2 = contract_kernel<LOG2M, NT>;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(contract)");
  }
  k1<<<a.D, NT, smem, ctx->stream>>>(a.fcsT, Jt, Jt, a.spec, ctx->twiddle);
  int rc = check_cuda(ctx, cudaGetLastError(), "spectrum_kernel");
  if (rc) return rc;
  k2<<<dim3(unsigned(a.B), unsigned(a.D)), NT, smem, ctx->stream>>>(a, ctx->twiddle);
  return check_cuda(ctx, cudaGetLastError(), "contract_kernel");
}

int launch_median(fcs_ctx *ctx, int D, const float *raw, int64_t B, int64_t width,
                  float *out) {
  const int64_t total = B * width;
  int blocks = int((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  switch (D) {
#define FCS_MED_CASE(K) \
  case K: median_kernel<K><<<blocks, 256, 0, ctx->stream>>>(raw, B, width, out); break;
    FCS_MED_CASE(1) FCS_MED_CASE(2) FCS_MED_CASE(3) FCS_MED_CASE(4) FCS_MED_CASE(5)
    FCS_MED_CASE(6) FCS_MED_CASE(7) FCS_MED_CASE(8) FCS_MED_CASE(9) FCS_MED_CASE(10)
    FCS_MED_CASE(11) FCS_MED_CASE(12) FCS_MED_CASE(13) FCS_MED_CASE(14) FCS_MED_CASE(15)
    FCS_MED_CASE(16)
#undef FCS_MED_CASE
    default:
      return set_error(ctx, FCS_EINVAL, "D=%d outside [1,16]", D);
  }
  return check_cuda(ctx, cudaGetLastError(), "median_kernel");
}

}  // namespace
}  // namespace fcs

using namespace fcs;

extern "C" int fcs_contract(fcs_ctx *ctx, int kind, int free_mode, int N,
                            const int64_t *host_I, const int32_t *host_J, int D,
                            const float *fcsT, int64_t B, const float *const *host_vecs,
                            const int32_t *h, const int8_t *s, int64_t ldh,
                            float *out_median, float *out_raw) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  ContractArgs a{};
  int rc = make_modes(ctx, N, host_I, host_J, ldh, &a.m);
  if (rc) return rc;
  if (kind != FCS_CONTRACT_ALL && kind != FCS_CONTRACT_FREE)
    return set_error(ctx, FCS_EINVAL, "unknown contraction kind %d", kind);
  if (kind == FCS_CONTRACT_FREE && (free_mode < 0 || free_mode >= N))
    return set_error(ctx, FCS_EINVAL, "free_mode=%d outside [0,%d)", free_mode, N);
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (B < 1 || B > 65535) return set_error(ctx, FCS_EINVAL, "B=%lld outside [1,65535]", (long long)B);
  if (!fcsT || !host_vecs || !h || !s || !out_median)
    return set_error(ctx, FCS_EINVAL, "NULL pointer argument");
  for (int n = 0; n < N; ++n) {
    if (kind == FCS_CONTRACT_FREE && n == free_mode) {
      a.vec[n] = nullptr;
      continue;
    }
    if (!host_vecs[n]) return set_error(ctx, FCS_EINVAL, "vector %d is NULL", n);
    a.vec[n] = host_vecs[n];
  }
  const int log2p = ilog2_ceil(a.m.Jt) < kMinLog2P ? kMinLog2P : ilog2_ceil(a.m.Jt);
  if (log2p > kMaxLog2P)
    return set_error(ctx, FCS_EUNSUPPORTED, "Jt=%lld needs FFT length > %d",
                     (long long)a.m.Jt, 1 << kMaxLog2P);
  const int log2m = log2p - 1;
  const int M = 1 << log2m;
  a.D = D;
  a.kind = kind;
  a.free_mode = free_mode;
  a.B = B;
  a.fcsT = fcsT;
  a.h = h;
  a.s = s;
  a.out = out_median;
  const int64_t width = kind == FCS_CONTRACT_ALL ? 1 : host_I[free_mode];
  const size_t sbytes = (sizeof(float2) * size_t(D) * size_t(M + 1) + 255) & ~size_t(255);
  const size_t rbytes = out_raw ? 0 : sizeof(float) * size_t(B) * D * size_t(width);
  void *ws = nullptr;
  rc = ensure_workspace(ctx, sbytes + rbytes, &ws);
  if (rc) return rc;
  a.spec = static_cast<float2 *>(ws);
  a.raw = out_raw ? out_raw : reinterpret_cast<float *>(static_cast<char *>(ws) + sbytes);
  DeviceGuard g(ctx->device);
  rc = FCS_EUNSUPPORTED;
  FCS_DISPATCH_LOG2M(log2m, rc = launch_contract<L>(ctx, a, a.m.Jt));
  if (rc) return rc;
  return launch_median(ctx, D, a.raw, B, width, out_median);
}
