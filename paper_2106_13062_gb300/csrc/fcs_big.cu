// fcs_big.cu -- the FFT-based calls for long sketches, 16384 < P <= 2^20
// (Jt up to 2^20): the CP-route sketch (eq. FCS_syn), the contractions
// (eqs. T_uvw, T_Ivw) and the outer-product combine, for FFT lengths beyond
// what one CTA holds in shared memory.
//
// Complex FFT of length M = P/2 = M1 * 2^14 (M1 = 1..32), decimation in time:
//   Z[q2 + 2^14 q1] = sum_{m1} W_M1^(m1 q1) W_M^(m1 q2) Y_m1[q2],
//   Y_m1 = FFT_{2^14}(z[m1 + M1 m2]),
// pass 1: one CTA per (transform, m1) loads the strided sub-sequence into
// shared memory and runs the block FFT of fcs_internal.cuh; pass 2: one
// thread per (transform, q2) applies the twiddles and the M1-point DFT in
// registers, in place (it reads and writes the same M1 addresses), with
// coalesced accesses across threads.  Twiddles W_P^k for P > 2^15 are a
// table entry times a fine factor W_P^j, j < P / 2^15, computed per CTA.
//
// The real transforms are the same packed-complex ones as the in-CTA path:
// z[m] = x[2m] + i x[2m+1], half spectrum unpacked pairwise (q, M - q); the
// inverse packs conj(Z) from the half spectrum, transforms forward, and
// conjugates and scales by 1/M.  Everything between transforms (Count
// Sketches, mode products, rank sums, Parseval sums, gathers) runs in the
// route kernels below; intermediate arrays live in the context workspace,
// processed in chunks of transforms that fit it.
#include <algorithm>

#include "fcs_fft.cuh"

namespace fcs {
namespace {

constexpr int kL2 = 14;                 // pass-1 FFT length 2^14
constexpr int kM2 = 1 << kL2;
constexpr int kNT1 = 1024;              // = fft_threads(14)
constexpr int kNT2 = 256;
constexpr int kMaxFine = 1 << (kMaxLog2PBig - kLogTwN);
constexpr size_t kBigWorkspaceCap = size_t(512) << 20;

// W_P^k for P = 2^lp (k < P): a global-table entry times a fine factor.
struct BigTw {
  const float2 *tw;
  const float2 *fine;   // W_P^j, j < 2^(lp - 15); unused for lp <= 15
  int lp;
  __device__ __forceinline__ float2 operator()(int64_t k) const {
    if (lp <= kLogTwN) return __ldg(&tw[k << (kLogTwN - lp)]);
    const int s = lp - kLogTwN;
    return cmul(__ldg(&tw[k >> s]), fine[k & ((int64_t(1) << s) - 1)]);
  }
};

// Fine factors W_P^j, evaluated in FP64 and rounded; all threads call it.
__device__ __forceinline__ void fill_fine(float2 *fine, int lp) {
  const int n = lp > kLogTwN ? 1 << (lp - kLogTwN) : 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * double(j) / double(int64_t(1) << lp), &sn, &cs);
    fine[j] = make_float2(float(cs), float(-sn));
  }
}

// ---------------------------------------------------------------- FFT passes
// Pass 1.  Transform t reads the real sequence src + t * src_ld (len_t
// floats, zero past them; len_t = lens[t % nlens]) as z[m] = x[2m] + i x[2m+1]
// and writes Y_m1 (natural order) to dst + t * M + m1 * 2^14.
struct Pass1Args {
  const float *src;
  int64_t src_ld;
  int nlens;
  int64_t lens[kMaxN];
  float2 *dst;
  int L1;
};

__global__ void __launch_bounds__(kNT1) pass1_kernel(Pass1Args a, const float2 *__restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2 *B = reinterpret_cast<float2 *>(smem);
  const int m1 = blockIdx.x;
  const int64_t t = blockIdx.y;
  const int64_t M1 = int64_t(1) << a.L1;
  const int64_t len = a.lens[t % a.nlens];
  const float *x = a.src + t * a.src_ld;
#pragma unroll
  for (int m2 = threadIdx.x; m2 < kM2; m2 += kNT1) {
    const int64_t m = m1 + M1 * m2;
    const float re = 2 * m < len ? __ldg(x + 2 * m) : 0.f;
    const float im = 2 * m + 1 < len ? __ldg(x + 2 * m + 1) : 0.f;
    B[pad(m2)] = make_float2(re, im);
  }
  __syncthreads();
  block_fft<kL2, kNT1>(B, tw);
  float2 *y = a.dst + t * (M1 << kL2) + int64_t(m1) * kM2;
#pragma unroll
  for (int q = threadIdx.x; q < kM2; q += kNT1) y[q] = B[pad(q)];
}

// Pass 2 (M1 = 2^L1 >= 2), in place on Y: Z[q2 + 2^14 q1].
template <int L1>
__global__ void __launch_bounds__(kNT2) pass2_kernel(float2 *Y, const float2 *__restrict__ tw) {
  constexpr int M1 = 1 << L1;
  constexpr int lp = kL2 + L1 + 1;                   // P = 2M
  __shared__ float2 fine[kMaxFine];
  fill_fine(fine, lp);
  __syncthreads();
  const BigTw W{tw, fine, lp};
  const int q2 = blockIdx.x * kNT2 + threadIdx.x;
  float2 *y = Y + int64_t(blockIdx.y) * (int64_t(M1) << kL2) + q2;
  float2 v[M1];
#pragma unroll
  for (int m1 = 0; m1 < M1; ++m1) v[m1] = y[int64_t(m1) * kM2];
  float2 wp[L1];                                     // W_M^(q2 2^b) = W_P^(2 q2 2^b)
#pragma unroll
  for (int b = 0; b < L1; ++b) wp[b] = W((int64_t(2) * q2) << b);
  twiddle_powers<L1>(v, wp);
  Dft<M1>::run(v);
#pragma unroll
  for (int q1 = 0; q1 < M1; ++q1) y[int64_t(q1) * kM2] = v[q1];
}

// Complex FFTs of length M = 2^(14 + L1) of T transforms: real inputs as in
// Pass1Args, result Z in `work` ([T][M] float2, natural order).
int big_fft(fcs_ctx *ctx, const Pass1Args &a0, int64_t T, float2 *work) {
  Pass1Args a = a0;
  a.dst = work;
  const size_t smem = sizeof(float2) * padded_len(kM2);
  cudaError_t e = cudaFuncSetAttribute(pass1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem));
  if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(pass1)");
  for (int64_t t0 = 0; t0 < T; t0 += 65535) {
    const int64_t nt = std::min<int64_t>(65535, T - t0);
    Pass1Args b = a;
    b.src = a.src + t0 * a.src_ld;
    b.dst = work + t0 * (int64_t(1) << (kL2 + a.L1));
    // lens are indexed by t % nlens; keep the phase when splitting
    if (a.nlens > 1) {
      for (int k = 0; k < a.nlens; ++k) b.lens[k] = a.lens[(t0 + k) % a.nlens];
    }
    pass1_kernel<<<dim3(1u << a.L1, unsigned(nt)), kNT1, smem, ctx->stream>>>(b, ctx->twiddle);
    int rc = check_cuda(ctx, cudaGetLastError(), "pass1_kernel");
    if (rc) return rc;
    if (a.L1 == 0) continue;
    float2 *y = b.dst;
    const dim3 g2(kM2 / kNT2, unsigned(nt));
    switch (a.L1) {
      case 1: pass2_kernel<1><<<g2, kNT2, 0, ctx->stream>>>(y, ctx->twiddle); break;
      case 2: pass2_kernel<2><<<g2, kNT2, 0, ctx->stream>>>(y, ctx->twiddle); break;
      case 3: pass2_kernel<3><<<g2, kNT2, 0, ctx->stream>>>(y, ctx->twiddle); break;
      case 4: pass2_kernel<4><<<g2, kNT2, 0, ctx->stream>>>(y, ctx->twiddle); break;
      case 5: pass2_kernel<5><<<g2, kNT2, 0, ctx->stream>>>(y, ctx->twiddle); break;
      default: return set_error(ctx, FCS_EUNSUPPORTED, "FFT length beyond 2^20");
    }
    rc = check_cuda(ctx, cudaGetLastError(), "pass2_kernel");
    if (rc) return rc;
  }
  return FCS_OK;
}

// ---------------------------------------------------------------- real-FFT glue
// Half-spectrum value of the real input of Z at bin k in [0, M] from the
// packed transform Z (pair helpers of fcs_internal.cuh).
__device__ __forceinline__ void half_pair(const float2 *Z, int64_t M, int64_t j,
                                          const BigTw &W, float2 &xa, float2 &xb) {
  // j in [0, M/2]: bins (j, M - j); j = 0 gives (X[0], X[M]) as two reals in
  // xa = (X[0], X[M]); j = M/2 gives xa = xb = X[M/2]
  if (j == 0) {
    const float2 z0 = Z[0];
    xa = make_float2(z0.x + z0.y, z0.x - z0.y);
    xb = xa;
  } else if (2 * j == M) {
    xa = xb = cconj(Z[j]);
  } else {
    unpack2(Z[j], Z[M - j], W(j), xa, xb);
  }
}

// Write the conj-packed inverse input (see pack_pair_conj) for the pair j of
// a half spectrum: xa = X[j], xb = X[M - j]; j = 0 carries (X[0], X[M]) in xa
// and writes position 0; j = M/2 writes position M/2 (X[M/2] itself).
__device__ __forceinline__ void store_packed_pair(float2 *zt, int64_t M, int64_t j, float2 xa,
                                                  float2 xb, const BigTw &W) {
  float2 cq, cm;
  if (j == 0) {
    pack_pair_conj_values_w(0, xa, xb, make_float2(1.f, 0.f), cq, cm);
    zt[0] = cq;
  } else if (2 * j == M) {
    zt[j] = xa;
  } else {
    pack_pair_conj_values_w(1, xa, xb, W(j), cq, cm);
    zt[j] = cq;
    zt[M - j] = cm;
  }
}

// Pair product with the packed-reals convention at j = 0.
__device__ __forceinline__ float2 pmul(float2 a, float2 b, bool packed) {
  return slot_mul(a, b, packed);
}
__device__ __forceinline__ float2 pmulconj(float2 a, float2 b, bool packed) {
  return slot_mulconj(a, b, packed);
}

// Scatter a Count Sketch: one CTA per transform, which first clears the
// first Jn floats of its row, then adds s(i) * w * vals[i * vstride] at h(i).
struct CsArgs {
  float *x;
  int64_t x_ld;                 // floats per transform
  int N;                        // transforms cycle over the modes listed in mode[]
  int nmode;
  int mode[kMaxN];
  Modes m;
  const int32_t *h;
  const int8_t *s;
  // value source: CP factor columns (U != null) or batch vectors
  const float *U[kMaxN];
  int64_t ldU[kMaxN];
  const float *lambda;
  int64_t R;
  const float *vec[kMaxN];
  int D;
  int64_t first;                // global index of transform 0 of this launch
};

// Transform g (global index) -> (outer item, sketch d, mode n):
//   CP:       g = ((d * R + r) * nmode + k), mode n = mode[k]
//   vectors:  g = ((b * D + d) * nmode + k)
__global__ void cs_kernel(CsArgs a) {
  const int64_t lt = blockIdx.x;
  const int64_t g = a.first + lt;
  const int k = int(g % a.nmode);
  const int64_t pair = g / a.nmode;
  const int n = a.mode[k];
  const int64_t In = a.m.I[n];
  const int Jn = a.m.J[n];
  float *x = a.x + lt * a.x_ld;
  for (int64_t j = threadIdx.x; j < Jn; j += blockDim.x) x[j] = 0.f;
  __syncthreads();
  int d;
  const float *src;
  int64_t stride;
  float w = 1.f;
  if (a.U[0]) {
    d = int(pair / a.R);
    const int64_t r = pair - int64_t(d) * a.R;
    src = a.U[n] + r;
    stride = a.ldU[n];
    if (n == 0 && a.lambda) w = __ldg(a.lambda + r);
  } else {
    d = int(pair % a.D);
    const int64_t b = pair / a.D;
    src = a.vec[n] + b * In;
    stride = 1;
  }
  const int32_t *hn = a.h + d * a.m.ldh + a.m.off[n];
  const int8_t *sn = a.s + d * a.m.ldh + a.m.off[n];
  for (int64_t i = threadIdx.x; i < In; i += blockDim.x) {
    const int hb = __ldg(hn + i);
    float v = __ldg(src + i * stride) * w;
    if (__ldg(sn + i) < 0) v = -v;
    if (unsigned(hb) < unsigned(Jn)) atomicAdd(x + hb, v);
  }
}

// ---------------------------------------------------------------- CP route
// G[d][k] += sum over the chunk's ranks of prod_n X_{d,n,r}[k] for the pairs
// (j, M - j) owned by each thread.  Z holds the chunk's transforms
// [(d*R + r) * N + n] - first.
__global__ void cp_accum_kernel(const float2 *__restrict__ Z, int64_t first, int64_t last,
                                int N, int64_t R, int64_t M, float2 *__restrict__ G, int lp,
                                const float2 *__restrict__ tw) {
  __shared__ float2 fine[kMaxFine];
  fill_fine(fine, lp);
  __syncthreads();
  const BigTw W{tw, fine, lp};
  const int d = blockIdx.y;
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j > M / 2) return;
  const int64_t p0 = std::max<int64_t>(first / N, int64_t(d) * R);
  const int64_t p1 = std::min<int64_t>(last / N, int64_t(d + 1) * R);
  if (p0 >= p1) return;
  const bool packed = j == 0;
  float2 sa = make_float2(0.f, 0.f), sb = sa;
  for (int64_t p = p0; p < p1; ++p) {
    float2 pa = make_float2(1.f, packed ? 1.f : 0.f), pb = pa;
    for (int n = 0; n < N; ++n) {
      const float2 *Zt = Z + (p * N + n - first) * M;
      float2 xa, xb;
      half_pair(Zt, M, j, W, xa, xb);
      pa = pmul(pa, xa, packed);
      pb = pmul(pb, xb, false);
    }
    sa = cadd(sa, pa);
    sb = cadd(sb, pb);
  }
  float2 *Gd = G + int64_t(d) * (M + 1);
  if (packed) {
    Gd[0].x += sa.x;
    Gd[M].x += sa.y;
  } else {
    Gd[j] = cadd(Gd[j], sa);
    if (2 * j != M) Gd[M - j] = cadd(Gd[M - j], sb);
  }
}

// conj-packed sequence for the inverse of the half spectra S [T][M+1] (row
// stride sld), written as complex rows [T][M] of z (the forward FFT of z,
// conjugated and scaled by 1/M, is the real inverse).
__global__ void pack_inverse_kernel(const float2 *__restrict__ S, int64_t sld, int64_t M,
                                    float2 *__restrict__ z, int lp, const float2 *__restrict__ tw) {
  __shared__ float2 fine[kMaxFine];
  fill_fine(fine, lp);
  __syncthreads();
  const BigTw W{tw, fine, lp};
  const int64_t t = blockIdx.y;
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= M / 2) return;
  const float2 *s = S + t * sld;
  float2 A, Bv;
  if (q == 0) {
    A = make_float2(s[0].x, s[M].x);
    Bv = s[M / 2];
  } else {
    A = s[q];
    Bv = s[M - q];
  }
  float2 cq, cm;
  pack_pair_conj_values_w(int(q == 0 ? 0 : 1), A, Bv, q ? W(q) : make_float2(1.f, 0.f), cq, cm);
  float2 *zt = z + t * M;
  zt[q] = cq;
  zt[q ? M - q : M / 2] = cm;
}

// out[t][p] = x[p] for p < len: x[2m] = Re Z[m] * sc, x[2m+1] = -Im Z[m] * sc.
__global__ void unpack_real_kernel(const float2 *__restrict__ Z, int64_t M, float sc,
                                   float *__restrict__ out, int64_t out_ld, int64_t len) {
  const int64_t t = blockIdx.y;
  const float2 *zt = Z + t * M;
  float *o = out + t * out_ld;
  for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < len;
       p += int64_t(gridDim.x) * blockDim.x) {
    const float2 v = zt[p >> 1];
    o[p] = (p & 1) ? -v.y * sc : v.x * sc;
  }
}

// ---------------------------------------------------------------- P = 2^15
// The CP route for P = 2^15 (M = 2^14: one block FFT per transform) in one
// kernel, with nothing but the running products leaving the SM.  An item is
// (sketch d, rank group g); a CTA takes items blockIdx.x, + gridDim.x, ...
// For every rank r of its group and every mode n it scatters the Count
// Sketch of column r of U_n (times lambda_r on mode 0) into shared memory,
// transforms it, and multiplies the half spectrum into the running product
// of rank r, which lives in the CTA's own slice of `prod` (pair q holds
// slots A and B, the unpack_pair convention); after the last mode the
// product is added to G_d with atomics.  The CTA that completes the last
// group of sketch d (ticket counter) runs the inverse real FFT of G_d and
// writes FCS_d.  Nothing waits on another CTA.
struct Cp15Args {
  Modes m;
  int64_t R;
  int D;
  int groups;                 // rank groups per sketch
  const float *U[kMaxN];
  int64_t ldU[kMaxN];
  const float *lambda;
  const int32_t *h;
  const int8_t *s;
  float2 *G;                  // [D][M + 1] half spectra, zero at start
  unsigned *ticket;           // [D], zero at start; the last group resets it
  float4 *prod;               // [gridDim.x][M / 2] running products
  float *out;                 // [D][Jt]
};

__global__ void __launch_bounds__(kNT1) cp15_kernel(Cp15Args a, const float2 *__restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int is_last;
  constexpr int M = kM2, HALF = M / 2, PAIRS = HALF / kNT1;
  float2 *B = reinterpret_cast<float2 *>(smem);
  float *Bf = reinterpret_cast<float *>(smem);
  float4 *B4 = reinterpret_cast<float4 *>(smem);
  const int tid = threadIdx.x;
  const int N = a.m.N;
  float4 *prod = a.prod + int64_t(blockIdx.x) * HALF;
  const int items = a.D * a.groups;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int d = item / a.groups, g = item - d * a.groups;
    const int64_t r0 = a.R * g / a.groups, r1 = a.R * (g + 1) / a.groups;
    float2 *Gd = a.G + int64_t(d) * (M + 1);
    for (int64_t r = r0; r < r1; ++r) {
      for (int n = 0; n < N; ++n) {
        for (int i = tid; i < padded_len(M) / 2; i += kNT1) B4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        const int64_t In = a.m.I[n];
        const int Jn = a.m.J[n];
        const int32_t *hn = a.h + d * a.m.ldh + a.m.off[n];
        const int8_t *sn = a.s + d * a.m.ldh + a.m.off[n];
        const float *col = a.U[n] + r;
        const int64_t ld = a.ldU[n];
        const float w = (n == 0 && a.lambda) ? __ldg(a.lambda + r) : 1.f;
        for (int64_t i = tid; i < In; i += kNT1) {
          const int hb = __ldg(hn + i);
          float v = __ldg(col + i * ld) * w;
          if (__ldg(sn + i) < 0) v = -v;
          if (unsigned(hb) < unsigned(Jn)) atomicAdd(Bf + real_off(hb), v);
        }
        __syncthreads();
        block_fft<kL2, kNT1>(B, tw);
        const bool last = n == N - 1;
#pragma unroll
        for (int e = 0; e < PAIRS; ++e) {
          const int q = tid + e * kNT1;
          float2 A, Bs;
          unpack_pair<kL2>(B, q, tw, A, Bs);
          if (n > 0) {
            const float4 p = prod[q];
            A = slot_mul(make_float2(p.x, p.y), A, q == 0);
            Bs = cmul(make_float2(p.z, p.w), Bs);
          }
          if (!last) {
            prod[q] = make_float4(A.x, A.y, Bs.x, Bs.y);
          } else if (q == 0) {
            atomicAdd(&Gd[0].x, A.x);
            atomicAdd(&Gd[M].x, A.y);
            atomicAdd(&Gd[HALF], Bs);
          } else {
            atomicAdd(&Gd[q], A);
            atomicAdd(&Gd[M - q], Bs);
          }
        }
        __syncthreads();              // B is cleared for the next transform
      }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(a.ticket + d, 1u) == unsigned(a.groups - 1);
    __syncthreads();
    if (!is_last) continue;
    __threadfence();
    // last group of sketch d: the inverse real FFT of G_d
    for (int q = tid; q < HALF; q += kNT1) {
      float2 Av, Bv;
      if (q == 0) {
        Av = make_float2(__ldcg(&Gd[0].x), __ldcg(&Gd[M].x));
        Bv = __ldcg(&Gd[HALF]);
      } else {
        Av = __ldcg(&Gd[q]);
        Bv = __ldcg(&Gd[M - q]);
      }
      pack_pair_conj<kL2>(B, q, Av, Bv, tw);
    }
    __syncthreads();
    block_fft<kL2, kNT1>(B, tw);
    const float sc = 1.0f / float(M);
    float *od = a.out + int64_t(d) * a.m.Jt;
    for (int64_t j = tid; j < a.m.Jt; j += kNT1) {
      const float v = Bf[real_off(int(j))];
      od[j] = (j & 1) ? -v * sc : v * sc;
    }
    if (tid == 0) a.ticket[d] = 0u;
    __syncthreads();                  // B is reused by the next item
  }
}

// The same items on the warp-DIT engine for M = 2^14 (wdit::w15, 512
// threads): per transform, the Count Sketch goes into a 32-row scatter
// buffer, each warp runs the 512-point FFTs of two rows, one block barrier,
// then thread t takes column q2(t), twiddles it, runs a 32-point DFT and the
// real-FFT unpack (lane shuffles), leaving TWICE the 32 half-spectrum values
// X[(j < 16 ? q2 : q2_partner(q2)) + 512 j] in registers.  The running
// product of the rank's modes is kept in the CTA's L2 slice (thread t's value
// pair c at prod[c * 512 + t]), the last mode's product is added to G_d with
// atomics, and the next column is scattered between the barriers, as in the
// P = 16384 engine.  G_d therefore holds 2^N times the spectrum, and the
// inverse scales by 2^-N.  The inverse runs on the same engine in place in
// the FFT buffer.  Hash ranges up to 32 * 2 * kRaMax15 real bins fit the
// scatter buffer (ra = ceil(max J_n / 64) <= kRaMax15).
struct Cp15wSmem {
  static constexpr size_t kB = 0;                                   // 32 x kRS float2
  static constexpr size_t kTw = kB + sizeof(float2) * 32 * wdit::kRS;
  static constexpr size_t kStash = kTw + sizeof(float2) * wdit::w15::kTwLen;
  static constexpr size_t kA = kStash + sizeof(float2) * 32;
  static size_t bytes(int ra) { return kA + sizeof(float2) * 32 * size_t(ra); }
};
constexpr int kRaMax15 = int((232448 - 1024 - Cp15wSmem::kA) / (sizeof(float2) * 32));   // 1 KiB for static shared memory

template <int CPT, int RMAX>
__global__ void __launch_bounds__(wdit::kNT) cp15w_kernel(Cp15Args a, const float2 *__restrict__ tw,
                                                          int ra) {
  namespace W = wdit::w15;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int is_last;
  constexpr int NT = wdit::kNT, M = W::kM, HALF = M / 2;
  float2 *B = reinterpret_cast<float2 *>(smem + Cp15wSmem::kB);
  float2 *tws = reinterpret_cast<float2 *>(smem + Cp15wSmem::kTw);
  float2 *stash = reinterpret_cast<float2 *>(smem + Cp15wSmem::kStash);
  float2 *A2 = reinterpret_cast<float2 *>(smem + Cp15wSmem::kA);
  float *A = reinterpret_cast<float *>(A2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = a.m.N;
  const int q2 = wdit::q2_of(tid), q2p = wdit::q2_partner(q2);
  float4 *prod = a.prod + int64_t(blockIdx.x) * HALF;
  W::fill_twiddles(tws, tw);
  for (int e = tid; e < 32 * ra; e += NT) A2[e] = make_float2(0.f, 0.f);
  __syncthreads();
  const int items = a.D * a.groups;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int d = item / a.groups, g = item - d * a.groups;
    const int64_t r0 = a.R * g / a.groups, r1 = a.R * (g + 1) / a.groups;
    float2 *Gd = a.G + int64_t(d) * (M + 1);
    // column (r, n): signed factor values (lambda on mode 0) and hash bins
    float pv[CPT];
    int ph[CPT];
    auto fetch = [&](int64_t r, int n) {
      const int64_t In = a.m.I[n], ld = a.ldU[n];
      const float *col = a.U[n] + r;
      const int32_t *hn = a.h + d * a.m.ldh + a.m.off[n];
      const int8_t *sn = a.s + d * a.m.ldh + a.m.off[n];
      const float w = (n == 0 && a.lambda) ? __ldg(a.lambda + r) : 1.f;
      const int Jn = a.m.J[n];
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int64_t i = tid + int64_t(c) * NT;
        ph[c] = -1;
        pv[c] = 0.f;
        if (i < In) {
          const float v = __ldg(col + i * ld) * w;
          pv[c] = __ldg(sn + i) < 0 ? -v : v;
          const int hb = __ldg(hn + i);
          ph[c] = unsigned(hb) < unsigned(Jn) ? hb : -1;
        }
      }
    };
    auto scatter = [&](int64_t r, int n) {
#pragma unroll
      for (int c = 0; c < CPT; ++c)
        if (ph[c] >= 0) atomicAdd(A + W::a_index(ph[c], ra), pv[c]);
      const int64_t In = a.m.I[n];
      if (In > int64_t(CPT) * NT) {
        const int64_t ld = a.ldU[n];
        const float *col = a.U[n] + r;
        const int32_t *hn = a.h + d * a.m.ldh + a.m.off[n];
        const int8_t *sn = a.s + d * a.m.ldh + a.m.off[n];
        const float w = (n == 0 && a.lambda) ? __ldg(a.lambda + r) : 1.f;
        const int Jn = a.m.J[n];
        for (int64_t i = int64_t(CPT) * NT + tid; i < In; i += NT) {
          const int hb = __ldg(hn + i);
          const float v = __ldg(col + i * ld) * w;
          if (unsigned(hb) < unsigned(Jn))
            atomicAdd(A + W::a_index(hb, ra), __ldg(sn + i) < 0 ? -v : v);
        }
      }
    };
    fetch(r0, 0);
    scatter(r0, 0);
    __syncthreads();
    for (int64_t r = r0; r < r1; ++r) {
      for (int n = 0; n < N; ++n) {
        int64_t rn = r;
        int nn = n + 1;
        if (nn == N) {
          nn = 0;
          ++rn;
        }
        const bool more = rn < r1;
        if (more) fetch(rn, nn);
        wdit::step1_row<RMAX, false, false>(A2 + warp * ra, ra, B + warp * wdit::kRS, tws, warp);
        wdit::step1_row<RMAX, false, false>(A2 + (warp + 16) * ra, ra, B + (warp + 16) * wdit::kRS,
                                         tws, warp + 16);
        __syncthreads();
        // half the warps scatter the next column before step 2, half after
        const bool early = tid < NT / 2;
        if (more && early) scatter(rn, nn);
        float2 v[32];
        W::step2(B, tws, stash, v);
        const bool first = n == 0, last = n == N - 1;
#pragma unroll
        for (int c0 = 0; c0 < 16; c0 += 4) {
          float4 pp[4];
          if (!first) {
#pragma unroll
            for (int c = 0; c < 4; ++c) pp[c] = __ldcg(prod + (c0 + c) * NT + tid);
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int j = 2 * (c0 + c);
            if (!first) {
              v[j] = slot_mul(make_float2(pp[c].x, pp[c].y), v[j], tid == 0 && j == 0);
              v[j + 1] = cmul(make_float2(pp[c].z, pp[c].w), v[j + 1]);
            }
            if (!last) {
              __stcg(prod + (c0 + c) * NT + tid, make_float4(v[j].x, v[j].y, v[j + 1].x, v[j + 1].y));
            } else {
#pragma unroll
              for (int k = 0; k < 2; ++k) {
                const int jj = j + k;
                const int bin = (jj < 16 ? q2 : q2p) + 512 * jj;
                if (tid == 0 && jj == 0) {
                  atomicAdd(&Gd[0].x, v[0].x);      // bins 0 and M, both real
                  atomicAdd(&Gd[M].x, v[0].y);
                } else {
                  atomicAdd(&Gd[bin], v[jj]);
                }
              }
            }
          }
        }
        if (more && !early) scatter(rn, nn);
        __syncthreads();
      }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(a.ticket + d, 1u) == unsigned(a.groups - 1);
    __syncthreads();
    if (is_last) {
      __threadfence();
      // conj-packed sequence of the summed spectrum, row-swizzled into B
      for (int k0 = 0; k0 < HALF / NT; k0 += 8) {
        float2 Av[8], Bv[8], Wv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int q = (k0 + k) * NT + tid;
          if (q == 0) {
            Av[k] = make_float2(__ldcg(&Gd[0].x), __ldcg(&Gd[M].x));
            Bv[k] = __ldcg(&Gd[HALF]);
            Wv[k] = make_float2(1.f, 0.f);
          } else {
            Av[k] = __ldcg(&Gd[q]);
            Bv[k] = __ldcg(&Gd[M - q]);
            Wv[k] = __ldg(&tw[q]);                   // W_P^q, P = 2^15
          }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int q = (k0 + k) * NT + tid;
          float2 cq, cm;
          pack_pair_conj_values_w(q, Av[k], Bv[k], Wv[k], cq, cm);
          B[W::row_pos_swz(q)] = cq;
          B[W::row_pos_swz(q ? M - q : HALF)] = cm;
        }
      }
      __syncthreads();
      wdit::step1_row<16, true, true>(B + warp * wdit::kRS, 512, B + warp * wdit::kRS, tws, warp);
      wdit::step1_row<16, true, true>(B + (warp + 16) * wdit::kRS, 512,
                                   B + (warp + 16) * wdit::kRS, tws, warp + 16);
      __syncthreads();
      float2 v[32];
      W::step2_complex(B, tws, v);                  // v[q1] = Z[q2 + 512 q1]
      // 1/M of the inverse and 2^-N for the doubled unpack of every mode
      const float sc = 1.0f / (float(M) * float(1 << N));
      float *od = a.out + int64_t(d) * a.m.Jt;
      const int64_t Jt = a.m.Jt;
#pragma unroll
      for (int q1 = 0; q1 < 32; ++q1) {
        const int64_t m = q2 + 512 * q1;
        if (2 * m < Jt) od[2 * m] = v[q1].x * sc;
        if (2 * m + 1 < Jt) od[2 * m + 1] = -v[q1].y * sc;
      }
      if (tid == 0) a.ticket[d] = 0u;
    }
    __syncthreads();                                  // B is reused by the next item
  }
  // launched as a programmatic dependent (after a batch chain), complete only
  // after the preceding grid; otherwise this returns at once
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------- contractions
// Half spectra of T transforms Z [T][M] into S [T][M+1] (bin 0 and M real).
__global__ void half_spectrum_kernel(const float2 *__restrict__ Z, int64_t M,
                                     float2 *__restrict__ S, int lp,
                                     const float2 *__restrict__ tw) {
  __shared__ float2 fine[kMaxFine];
  fill_fine(fine, lp);
  __syncthreads();
  const BigTw W{tw, fine, lp};
  const int64_t t = blockIdx.y;
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j > M / 2) return;
  float2 xa, xb;
  half_pair(Z + t * M, M, j, W, xa, xb);
  float2 *s = S + t * (M + 1);
  if (j == 0) {
    s[0] = make_float2(xa.x, 0.f);
    s[M] = make_float2(xa.y, 0.f);
  } else {
    s[j] = xa;
    if (2 * j != M) s[M - j] = xb;
  }
}

// ALL: raw[b][d] += (1/P) sum_k conj(F_d[k]) prod_n X_{b,d,n}[k] over the
// pairs of this block (half-spectrum weights: bins 0 and M once, others
// twice); raw must be zero before the first chunk.  FREE: the product
// F_d prod_{n != m} conj X_{b,d,n} is packed for the inverse into zout
// [(b*D + d) - first/nmode][M].
__global__ void contract_combine_kernel(const float2 *__restrict__ Z, int64_t first,
                                        int nmode, int D, int64_t M,
                                        const float2 *__restrict__ F, int all, float *raw,
                                        float2 *__restrict__ zout, int lp,
                                        const float2 *__restrict__ tw) {
  __shared__ float2 fine[kMaxFine];
  __shared__ float red[32];
  fill_fine(fine, lp);
  __syncthreads();
  const BigTw W{tw, fine, lp};
  const int64_t item = first / nmode + blockIdx.y;       // b * D + d
  const int d = int(item % D);
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool live = j <= M / 2;
  const bool packed = j == 0;
  const float2 *Fd = F + int64_t(d) * (M + 1);
  float2 fa = make_float2(0.f, 0.f), fb = fa, pa = fa, pb = fa;
  if (live) {
    fa = packed ? make_float2(Fd[0].x, Fd[M].x) : Fd[j];
    fb = Fd[M - j];
    pa = all ? make_float2(1.f, packed ? 1.f : 0.f) : fa;
    pb = all ? make_float2(1.f, 0.f) : fb;
    for (int k = 0; k < nmode; ++k) {
      const float2 *Zt = Z + ((item * nmode + k) - first) * M;
      float2 xa, xb;
      half_pair(Zt, M, j, W, xa, xb);
      pa = all ? pmul(pa, xa, packed) : pmulconj(pa, xa, packed);
      pb = all ? pmul(pb, xb, false) : pmulconj(pb, xb, false);
    }
  }
  if (all) {
    float part = 0.f;
    if (live) {
      if (packed) {
        part = fa.x * pa.x + fa.y * pa.y;                  // bins 0 and M
      } else {
        part = 2.f * (fa.x * pa.x + fa.y * pa.y);
        if (2 * j != M) part += 2.f * (fb.x * pb.x + fb.y * pb.y);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      float tsum = 0.f;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) tsum += red[w];
      atomicAdd(raw + item, tsum / float(2 * M));
    }
    return;
  }
  if (!live) return;
  store_packed_pair(zout + (item - first / nmode) * M, M, j, pa, pb, W);
}

// FREE gather: raw[b][d][i] = s_m(i) z_{b,d}[h_m(i)] with z = the real
// inverse (from the forward transform Z of the packed conj sequence).
__global__ void free_gather_kernel(const float2 *__restrict__ Z, int64_t first_item, int D,
                                   int64_t M, Modes m, int free_mode,
                                   const int32_t *__restrict__ h, const int8_t *__restrict__ s,
                                   float *__restrict__ raw) {
  const int64_t item = first_item + blockIdx.y;          // b * D + d
  const int d = int(item % D);
  const int64_t Im = m.I[free_mode];
  const int32_t *hm = h + d * m.ldh + m.off[free_mode];
  const int8_t *sm = s + d * m.ldh + m.off[free_mode];
  const float2 *zt = Z + int64_t(blockIdx.y) * M;
  const float sc = 1.0f / float(M);
  float *r = raw + item * Im;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < Im;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int p = __ldg(hm + i);
    float v = __int_as_float(0x7fc00000);
    if (unsigned(p) < unsigned(2 * M)) {
      const float2 c = zt[p >> 1];
      v = (p & 1) ? -c.y * sc : c.x * sc;
    }
    r[i] = __ldg(sm + i) < 0 ? -v : v;
  }
}

// ---------------------------------------------------------------- outer combine
// S[d][k] (+)= sum over the nl slices of the chunk of X_a[k] X_b[k] for the
// pairs j of sketch d; Za/Zb hold transforms [l][d] of the chunk.  S is the
// half spectrum [D][M+1] (bins 0 and M as reals in .x).
__global__ void outer_accum_kernel(const float2 *__restrict__ Za, const float2 *__restrict__ Zb,
                                   int64_t nl, int D, int64_t M, float2 *__restrict__ S,
                                   int accumulate, int lp, const float2 *__restrict__ tw) {
  __shared__ float2 fine[kMaxFine];
  fill_fine(fine, lp);
  __syncthreads();
  const BigTw W{tw, fine, lp};
  const int d = blockIdx.y;
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j > M / 2) return;
  const bool packed = j == 0;
  float2 sa = make_float2(0.f, 0.f), sb = sa;
  for (int64_t l = 0; l < nl; ++l) {
    const int64_t t = l * D + d;
    float2 aa, ab, ba, bb;
    half_pair(Za + t * M, M, j, W, aa, ab);
    half_pair(Zb + t * M, M, j, W, ba, bb);
    sa = cadd(sa, pmul(aa, ba, packed));
    sb = cadd(sb, pmul(ab, bb, false));
  }
  float2 *Sd = S + int64_t(d) * (M + 1);
  if (packed) {
    const float x0 = accumulate ? Sd[0].x : 0.f, xm = accumulate ? Sd[M].x : 0.f;
    Sd[0] = make_float2(x0 + sa.x, 0.f);
    Sd[M] = make_float2(xm + sa.y, 0.f);
  } else {
    Sd[j] = accumulate ? cadd(Sd[j], sa) : sa;
    if (2 * j != M) Sd[M - j] = accumulate ? cadd(Sd[M - j], sb) : sb;
  }
}

unsigned blocks_for(int64_t n, int per) { return unsigned((n + per - 1) / per); }

}  // namespace

// ---------------------------------------------------------------- host routes
namespace {
// Chunk size (transforms) and workspace bytes of the long CP route under `cap`.
void big_cp_plan(const Modes &m, int64_t R, int D, int log2p, size_t cap, int64_t *tc_out,
                 size_t *bytes_out) {
  const int64_t M = int64_t(1) << (log2p - 1), P = 2 * M;
  const int N = m.N;
  const size_t gbytes = (sizeof(float2) * size_t(D) * size_t(M + 1) + 255) & ~size_t(255);
  const size_t per_t = sizeof(float) * size_t(P) * 2;          // real input + transform
  const int64_t total = int64_t(D) * R * N;
  int64_t tc = cap > gbytes ? int64_t((cap - gbytes) / per_t) : 0;
  tc = std::min(std::max<int64_t>(tc / N * N, N), total);         // whole ranks per chunk
  const int64_t nbuf = std::max<int64_t>(tc, D);                   // D rows for the inverse
  *tc_out = tc;
  *bytes_out = gbytes + per_t * size_t(nbuf);
}
}  // namespace

namespace {
// The fused route for P = 2^15 (cp15_kernel): rank groups per sketch, CTAs
// (at most one per SM; each owns a running-product slice of M/2 float4) and
// bytes under `cap`.  ctas = 0 when not even one slice fits.
struct Cp15Plan {
  int groups = 0;
  int ctas = 0;
  size_t gbytes = 0;          // G, then the tickets
  size_t bytes = 0;
};
Cp15Plan cp15_plan(int64_t R, int D, int nsm, size_t cap) {
  Cp15Plan p;
  const size_t slice = sizeof(float4) * size_t(kM2 / 2);
  p.gbytes = (sizeof(float2) * size_t(D) * size_t(kM2 + 1) + sizeof(unsigned) * size_t(D) + 255) &
             ~size_t(255);
  if (cap < p.gbytes + slice) return p;
  nsm = std::max(nsm, 1);
  const int64_t groups = std::max<int64_t>(1, std::min<int64_t>(R, nsm / D));
  int64_t ctas = std::min<int64_t>(int64_t(D) * groups, nsm);
  ctas = std::min<int64_t>(ctas, int64_t((cap - p.gbytes) / slice));
  p.groups = int(groups);
  p.ctas = int(ctas);
  p.bytes = p.gbytes + slice * size_t(ctas);
  return p;
}
}  // namespace

size_t big_sketch_cp_bytes(const Modes &m, int64_t R, int D, int log2p, size_t cap, int nsm) {
  if (log2p == kL2 + 1) {
    const Cp15Plan f = cp15_plan(R, D, nsm, cap);
    if (f.ctas > 0) return f.bytes;
  }
  int64_t tc;
  size_t bytes;
  big_cp_plan(m, R, D, log2p, cap, &tc, &bytes);
  return bytes;
}

int big_sketch_cp(fcs_ctx *ctx, const Modes &m, int64_t R, int D, const float *const *host_U,
                  const int64_t *host_ldU, const float *lambda, const int32_t *h,
                  const int8_t *s, float *out, int log2p, void *ext_ws, size_t ext_bytes,
                  int stage, bool *split) {
  if (split) *split = false;
  const int L1 = log2p - 1 - kL2;
  const int64_t M = int64_t(1) << (log2p - 1), P = 2 * M;
  const int N = m.N;
  const size_t gbytes = (sizeof(float2) * size_t(D) * size_t(M + 1) + 255) & ~size_t(255);
  const int64_t total = int64_t(D) * R * N;
  const size_t cap = ext_ws ? ext_bytes : std::min(ctx->budget, kBigWorkspaceCap);
  if (L1 == 0) {
    const Cp15Plan f = cp15_plan(R, D, ctx->sm_count, cap);
    if (f.ctas > 0) {
      void *ws = ext_ws;
      if (!ws) {
        int rc = ensure_workspace(ctx, f.bytes, &ws);
        if (rc) return rc;
      }
      Cp15Args a{};
      a.m = m;
      a.R = R;
      a.D = D;
      a.groups = f.groups;
      for (int n = 0; n < N; ++n) {
        a.U[n] = host_U[n];
        a.ldU[n] = host_ldU[n];
      }
      a.lambda = lambda;
      a.h = h;
      a.s = s;
      a.G = static_cast<float2 *>(ws);
      a.ticket = reinterpret_cast<unsigned *>(a.G + size_t(D) * size_t(M + 1));
      a.prod = reinterpret_cast<float4 *>(static_cast<char *>(ws) + f.gbytes);
      a.out = out;
      int64_t jmax = 1, imax = 1;
      for (int n = 0; n < N; ++n) {
        jmax = std::max<int64_t>(jmax, m.J[n]);
        imax = std::max<int64_t>(imax, m.I[n]);
      }
      const int ra = int((jmax + 63) >> 6);
      if (stage != 0 && ra > kRaMax15) return FCS_OK;     // not split: stage 0 runs it
      if (stage != 2) {
        int rc = check_cuda(ctx, cudaMemsetAsync(ws, 0, f.gbytes, ctx->stream),
                            "cudaMemsetAsync(G)");
        if (rc) return rc;
      }
      if (stage == 1) {
        if (split) *split = true;
        return FCS_OK;
      }
      if (ra <= kRaMax15) {
        // the warp-DIT engine: scatter buffer of 32 rows of ra float2
        const int cpt = int((imax + wdit::kNT - 1) / wdit::kNT);
        const void *kern;
        if (ra <= 128)
          kern = cpt <= 1   ? reinterpret_cast<const void *>(cp15w_kernel<1, 4>)
                 : cpt <= 2 ? reinterpret_cast<const void *>(cp15w_kernel<2, 4>)
                            : reinterpret_cast<const void *>(cp15w_kernel<4, 4>);
        else
          kern = cpt <= 1   ? reinterpret_cast<const void *>(cp15w_kernel<1, 8>)
                 : cpt <= 2 ? reinterpret_cast<const void *>(cp15w_kernel<2, 8>)
                            : reinterpret_cast<const void *>(cp15w_kernel<4, 8>);
        const size_t smem = Cp15wSmem::bytes(ra);
        cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(cp15w)");
        const float2 *twp = ctx->twiddle;
        int rap = ra;
        void *args[] = {&a, &twp, &rap};
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(f.ctas));
        cfg.blockDim = dim3(wdit::kNT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = ctx->stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = stage == 2 ? 1 : 0;
        e = cudaLaunchKernelExC(&cfg, kern, args);
        return check_cuda(ctx, e, "cp15w_kernel");
      }
      // the block-FFT kernel (stage 0 only; G was cleared above)
      const size_t smem = sizeof(float2) * padded_len(kM2);
      cudaError_t e = cudaFuncSetAttribute(cp15_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(smem));
      if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(cp15)");
      cp15_kernel<<<unsigned(f.ctas), kNT1, smem, ctx->stream>>>(a, ctx->twiddle);
      return check_cuda(ctx, cudaGetLastError(), "cp15_kernel");
    }
  }
  if (stage != 0) return FCS_OK;                       // not split: stage 0 runs it
  int64_t tc;
  size_t need;
  big_cp_plan(m, R, D, log2p, cap, &tc, &need);
  void *ws = ext_ws;
  int rc = FCS_OK;
  if (ws) {
    if (need > ext_bytes)
      return set_error(ctx, FCS_ENOMEM_BUDGET, "long CP sketch needs %zu bytes, plan holds %zu",
                       need, ext_bytes);
  } else {
    rc = ensure_workspace(ctx, need, &ws);
    if (rc) return rc;
  }
  const int64_t nbuf = std::max<int64_t>(tc, D);
  float2 *G = static_cast<float2 *>(ws);
  float *xb = reinterpret_cast<float *>(static_cast<char *>(ws) + gbytes);
  float2 *Zb = reinterpret_cast<float2 *>(xb + size_t(nbuf) * P);
  rc = check_cuda(ctx, cudaMemsetAsync(G, 0, gbytes, ctx->stream), "cudaMemsetAsync(G)");
  if (rc) return rc;

  CsArgs cs{};
  cs.x = xb;
  cs.x_ld = P;
  cs.nmode = N;
  for (int n = 0; n < N; ++n) {
    cs.mode[n] = n;
    cs.U[n] = host_U[n];
    cs.ldU[n] = host_ldU[n];
  }
  cs.m = m;
  cs.h = h;
  cs.s = s;
  cs.lambda = lambda;
  cs.R = R;
  cs.D = D;
  Pass1Args pa{};
  pa.src = xb;
  pa.src_ld = P;
  pa.nlens = N;
  for (int n = 0; n < N; ++n) pa.lens[n] = m.J[n];
  pa.L1 = L1;
  for (int64_t g0 = 0; g0 < total; g0 += tc) {
    const int64_t nt = std::min(tc, total - g0);
    cs.first = g0;
    cs_kernel<<<unsigned(nt), 256, 0, ctx->stream>>>(cs);
    rc = check_cuda(ctx, cudaGetLastError(), "cs_kernel");
    if (rc) return rc;
    rc = big_fft(ctx, pa, nt, Zb);
    if (rc) return rc;
    cp_accum_kernel<<<dim3(blocks_for(M / 2 + 1, 256), unsigned(D)), 256, 0, ctx->stream>>>(
        Zb, g0, g0 + nt, N, R, M, G, log2p, ctx->twiddle);
    rc = check_cuda(ctx, cudaGetLastError(), "cp_accum_kernel");
    if (rc) return rc;
  }
  // inverse per sketch: G -> packed conj rows in xb -> forward FFT -> out
  float2 *zp = reinterpret_cast<float2 *>(xb);
  pack_inverse_kernel<<<dim3(blocks_for(M / 2, 256), unsigned(D)), 256, 0, ctx->stream>>>(
      G, M + 1, M, zp, log2p, ctx->twiddle);
  rc = check_cuda(ctx, cudaGetLastError(), "pack_inverse_kernel");
  if (rc) return rc;
  Pass1Args pi{};
  pi.src = xb;
  pi.src_ld = P;
  pi.nlens = 1;
  pi.lens[0] = P;
  pi.L1 = L1;
  rc = big_fft(ctx, pi, D, Zb);
  if (rc) return rc;
  unpack_real_kernel<<<dim3(blocks_for(m.Jt, 256), unsigned(D)), 256, 0, ctx->stream>>>(
      Zb, M, 1.0f / float(M), out, m.Jt, m.Jt);
  return check_cuda(ctx, cudaGetLastError(), "unpack_real_kernel");
}

int big_contract(fcs_ctx *ctx, const Modes &m, int kind, int free_mode, int D,
                 const float *fcsT, int64_t B, const float *const *vec, const int32_t *h,
                 const int8_t *s, float2 *spec, bool need_spec, cudaEvent_t spec_ready,
                 float *raw, int log2p) {
  const int L1 = log2p - 1 - kL2;
  const int64_t M = int64_t(1) << (log2p - 1), P = 2 * M;
  const bool all = kind == FCS_CONTRACT_ALL;
  int nmode = 0;
  int modes[kMaxN];
  for (int n = 0; n < m.N; ++n)
    if (all || n != free_mode) modes[nmode++] = n;
  const size_t sbytes =
      spec ? 0 : (sizeof(float2) * size_t(D) * size_t(M + 1) + 255) & ~size_t(255);
  const size_t per_t = sizeof(float) * size_t(P) * 2;
  const size_t cap = std::min(ctx->budget, kBigWorkspaceCap);
  const int64_t unit = std::max<int64_t>(nmode, 1);               // transforms per (b, d)
  const int64_t total = B * D * unit;
  int64_t tc = cap > sbytes ? int64_t((cap - sbytes) / per_t) : 0;
  tc = std::min(std::max<int64_t>(tc / unit * unit, unit), total);  // whole items per chunk
  const int64_t nbuf = std::max<int64_t>(tc, D);                     // D rows for the spectra
  void *ws = nullptr;
  int rc = ensure_workspace(ctx, sbytes + per_t * size_t(nbuf), &ws);
  if (rc) return rc;
  float2 *F = spec ? spec : static_cast<float2 *>(ws);
  float *xb = reinterpret_cast<float *>(static_cast<char *>(ws) + sbytes);
  float2 *Zb = reinterpret_cast<float2 *>(xb + size_t(nbuf) * P);
  if (need_spec) {
    Pass1Args ps{};
    ps.src = fcsT;
    ps.src_ld = m.Jt;
    ps.nlens = 1;
    ps.lens[0] = m.Jt;
    ps.L1 = L1;
    rc = big_fft(ctx, ps, D, Zb);
    if (rc) return rc;
    half_spectrum_kernel<<<dim3(blocks_for(M / 2 + 1, 256), unsigned(D)), 256, 0,
                           ctx->stream>>>(Zb, M, F, log2p, ctx->twiddle);
    rc = check_cuda(ctx, cudaGetLastError(), "half_spectrum_kernel");
    if (rc) return rc;
    if (spec_ready) {
      rc = check_cuda(ctx, cudaEventRecord(spec_ready, ctx->stream), "cudaEventRecord");
      if (rc) return rc;
    }
  }
  if (all) {
    rc = check_cuda(ctx, cudaMemsetAsync(raw, 0, sizeof(float) * size_t(B) * D, ctx->stream),
                    "cudaMemsetAsync(raw)");
    if (rc) return rc;
  }
  CsArgs cs{};
  cs.x = xb;
  cs.x_ld = P;
  cs.nmode = nmode;
  for (int k = 0; k < nmode; ++k) cs.mode[k] = modes[k];
  for (int n = 0; n < m.N; ++n) cs.vec[n] = vec[n];
  cs.m = m;
  cs.h = h;
  cs.s = s;
  cs.D = D;
  Pass1Args pa{};
  pa.src = xb;
  pa.src_ld = P;
  pa.nlens = nmode;
  for (int k = 0; k < nmode; ++k) pa.lens[k] = m.J[modes[k]];
  pa.L1 = L1;
  for (int64_t g0 = 0; g0 < total; g0 += tc) {
    const int64_t nt = std::min(tc, total - g0);
    const int64_t items = nt / unit;
    cs.first = g0;
    cs_kernel<<<unsigned(nt), 256, 0, ctx->stream>>>(cs);
    rc = check_cuda(ctx, cudaGetLastError(), "cs_kernel");
    if (rc) return rc;
    rc = big_fft(ctx, pa, nt, Zb);
    if (rc) return rc;
    float2 *zp = reinterpret_cast<float2 *>(xb);       // FREE: packed products, one per item
    contract_combine_kernel<<<dim3(blocks_for(M / 2 + 1, 256), unsigned(items)), 256, 0,
                              ctx->stream>>>(Zb, g0, nmode, D, M, F, all ? 1 : 0, raw,
                                             zp, log2p, ctx->twiddle);
    rc = check_cuda(ctx, cudaGetLastError(), "contract_combine_kernel");
    if (rc) return rc;
    if (all) continue;
    Pass1Args pi{};
    pi.src = xb;
    pi.src_ld = P;
    pi.nlens = 1;
    pi.lens[0] = P;
    pi.L1 = L1;
    rc = big_fft(ctx, pi, items, Zb);
    if (rc) return rc;
    free_gather_kernel<<<dim3(blocks_for(m.I[free_mode], 256), unsigned(items)), 256, 0,
                         ctx->stream>>>(Zb, g0 / unit, D, M, m, free_mode, h, s, raw);
    rc = check_cuda(ctx, cudaGetLastError(), "free_gather_kernel");
    if (rc) return rc;
  }
  return FCS_OK;
}

int big_outer(fcs_ctx *ctx, int64_t nbatch, int64_t L, int D, int64_t La, int64_t Lb,
              const float *fa, const float *fb, float *out, int log2p) {
  const int L1 = log2p - 1 - kL2;
  const int64_t M = int64_t(1) << (log2p - 1), P = 2 * M;
  const size_t sbytes = (sizeof(float2) * size_t(D) * size_t(M + 1) + 255) & ~size_t(255);
  const size_t per_t = sizeof(float) * size_t(P);               // one transform
  const size_t cap = std::min(ctx->budget, kBigWorkspaceCap);
  // slices per chunk: Za and Zb hold nl * D transforms each; the packed
  // inverse input (D transforms) reuses Za
  int64_t nl = cap > sbytes ? int64_t((cap - sbytes) / (2 * per_t * D)) : 0;
  nl = std::min(std::max<int64_t>(nl, 1), L);
  const int64_t nbuf = nl * D;
  void *ws = nullptr;
  int rc = ensure_workspace(ctx, sbytes + 2 * per_t * size_t(nbuf), &ws);
  if (rc) return rc;
  float2 *S = static_cast<float2 *>(ws);
  float2 *Za = reinterpret_cast<float2 *>(static_cast<char *>(ws) + sbytes);
  float2 *Zb = Za + size_t(nbuf) * M;
  const int64_t Lo = La + Lb - 1;
  for (int64_t b = 0; b < nbatch; ++b) {
    for (int64_t l0 = 0; l0 < L; l0 += nl) {
      const int64_t cl = std::min(nl, L - l0);
      const int64_t first = (b * L + l0) * D;                  // slice-sketch index
      Pass1Args p{};
      p.nlens = 1;
      p.L1 = L1;
      p.src = fa + first * La;
      p.src_ld = La;
      p.lens[0] = La;
      rc = big_fft(ctx, p, cl * D, Za);
      if (rc) return rc;
      p.src = fb + first * Lb;
      p.src_ld = Lb;
      p.lens[0] = Lb;
      rc = big_fft(ctx, p, cl * D, Zb);
      if (rc) return rc;
      outer_accum_kernel<<<dim3(blocks_for(M / 2 + 1, 256), unsigned(D)), 256, 0,
                           ctx->stream>>>(Za, Zb, cl, D, M, S, l0 > 0 ? 1 : 0, log2p,
                                          ctx->twiddle);
      rc = check_cuda(ctx, cudaGetLastError(), "outer_accum_kernel");
      if (rc) return rc;
    }
    float2 *zp = Za;
    pack_inverse_kernel<<<dim3(blocks_for(M / 2, 256), unsigned(D)), 256, 0, ctx->stream>>>(
        S, M + 1, M, zp, log2p, ctx->twiddle);
    rc = check_cuda(ctx, cudaGetLastError(), "pack_inverse_kernel");
    if (rc) return rc;
    Pass1Args pi{};
    pi.src = reinterpret_cast<const float *>(zp);
    pi.src_ld = P;
    pi.nlens = 1;
    pi.lens[0] = P;
    pi.L1 = L1;
    rc = big_fft(ctx, pi, D, Zb);
    if (rc) return rc;
    unpack_real_kernel<<<dim3(blocks_for(Lo, 256), unsigned(D)), 256, 0, ctx->stream>>>(
        Zb, M, 1.0f / float(M), out + b * D * Lo, Lo, Lo);
    rc = check_cuda(ctx, cudaGetLastError(), "unpack_real_kernel");
    if (rc) return rc;
  }
  return FCS_OK;
}

}  // namespace fcs
