// fcs_cp.cu -- fcs_sketch_cp: FCS of a CP tensor by eq. (FCS_syn):
//   FCS(T) = sum_r lambda_r IFFT( prod_n FFT_P( CS_n(U_n(:, r)) ) ),
// with P the smallest power of two >= Jt (any P >= Jt gives the exact linear
// convolution, so out = the first Jt samples).
//
// Two kernels.  (1) prep_kernel writes the factor columns contiguously
// (lambda folded into mode 1) so every column load is coalesced, and clears
// the spectrum accumulator.  (2) The fused sketch kernel: CTA (g, d) owns sketch d and a contiguous group of
// ranks.  For each rank and mode it scatters the signed factor column into a
// compact shared-memory buffer of max_n J_n reals (the Count Sketch of
// Def. 1; the zero padding up to P is never stored), runs the block real FFT
// of fcs_fft.cuh whose last pass leaves the half spectrum in registers, and
// multiplies it into the per-thread mode product; after the last mode the
// product is added into a shared-memory rank accumulator.  The rank sum thus
// stays in the frequency domain (linearity moves the paper's sum of inverse
// transforms inside one inverse transform).  Each CTA adds its partial
// spectrum into a global accumulator with float2 atomics; the last CTA to
// finish for sketch d (ticket counter) runs the one inverse real FFT and
// writes FCS_d.  The next column's factor values and hashes are prefetched
// into registers while the current column is transformed.  For P = 16384
// the kernel runs on the warp-DIT engine instead (cp13_kernel): two block
// barriers per transform, the next column scattered between them.
#include <algorithm>
#include <cstdarg>
#include <mutex>

#include "fcs_fft.cuh"

namespace fcs {
namespace {

struct CpArgs {
  Modes m;
  int D;
  int64_t R;
  int64_t ranks_per_cta;
  const float *UT;       // [sum_n R*I_n]: mode n column r at ut_off[n] + r*I_n
  int64_t ut_off[kMaxN];
  const int32_t *h;
  const int8_t *s;
  float2 *G;             // [D][M+2] spectrum accumulator (bins 0..M), zeroed per call
  unsigned *counter;     // [D] tickets, zero at launch, reset by the last CTA
  float *out;            // [D][Jt]
  int sb;                // scatter buffer length (floats): max J_n rounded up to 4
};

// All modes in one launch: mode n = blockIdx.z.
struct TransposeArgs {
  const float *U[kMaxN];
  int64_t I[kMaxN], ld[kMaxN], ut_off[kMaxN];
  int64_t R;
  const float *lambda;
  float *UT;
};

// Shared-memory layout of cp_kernel; every region starts on a 16-byte
// boundary (the scatter buffer is cleared with float4 stores).
template <int LOG2M, int NT>
struct CpSmem {
  static constexpr size_t up16(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t kB = 0;
  static constexpr size_t kAcc = up16(kB + sizeof(float2) * padded_len(1 << LOG2M));
  static constexpr size_t kTw =
      up16(kAcc + sizeof(float2) * LastPass<LOG2M, NT>::NV * NT);
  static constexpr size_t kA = up16(kTw + sizeof(float2) * plan_twlen(LOG2M));
  static size_t bytes(int sb) { return kA + sizeof(float) * size_t(sb); }
};

template <int LOG2M, int NT, int CPT>
__global__ void __launch_bounds__(NT) cp_kernel(CpArgs a, const float2 *__restrict__ tw) {
  using LPs = LastPass<LOG2M, NT>;
  constexpr int M = 1 << LOG2M;
  constexpr int HALF = M / 2;
  constexpr int RL = LPs::RL, EPS = LPs::EPS, NV = LPs::NV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using Lay = CpSmem<LOG2M, NT>;
  float2 *B = reinterpret_cast<float2 *>(smem_raw + Lay::kB);      // padded_len(M)
  float2 *accS = reinterpret_cast<float2 *>(smem_raw + Lay::kAcc); // NV * NT
  float2 *tws = reinterpret_cast<float2 *>(smem_raw + Lay::kTw);   // plan_twlen
  float *A = reinterpret_cast<float *>(smem_raw + Lay::kA);        // a.sb floats
  __shared__ int is_last;
  const int tid = threadIdx.x;
  const int d = blockIdx.y;
  const int N = a.m.N;
  const int64_t r0 = blockIdx.x * a.ranks_per_cta;
  const int64_t r1 = min(a.R, r0 + a.ranks_per_cta);
  const int sb = a.sb;

  fill_twiddles<LOG2M, NT>(tws, tw);
  for (int e = tid; e < sb / 4; e += NT) reinterpret_cast<float4 *>(A)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int v = 0; v < NV; ++v) accS[v * NT + tid] = make_float2(0.f, 0.f);

  // prefetched column: signed factor values and hash bins
  float pv[CPT];
  int ph[CPT];
  auto fetch = [&](int64_t r, int n) {
    const int64_t In = a.m.I[n];
    const float *col = a.UT + a.ut_off[n] + r * In;
    const int32_t *hn = a.h + d * a.m.ldh + a.m.off[n];
    const int8_t *sn = a.s + d * a.m.ldh + a.m.off[n];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int64_t i = tid + int64_t(c) * NT;
      ph[c] = -1;
      pv[c] = 0.f;
      if (i < In) {
        const float v = __ldg(col + i);
        pv[c] = __ldg(sn + i) < 0 ? -v : v;
        ph[c] = __ldg(hn + i);
      }
    }
  };
  fetch(r0, 0);
  __syncthreads();

  float2 X[EPS][2][RL], p[EPS][2][RL];
  for (int64_t r = r0; r < r1; ++r) {
    for (int n = 0; n < N; ++n) {
#pragma unroll
      for (int c = 0; c < CPT; ++c)
        if (unsigned(ph[c]) < unsigned(sb)) atomicAdd(A + ph[c], pv[c]);
      if (a.m.I[n] > int64_t(CPT) * NT) {
        // entries beyond the prefetched chunk: load and scatter directly
        const int64_t In = a.m.I[n];
        const float *col = a.UT + a.ut_off[n] + r * In;
        const int32_t *hn = a.h + d * a.m.ldh + a.m.off[n];
        const int8_t *sn = a.s + d * a.m.ldh + a.m.off[n];
        for (int64_t i = int64_t(CPT) * NT + tid; i < In; i += NT) {
          const int hb = __ldg(hn + i);
          const float v = __ldg(col + i);
          if (unsigned(hb) < unsigned(sb)) atomicAdd(A + hb, __ldg(sn + i) < 0 ? -v : v);
        }
      }
      // prefetch the next column while this one is transformed
      if (n + 1 < N)
        fetch(r, n + 1);
      else if (r + 1 < r1)
        fetch(r + 1, 0);
      __syncthreads();
      fft_first_pass<LOG2M, NT>(A, sb, B);
      __syncthreads();
      for (int e = tid; e < sb / 4; e += NT)
        reinterpret_cast<float4 *>(A)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
      fft_middle_passes<LOG2M, NT, 1>(B, tws);
      fft_last_pass_unpack<LOG2M, NT>(B, tw, X);
#pragma unroll
      for (int e = 0; e < EPS; ++e)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int q = 0; q < RL; ++q) {
            if (n == 0) {
              p[e][b][q] = X[e][b][q];
            } else {
              const bool packed = (b == 0 && q == 0 && tid + e * NT == 0);
              p[e][b][q] = slot_mul(p[e][b][q], X[e][b][q], packed);
            }
          }
    }
#pragma unroll
    for (int e = 0; e < EPS; ++e)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int q = 0; q < RL; ++q) {
          float2 &acc = accS[((e * 2 + b) * RL + q) * NT + tid];
          acc = cadd(acc, p[e][b][q]);
        }
  }

  // publish the partial spectrum
  float2 *Gd = a.G + d * int64_t(M + 2);
#pragma unroll
  for (int e = 0; e < EPS; ++e) {
    if (LPs::SLOTS % NT != 0 && tid + e * NT >= LPs::SLOTS) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int q = 0; q < RL; ++q) {
        const float2 v = accS[((e * 2 + b) * RL + q) * NT + tid];
        const int k = last_pass_index<LOG2M, NT>(e, b, q);
        if (k == 0) {
          atomicAdd(&Gd[0].x, v.x);
          atomicAdd(&Gd[M].x, v.y);
        } else {
          atomicAdd(&Gd[k], v);
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
  for (int q = tid; q < HALF; q += NT) {
    float2 Av, Bv;
    if (q == 0) {
      Av = make_float2(__ldcg(&Gd[0].x), __ldcg(&Gd[M].x));
      Bv = __ldcg(&Gd[HALF]);
    } else {
      Av = __ldcg(&Gd[q]);
      Bv = __ldcg(&Gd[M - q]);
    }
    pack_pair_conj<LOG2M>(B, q, Av, Bv, tw);
  }
  __syncthreads();
  block_fft<LOG2M, NT>(B, tw);
  const float sc = 1.0f / float(M);
  float *od = a.out + d * a.m.Jt;
  float *Br = reinterpret_cast<float *>(B);
  for (int64_t j = tid; j < a.m.Jt; j += NT) {
    const float v = Br[real_off(int(j))];
    od[j] = (j & 1) ? -v * sc : v * sc;
  }
  if (tid == 0) a.counter[d] = 0u;
}

// cp_kernel for P = 16384 on the warp-DIT engine (wdit:: in fcs_fft.cuh):
// the same work split, prefetch, rank accumulation and last-CTA inverse, but
// two block barriers per transform.  The next column is scattered into the
// row-wise buffer between them, overlapping step 2 of the current one.
// RMAX = number of 32-entry blocks per scatter-buffer row (ra <= 32 RMAX).
struct Cp13Smem {
  static constexpr size_t kB = 0;                                   // 16 x kRS float2
  static constexpr size_t kAcc = kB + sizeof(float2) * 16 * wdit::kRS;
  static constexpr size_t kTw = kAcc + sizeof(float2) * 16 * wdit::kNT;
  static constexpr size_t kStash = kTw + sizeof(float2) * wdit::kTwLen;
  static constexpr size_t kA = kStash + sizeof(float2) * 16;
  static size_t bytes(int ra) { return kA + sizeof(float2) * 16 * size_t(ra); }
};

template <int CPT, int RMAX>
__global__ void __launch_bounds__(wdit::kNT) cp13_kernel(CpArgs a, const float2 *__restrict__ tw) {
  constexpr int NT = wdit::kNT, M = wdit::kM, HALF = M / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *B = reinterpret_cast<float2 *>(smem_raw + Cp13Smem::kB);
  float4 *acc4 = reinterpret_cast<float4 *>(smem_raw + Cp13Smem::kAcc);   // [8][NT] pairs
  float2 *tws = reinterpret_cast<float2 *>(smem_raw + Cp13Smem::kTw);
  float2 *stash = reinterpret_cast<float2 *>(smem_raw + Cp13Smem::kStash);
  float2 *A2 = reinterpret_cast<float2 *>(smem_raw + Cp13Smem::kA);
  float *A = reinterpret_cast<float *>(A2);
  __shared__ int is_last;
  const int tid = threadIdx.x;
  const int d = blockIdx.y;
  const int N = a.m.N;
  const int64_t r0 = blockIdx.x * a.ranks_per_cta;
  const int64_t r1 = min(a.R, r0 + a.ranks_per_cta);
  const int sb = a.sb;
  const int ra = (sb + 31) >> 5;

  float pv[CPT];
  int ph[CPT];
  auto fetch = [&](int64_t r, int n) {
    const int64_t In = a.m.I[n];
    const float *col = a.UT + a.ut_off[n] + r * In;
    const int32_t *hn = a.h + d * a.m.ldh + a.m.off[n];
    const int8_t *sn = a.s + d * a.m.ldh + a.m.off[n];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int64_t i = tid + int64_t(c) * NT;
      ph[c] = -1;
      pv[c] = 0.f;
      if (i < In) {
        const float v = __ldg(col + i);
        pv[c] = __ldg(sn + i) < 0 ? -v : v;
        ph[c] = __ldg(hn + i);
      }
    }
  };
  // scatter the fetched column (and, for I_n > CPT NT, the rest of it)
  auto scatter = [&](int64_t r, int n) {
#pragma unroll
    for (int c = 0; c < CPT; ++c)
      if (unsigned(ph[c]) < unsigned(sb)) atomicAdd(A + wdit::a_index(ph[c], ra), pv[c]);
    const int64_t In = a.m.I[n];
    if (In > int64_t(CPT) * NT) {
      const float *col = a.UT + a.ut_off[n] + r * In;
      const int32_t *hn = a.h + d * a.m.ldh + a.m.off[n];
      const int8_t *sn = a.s + d * a.m.ldh + a.m.off[n];
      for (int64_t i = int64_t(CPT) * NT + tid; i < In; i += NT) {
        const int hb = __ldg(hn + i);
        const float v = __ldg(col + i);
        if (unsigned(hb) < unsigned(sb))
          atomicAdd(A + wdit::a_index(hb, ra), __ldg(sn + i) < 0 ? -v : v);
      }
    }
  };
  // the first column's loads and the twiddle loads overlap
  fetch(r0, 0);
  wdit::fill_twiddles(tws, tw);
  for (int e = tid; e < 16 * ra; e += NT) A2[e] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < 8; ++q) acc4[q * NT + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  scatter(r0, 0);
  __syncthreads();

  float2 p[16];
  for (int64_t r = r0; r < r1; ++r) {
    for (int n = 0; n < N; ++n) {
      // the scatter buffer holds column (r, n); fetch the next one
      int64_t rn = r;
      int nn = n + 1;
      if (nn == N) {
        nn = 0;
        ++rn;
      }
      const bool more = rn < r1;
      if (more) fetch(rn, nn);
      wdit::step1<RMAX>(A2, ra, B, tws);
      __syncthreads();
      // warps 0-7 scatter the next column before step 2, warps 8-15 after it,
      // so each scheduler overlaps the atomics' latency with step-2 work
      const bool early = tid < NT / 2;
      if (more && early) scatter(rn, nn);
      float2 v[16];
      wdit::step2(B, tws, stash, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (n == 0)
          p[j] = v[j];
        else
          p[j] = slot_mul(p[j], v[j], tid == 0 && j == 0);
      }
      if (n == N - 1) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float4 &acc = acc4[q * NT + tid];
          float4 x = acc;
          x.x += p[2 * q].x;
          x.y += p[2 * q].y;
          x.z += p[2 * q + 1].x;
          x.w += p[2 * q + 1].y;
          acc = x;
        }
      }
      if (more && !early) scatter(rn, nn);
      __syncthreads();
    }
  }

  // publish the partial spectrum as 16-byte atomics over bin pairs (k, k+1);
  // value j of thread t is 2^N X[spectrum_index(q2(t), j)]
  float2 *Gd = a.G + d * int64_t(M + 2);
  const float2 *accv = reinterpret_cast<const float2 *>(acc4);
  auto acc_at = [&](int k) -> float2 {       // accumulated value of bin k (k < M)
    const int jj = k >> 9, c = k & 511;
    const int q2 = jj < 8 ? c : wdit::q2_partner(c);
    const int u = q2 <= 256 ? (q2 == 256 ? 0 : q2) : 512 - q2;
    const int e = q2 >= 256 ? 1 : 0;
    const int t = ((u >> 4) << 5) | (e << 4) | (u & 15);
    return accv[((jj >> 1) * NT + t) * 2 + (jj & 1)];
  };
  for (int f = tid; f < M / 2; f += NT) {
    const float2 x0 = acc_at(2 * f), x1 = acc_at(2 * f + 1);
    if (f == 0) {
      atomicAdd(&Gd[M].x, x0.y);            // bin M (packed with bin 0)
      atomicAdd(reinterpret_cast<float4 *>(Gd), make_float4(x0.x, 0.f, x1.x, x1.y));
    } else {
      atomicAdd(reinterpret_cast<float4 *>(Gd) + f, make_float4(x0.x, x0.y, x1.x, x1.y));
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = (atomicAdd(&a.counter[d], 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  // last CTA for sketch d: one inverse real FFT of the summed spectrum on the
  // same engine.  The conj-packed sequence goes row-wise (ra = 512) into the
  // accumulator region; a forward complex FFT, conj and scaling give FCS_d.
  float2 *Z2 = reinterpret_cast<float2 *>(acc4);
  {
    // all (coalesced) loads first: one L2 round trip
    constexpr int PER = HALF / NT;
    float2 Av[PER], Bv[PER], Wv[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int q = k * NT + tid;
      if (q == 0) {
        Av[k] = make_float2(__ldcg(&Gd[0].x), __ldcg(&Gd[M].x));
        Bv[k] = __ldcg(&Gd[HALF]);
        Wv[k] = make_float2(1.f, 0.f);
      } else {
        Av[k] = __ldcg(&Gd[q]);
        Bv[k] = __ldcg(&Gd[M - q]);
        Wv[k] = __ldg(&tw[q << (kLogTwN - wdit::kL - 1)]);   // W_P^q
      }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int q = k * NT + tid;
      float2 cq, cm;
      pack_pair_conj_values_w(q, Av[k], Bv[k], Wv[k], cq, cm);
      Z2[wdit::row_pos_swz(q)] = cq;
      Z2[wdit::row_pos_swz(q ? M - q : HALF)] = cm;
    }
  }
  __syncthreads();
  wdit::step1<16, true>(Z2, 512, B, tws);
  __syncthreads();
  float2 v[16];
  wdit::step2_complex(B, tws, v);                   // v[q1] = Z[q2 + 512 q1]
  // 1/M of the inverse and 2^-N for the doubled unpack of every mode
  const float sc = 1.0f / float(int64_t(M) << N);
  float *od = a.out + d * a.m.Jt;
  const int64_t Jt = a.m.Jt;
  const int q2 = wdit::q2_of(tid);
#pragma unroll
  for (int q1 = 0; q1 < 16; ++q1) {
    const int64_t m = q2 + 512 * q1;
    if (2 * m < Jt) od[2 * m] = v[q1].x * sc;
    if (2 * m + 1 < Jt) od[2 * m + 1] = -v[q1].y * sc;
  }
  if (tid == 0) a.counter[d] = 0u;
}

// prep_kernel: in one launch, the factor transpose in 32 x 32 tiles,
// UT[n][r][i] = U_n[i*ld + r] (times lambda_r for n = 0), and the clearing
// of the spectrum accumulator and tickets.  256 threads per block.
struct PrepArgs {
  TransposeArgs t;
  int64_t tiles_x, tiles_y, ntile;     // transpose tiles per mode and in total
  float4 *zero;
  int64_t zero_n4;
  int zero_blocks;
};

__global__ void __launch_bounds__(256) prep_kernel(PrepArgs a) {
  const int64_t b = blockIdx.x;
  const int tid = threadIdx.x;
  if (b < a.ntile) {
    __shared__ float tile[32][33];
    const int64_t per = a.tiles_x * a.tiles_y;
    const int n = int(b / per);
    const int64_t rem = b % per;
    const int64_t bx = rem % a.tiles_x, by = rem / a.tiles_x;
    const int64_t I = a.t.I[n], R = a.t.R, ld = a.t.ld[n];
    const float *U = a.t.U[n];
    const float *lambda = n == 0 ? a.t.lambda : nullptr;
    float *UT = a.t.UT + a.t.ut_off[n];
    const int64_t i0 = bx * 32, rr0 = by * 32;
    if (i0 >= I) return;
    const int tx = tid & 31, ty = tid >> 5;
    for (int k = ty; k < 32; k += 8) {
      const int64_t i = i0 + k, r = rr0 + tx;
      if (i < I && r < R) tile[k][tx] = U[i * ld + r];
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
      const int64_t r = rr0 + k, i = i0 + tx;
      if (i < I && r < R) {
        const float lam = lambda ? __ldg(lambda + r) : 1.f;
        UT[r * I + i] = tile[tx][k] * lam;
      }
    }
    return;
  }
  const int64_t zb = b - a.ntile;
  for (int64_t e = zb * 256 + tid; e < a.zero_n4; e += int64_t(a.zero_blocks) * 256)
    a.zero[e] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Kernel for the given prefetch depth and scatter-buffer height.
template <int CPT>
const void *cp13_pick_rmax(int ra) {
  if (ra <= 128) return reinterpret_cast<const void *>(cp13_kernel<CPT, 4>);
  if (ra <= 256) return reinterpret_cast<const void *>(cp13_kernel<CPT, 8>);
  return reinterpret_cast<const void *>(cp13_kernel<CPT, 16>);
}
const void *cp13_pick(int64_t Imax, int sb) {
  const int ra = (sb + 31) >> 5;
  const int cpt = int((Imax + wdit::kNT - 1) / wdit::kNT);
  if (cpt <= 1) return cp13_pick_rmax<1>(ra);
  if (cpt <= 2) return cp13_pick_rmax<2>(ra);
  return cp13_pick_rmax<4>(ra);
}

int launch_cp13(fcs_ctx *ctx, CpArgs &a, int64_t groups, int64_t Imax) {
  const size_t smem = Cp13Smem::bytes((a.sb + 31) >> 5);
  const void *kern = cp13_pick(Imax, a.sb);
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(cp13)");
  const float2 *twp = ctx->twiddle;
  void *args[] = {&a, &twp};
  e = cudaLaunchKernel(kern, dim3(unsigned(groups), unsigned(a.D)), dim3(wdit::kNT), args, smem,
                       ctx->stream);
  return check_cuda(ctx, e, "cp13_kernel");
}

template <int LOG2M>
int launch_cp(fcs_ctx *ctx, CpArgs &a, int64_t groups, int64_t Imax) {
  if constexpr (LOG2M == wdit::kL) {
    return launch_cp13(ctx, a, groups, Imax);
  } else {
    constexpr int NT = fft_threads(LOG2M);
    const size_t smem = CpSmem<LOG2M, NT>::bytes(a.sb);
    const int cpt = int((Imax + NT - 1) / NT);
    auto go = [&](auto kern) -> int {
      if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(cp)");
      }
      kern<<<dim3(unsigned(groups), unsigned(a.D)), NT, smem, ctx->stream>>>(a, ctx->twiddle);
      return check_cuda(ctx, cudaGetLastError(), "cp_kernel");
    };
    if (cpt <= 1) return go(cp_kernel<LOG2M, NT, 1>);
    if (cpt <= 2) return go(cp_kernel<LOG2M, NT, 2>);
    return go(cp_kernel<LOG2M, NT, 4>);       // larger modes add a direct tail loop
  }
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
  }
  const int log2p = ilog2_ceil(a.m.Jt) < kMinLog2P ? kMinLog2P : ilog2_ceil(a.m.Jt);
  if (log2p > kMaxLog2PBig)
    return set_error(ctx, FCS_EUNSUPPORTED, "Jt=%lld needs FFT length > %d",
                     (long long)a.m.Jt, 1 << kMaxLog2PBig);
  if (log2p > kMaxLog2P) {
    DeviceGuard g(ctx->device);
    spec_cache_invalidate(ctx, out, sizeof(float) * size_t(D) * size_t(a.m.Jt));
    return big_sketch_cp(ctx, a.m, R, D, host_U, host_ldU, lambda, h, s, out, log2p);
  }
  const int log2m = log2p - 1;
  const int M = 1 << log2m;
  a.D = D;
  a.R = R;
  a.h = h;
  a.s = s;
  a.out = out;
  // rank groups: about one CTA per SM over all sketches
  int64_t groups = (int64_t(ctx->sm_count) + D - 1) / D;
  if (groups < 1) groups = 1;
  if (groups > R) groups = R;
  a.ranks_per_cta = (R + groups - 1) / groups;
  groups = (R + a.ranks_per_cta - 1) / a.ranks_per_cta;

  int64_t Imax = 0, Jmax = 0, utlen = 0;
  for (int n = 0; n < N; ++n) {
    a.ut_off[n] = utlen;
    utlen += R * host_I[n];
    if (host_I[n] > Imax) Imax = host_I[n];
    if (host_J[n] > Jmax) Jmax = host_J[n];
  }
  a.sb = int((Jmax + 3) / 4 * 4);
  const size_t gbytes = (sizeof(float2) * size_t(D) * size_t(M + 2) + 255) & ~size_t(255);
  const size_t cbytes = 256;
  void *ws = nullptr;
  rc = ensure_workspace(ctx, gbytes + cbytes + sizeof(float) * size_t(utlen), &ws);
  if (rc) return rc;
  a.G = static_cast<float2 *>(ws);
  a.counter = reinterpret_cast<unsigned *>(static_cast<char *>(ws) + gbytes);
  float *UT = reinterpret_cast<float *>(static_cast<char *>(ws) + gbytes + cbytes);
  a.UT = UT;
  DeviceGuard g(ctx->device);
  spec_cache_invalidate(ctx, out, sizeof(float) * size_t(D) * size_t(a.m.Jt));
  {
    // one launch: factor transpose (lambda folded into mode 1) and clearing
    // of the accumulator and tickets
    PrepArgs pa{};
    for (int n = 0; n < N; ++n) {
      pa.t.U[n] = host_U[n];
      pa.t.I[n] = host_I[n];
      pa.t.ld[n] = host_ldU[n];
      pa.t.ut_off[n] = a.ut_off[n];
    }
    pa.t.R = R;
    pa.t.lambda = lambda;
    pa.t.UT = UT;
    pa.tiles_x = (Imax + 31) / 32;
    pa.tiles_y = (R + 31) / 32;
    pa.ntile = pa.tiles_x * pa.tiles_y * N;
    pa.zero = static_cast<float4 *>(ws);
    pa.zero_n4 = int64_t(gbytes + cbytes) / 16;
    pa.zero_blocks = int(std::min<int64_t>(64, (pa.zero_n4 + 255) / 256));
    const int64_t blocks = pa.ntile + pa.zero_blocks;
    if (blocks > 0x7fffffffLL) return set_error(ctx, FCS_EUNSUPPORTED, "factor matrices too large");
    prep_kernel<<<unsigned(blocks), 256, 0, ctx->stream>>>(pa);
    rc = check_cuda(ctx, cudaGetLastError(), "prep_kernel");
    if (rc) return rc;
  }
  rc = FCS_EUNSUPPORTED;
  FCS_DISPATCH_LOG2M(log2m, rc = launch_cp<L>(ctx, a, groups, Imax));
  return rc;
}

// ---------------------------------------------------------------------------
// fcs_sketch_cp_noalloc: the CP-route sketch for callers that cannot allocate
// device memory.  It runs the same two kernels as fcs_sketch_cp, but its
// scratch (spectrum accumulator, tickets, transposed factor columns) and its
// twiddle table live in file-scope __device__ arrays of fixed size instead of
// a context workspace, so the call makes no cudaMalloc / cudaFree and needs
// no fcs_ctx.
namespace fcs {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;   // 4 MiB
constexpr int kNoAllocMaxDevices = 64;

// One copy of each array exists on every GPU that loads the library and is
// held until the process exits.  In host code these names are host-side
// stand-ins, not device addresses: kernels get the addresses that
// cudaGetSymbolAddress returns at set-up.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
__device__ __align__(256) float2 g_noalloc_twiddle[kTwN];

struct NoAllocDevice {
  bool ready;
  unsigned char *scratch;
  float2 *twiddle;
  int sm_count;
};
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// tw[k] = exp(-2 pi i k / kTwN) in FP64, rounded to FP32.
__global__ void noalloc_twiddle_kernel(float2 *tw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < kTwN) {
    double sn, cs;
    sincospi(2.0 * double(k) / double(kTwN), &sn, &cs);
    tw[k] = make_float2(float(cs), float(-sn));
  }
}

int noalloc_fail(char *err, size_t n, int code, const char *fmt, ...) {
  if (err && n) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, n, fmt, ap);
    va_end(ap);
  }
  return code;
}

// First call on a device (with that device current): look up the device
// addresses of the static arrays and fill the twiddle table (the stream is
// synchronised once so any later stream sees the table).
int noalloc_setup(int dev, cudaStream_t st, NoAllocDevice **out, char *err, size_t n) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocDevice &s = g_noalloc_dev[dev];
  if (!s.ready) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "cudaGetSymbolAddress(scratch): %s",
                          cudaGetErrorString(e));
    s.scratch = static_cast<unsigned char *>(p);
    e = cudaGetSymbolAddress(&p, g_noalloc_twiddle);
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "cudaGetSymbolAddress(twiddle): %s",
                          cudaGetErrorString(e));
    s.twiddle = static_cast<float2 *>(p);
    e = cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
    noalloc_twiddle_kernel<<<kTwN / 256, 256, 0, st>>>(s.twiddle);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "twiddle set-up: %s", cudaGetErrorString(e));
    s.ready = true;
  }
  *out = &s;
  return FCS_OK;
}

template <int LOG2M>
int noalloc_launch_cp(CpArgs &a, int64_t groups, int64_t Imax, const float2 *tw,
                      cudaStream_t st, char *err, size_t n) {
  constexpr int NT = fft_threads(LOG2M);
  const size_t smem = LOG2M == wdit::kL ? Cp13Smem::bytes((a.sb + 31) >> 5)
                                        : CpSmem<LOG2M, NT>::bytes(a.sb);
  const int cpt = int((Imax + NT - 1) / NT);
  auto go = [&](auto kern) -> int {
    if (smem > 48 * 1024) {
      cudaError_t e =
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess)
        return noalloc_fail(err, n, FCS_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    }
    kern<<<dim3(unsigned(groups), unsigned(a.D)), NT, smem, st>>>(a, tw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "cp_kernel: %s", cudaGetErrorString(e));
    return FCS_OK;
  };
  if constexpr (LOG2M == wdit::kL) {
    const void *kern = cp13_pick(Imax, a.sb);
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    void *args[] = {&a, &tw};
    e = cudaLaunchKernel(kern, dim3(unsigned(groups), unsigned(a.D)), dim3(NT), args, smem, st);
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "cp13_kernel: %s", cudaGetErrorString(e));
    return FCS_OK;
  } else {
    if (cpt <= 1) return go(cp_kernel<LOG2M, NT, 1>);
    if (cpt <= 2) return go(cp_kernel<LOG2M, NT, 2>);
    return go(cp_kernel<LOG2M, NT, 4>);
  }
}

}  // namespace
}  // namespace fcs

extern "C" int fcs_sketch_cp_noalloc(void *stream, int N, const int64_t *host_I,
                                     const int32_t *host_J, int64_t R, int D,
                                     const float *const *host_U, const int64_t *host_ldU,
                                     const float *lambda, const int32_t *h, const int8_t *s,
                                     int64_t ldh, float *out, char *err, size_t err_len) {
  if (err && err_len) err[0] = '\0';
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CpArgs a{};
  if (make_modes(nullptr, N, host_I, host_J, ldh, &a.m) != FCS_OK)
    return noalloc_fail(err, err_len, FCS_EINVAL,
                        "invalid N, I_n, J_n or ldh (1 <= N <= %d, I_n >= 1, J_n >= 1)", kMaxN);
  if (D < 1 || D > kMaxD)
    return noalloc_fail(err, err_len, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (R < 1) return noalloc_fail(err, err_len, FCS_EINVAL, "R=%lld must be >= 1", (long long)R);
  if (!host_U || !host_ldU || !h || !s || !out)
    return noalloc_fail(err, err_len, FCS_EINVAL, "NULL pointer argument");
  for (int n = 0; n < N; ++n) {
    if (!host_U[n]) return noalloc_fail(err, err_len, FCS_EINVAL, "U[%d] is NULL", n);
    if (host_ldU[n] < R)
      return noalloc_fail(err, err_len, FCS_EINVAL, "ldU[%d]=%lld < R", n,
                          (long long)host_ldU[n]);
  }
  const int log2p = ilog2_ceil(a.m.Jt) < kMinLog2P ? kMinLog2P : ilog2_ceil(a.m.Jt);
  if (log2p > kMaxLog2P)
    return noalloc_fail(err, err_len, FCS_EUNSUPPORTED, "Jt=%lld needs FFT length > %d",
                        (long long)a.m.Jt, 1 << kMaxLog2P);
  const int log2m = log2p - 1;
  const int M = 1 << log2m;
  int64_t Imax = 0, Jmax = 0, utlen = 0;
  for (int n = 0; n < N; ++n) {
    a.ut_off[n] = utlen;
    utlen += R * host_I[n];
    if (host_I[n] > Imax) Imax = host_I[n];
    if (host_J[n] > Jmax) Jmax = host_J[n];
  }
  const size_t gbytes = (sizeof(float2) * size_t(D) * size_t(M + 2) + 255) & ~size_t(255);
  const size_t cbytes = 256;
  const size_t need = gbytes + cbytes + sizeof(float) * size_t(utlen);
  if (need > kNoAllocScratchBytes)
    return noalloc_fail(err, err_len, FCS_ENOMEM_BUDGET,
                        "problem needs %zu bytes of scratch; the static scratch array holds "
                        "%zu bytes (D*(P/2+1)*8 + R*sum(I_n)*4 must fit)",
                        need, kNoAllocScratchBytes);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return noalloc_fail(err, err_len, FCS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return noalloc_fail(err, err_len, FCS_EUNSUPPORTED, "device %d beyond %d", dev,
                        kNoAllocMaxDevices);
  NoAllocDevice *sd = nullptr;
  int rc = noalloc_setup(dev, st, &sd, err, err_len);
  if (rc) return rc;

  a.D = D;
  a.R = R;
  a.h = h;
  a.s = s;
  a.out = out;
  a.sb = int((Jmax + 3) / 4 * 4);
  int64_t groups = (int64_t(sd->sm_count) + D - 1) / D;
  if (groups < 1) groups = 1;
  if (groups > R) groups = R;
  a.ranks_per_cta = (R + groups - 1) / groups;
  groups = (R + a.ranks_per_cta - 1) / a.ranks_per_cta;
  a.G = reinterpret_cast<float2 *>(sd->scratch);
  a.counter = reinterpret_cast<unsigned *>(sd->scratch + gbytes);
  float *UT = reinterpret_cast<float *>(sd->scratch + gbytes + cbytes);
  a.UT = UT;
  // the accumulator and tickets must start at zero (the array keeps the
  // previous call's contents); the same launch transposes the factors
  {
    PrepArgs pa{};
    for (int n = 0; n < N; ++n) {
      pa.t.U[n] = host_U[n];
      pa.t.I[n] = host_I[n];
      pa.t.ld[n] = host_ldU[n];
      pa.t.ut_off[n] = a.ut_off[n];
    }
    pa.t.R = R;
    pa.t.lambda = lambda;
    pa.t.UT = UT;
    pa.tiles_x = (Imax + 31) / 32;
    pa.tiles_y = (R + 31) / 32;
    pa.ntile = pa.tiles_x * pa.tiles_y * N;
    pa.zero = reinterpret_cast<float4 *>(sd->scratch);
    pa.zero_n4 = int64_t(gbytes + cbytes) / 16;
    pa.zero_blocks = int(std::min<int64_t>(64, (pa.zero_n4 + 255) / 256));
    prep_kernel<<<unsigned(pa.ntile + pa.zero_blocks), 256, 0, st>>>(pa);
    e = cudaGetLastError();
    if (e != cudaSuccess)
      return noalloc_fail(err, err_len, FCS_ECUDA, "prep: %s", cudaGetErrorString(e));
  }
  rc = FCS_EUNSUPPORTED;
  FCS_DISPATCH_LOG2M(log2m, rc = noalloc_launch_cp<L>(a, groups, Imax, sd->twiddle, st, err,
                                                      err_len));
  return rc;
}
