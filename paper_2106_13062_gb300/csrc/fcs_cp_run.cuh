// fcs_cp_run.cuh -- the CP-route work of one (sketch d, rank group), eq.
// (FCS_syn), shared by the single-problem kernels (fcs_cp.cu) and the batch
// kernels (fcs_batch.cu).  For each rank r and mode n the signed factor
// column is count-sketched (Def. 1) into a compact shared buffer (the zero
// padding up to P is never stored), transformed by a block real FFT whose
// output half spectrum stays in registers, and multiplied into the
// per-thread mode product; the product is added into a shared rank
// accumulator, so the rank sum stays in the frequency domain.  The next
// column's factor values and hashes are prefetched into registers while the
// current one is transformed.  The group's partial spectrum then goes into
// the sketch's global accumulator with atomics, and the group that completes
// sketch d (ticket counter) runs the one inverse real FFT and writes FCS_d.
//
// Two engines:
//   cp_run<L, NT, CPT>   P = 2^(L+1) <= 8192 on the slot FFT of fcs_fft.cuh
//                        (NT = 2^(L-4) threads, 16 points each, >= 32);
//   cp13_run<CPT, RMAX>  P = 16384 on the warp-DIT engine (wdit::, M = 2^13,
//                        512 threads, two block barriers per transform).
//
// The problem is read through a small accessor interface (Prob):
//   int modes(), int64_t dim(n), const float *column(n, r),
//   const int32_t *hashes(d, n), const int8_t *signs(d, n), int64_t length(),
//   float *sketch(d), float2 *spectrum() ([D][M + 2] float2, 16-byte
//   aligned, zero before the first group of a sketch adds into it),
//   unsigned *ticket(d) (zero at start; reset by the last group), int sb
//   (scatter-buffer length in floats: max J_n rounded up to 4).
#pragma once

#include "fcs_fft.cuh"

namespace fcs {

// Shared-memory layout of cp_run; every region starts on a 16-byte
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

// Ranks [r0, r1) of sketch d on the slot FFT (M = 2^LOG2M complex points,
// NT threads).  CPT = factor entries prefetched per thread (the rest of a
// longer column is scattered by a direct loop); `groups` = number of groups
// that add into sketch d.  Every thread of the block calls it; it returns
// with no barrier pending.
template <int LOG2M, int NT, int CPT, class Prob>
__device__ __forceinline__ void cp_run(const Prob &a, int d, int64_t r0, int64_t r1,
                                       unsigned groups, unsigned char *smem_raw,
                                       const float2 *__restrict__ tw, int *is_last) {
  using LPs = LastPass<LOG2M, NT>;
  constexpr int M = 1 << LOG2M;
  constexpr int HALF = M / 2;
  constexpr int RL = LPs::RL, EPS = LPs::EPS, NV = LPs::NV;
  using Lay = CpSmem<LOG2M, NT>;
  float2 *B = reinterpret_cast<float2 *>(smem_raw + Lay::kB);      // padded_len(M)
  float2 *accS = reinterpret_cast<float2 *>(smem_raw + Lay::kAcc); // NV * NT
  float2 *tws = reinterpret_cast<float2 *>(smem_raw + Lay::kTw);   // plan_twlen
  float *A = reinterpret_cast<float *>(smem_raw + Lay::kA);        // sb floats
  const int tid = threadIdx.x;
  const int N = a.modes();
  const int sb = a.sb;

  fill_twiddles<LOG2M, NT>(tws, tw);
  LastPassTw<LOG2M, NT> ltw;
  ltw.load(tw);
  for (int e = tid; e < sb / 4; e += NT) reinterpret_cast<float4 *>(A)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int v = 0; v < NV; ++v) accS[v * NT + tid] = make_float2(0.f, 0.f);

  // prefetched column: signed factor values and hash bins
  float pv[CPT];
  int ph[CPT];
  auto fetch = [&](int64_t r, int n) {
    const int64_t In = a.dim(n);
    const float *col = a.column(n, r);
    const int32_t *hn = a.hashes(d, n);
    const int8_t *sn = a.signs(d, n);
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int64_t i = tid + int64_t(c) * NT;
      ph[c] = -1;
      pv[c] = 0.f;
      if (i < In) {
        const float v = a.ld(col + i);
        pv[c] = a.ld(sn + i) < 0 ? -v : v;
        ph[c] = a.ld(hn + i);
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
      const int64_t In = a.dim(n);
      if (In > int64_t(CPT) * NT) {
        // entries beyond the prefetched chunk: load and scatter directly
        const float *col = a.column(n, r);
        const int32_t *hn = a.hashes(d, n);
        const int8_t *sn = a.signs(d, n);
        for (int64_t i = int64_t(CPT) * NT + tid; i < In; i += NT) {
          const int hb = a.ld(hn + i);
          const float v = a.ld(col + i);
          if (unsigned(hb) < unsigned(sb)) atomicAdd(A + hb, a.ld(sn + i) < 0 ? -v : v);
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
      fft_last_pass_unpack<LOG2M, NT>(B, ltw, X);
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
  float2 *Gd = a.spectrum() + d * int64_t(M + 2);
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
  unsigned *ticket = a.ticket(d);
  if (tid == 0) *is_last = (atomicAdd(ticket, 1u) == groups - 1);
  __syncthreads();
  if (!*is_last) return;
  __threadfence();

  // last group for sketch d: one inverse real FFT of the summed spectrum
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
  float *od = a.sketch(d);
  const int64_t Jt = a.length();
  float *Br = reinterpret_cast<float *>(B);
  for (int64_t j = tid; j < Jt; j += NT) {
    const float v = Br[real_off(int(j))];
    od[j] = (j & 1) ? -v * sc : v * sc;
  }
  if (tid == 0) *ticket = 0u;
}

// Shared-memory layout of cp13_run; every region starts on a 16-byte
// boundary.  ra = number of float2 columns of the scatter buffer.
struct Cp13Smem {
  static constexpr size_t kB = 0;                                   // 16 x kRS float2
  static constexpr size_t kAcc = kB + sizeof(float2) * 16 * wdit::kRS;
  static constexpr size_t kTw = kAcc + sizeof(float2) * 16 * wdit::kNT;
  static constexpr size_t kStash = kTw + sizeof(float2) * wdit::kTwLen;
  static constexpr size_t kA = kStash + sizeof(float2) * 16;
  static size_t bytes(int ra) { return kA + sizeof(float2) * 16 * size_t(ra); }
};

// Ranks [r0, r1) of sketch d on the warp-DIT engine.  CPT and `groups` as
// for cp_run; RMAX = number of 32-entry blocks per scatter-buffer row
// (ra <= 32 RMAX).  The next column is scattered into the row-wise buffer
// between the two barriers of a transform, overlapping step 2 of the
// current one.  Every thread of the 512-thread
// block calls it; it returns with no barrier pending.
template <int CPT, int RMAX, class Prob>
__device__ __forceinline__ void cp13_run(const Prob &a, int d, int64_t r0, int64_t r1,
                                         unsigned groups, unsigned char *smem_raw,
                                         const float2 *__restrict__ tw, int *is_last) {
  constexpr int NT = wdit::kNT, M = wdit::kM, HALF = M / 2;
  float2 *B = reinterpret_cast<float2 *>(smem_raw + Cp13Smem::kB);
  float4 *acc4 = reinterpret_cast<float4 *>(smem_raw + Cp13Smem::kAcc);   // [8][NT] pairs
  float2 *tws = reinterpret_cast<float2 *>(smem_raw + Cp13Smem::kTw);
  float2 *stash = reinterpret_cast<float2 *>(smem_raw + Cp13Smem::kStash);
  float2 *A2 = reinterpret_cast<float2 *>(smem_raw + Cp13Smem::kA);
  float *A = reinterpret_cast<float *>(A2);
  const int tid = threadIdx.x;
  const int N = a.modes();
  const int sb = a.sb;
  const int ra = (sb + 31) >> 5;

  float pv[CPT];
  int ph[CPT];
  auto fetch = [&](int64_t r, int n) {
    const int64_t In = a.dim(n);
    const float *col = a.column(n, r);
    const int32_t *hn = a.hashes(d, n);
    const int8_t *sn = a.signs(d, n);
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int64_t i = tid + int64_t(c) * NT;
      ph[c] = -1;
      pv[c] = 0.f;
      if (i < In) {
        const float v = a.ld(col + i);
        pv[c] = a.ld(sn + i) < 0 ? -v : v;
        ph[c] = a.ld(hn + i);
      }
    }
  };
  // scatter the fetched column (and, for I_n > CPT NT, the rest of it)
  auto scatter = [&](int64_t r, int n) {
#pragma unroll
    for (int c = 0; c < CPT; ++c)
      if (unsigned(ph[c]) < unsigned(sb)) atomicAdd(A + wdit::a_index(ph[c], ra), pv[c]);
    const int64_t In = a.dim(n);
    if (In > int64_t(CPT) * NT) {
      const float *col = a.column(n, r);
      const int32_t *hn = a.hashes(d, n);
      const int8_t *sn = a.signs(d, n);
      for (int64_t i = int64_t(CPT) * NT + tid; i < In; i += NT) {
        const int hb = a.ld(hn + i);
        const float v = a.ld(col + i);
        if (unsigned(hb) < unsigned(sb))
          atomicAdd(A + wdit::a_index(hb, ra), a.ld(sn + i) < 0 ? -v : v);
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
  float2 *Gd = a.spectrum() + d * int64_t(M + 2);
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
  unsigned *ticket = a.ticket(d);
  if (tid == 0) *is_last = (atomicAdd(ticket, 1u) == groups - 1);
  __syncthreads();
  if (!*is_last) return;
  __threadfence();

  // last group for sketch d: one inverse real FFT of the summed spectrum on
  // the same engine.  The conj-packed sequence goes row-wise (ra = 512) into
  // the accumulator region; a forward complex FFT, conj and scaling give FCS_d.
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
  float *od = a.sketch(d);
  const int64_t Jt = a.length();
  const int q2 = wdit::q2_of(tid);
#pragma unroll
  for (int q1 = 0; q1 < 16; ++q1) {
    const int64_t m = q2 + 512 * q1;
    if (2 * m < Jt) od[2 * m] = v[q1].x * sc;
    if (2 * m + 1 < Jt) od[2 * m + 1] = -v[q1].y * sc;
  }
  if (tid == 0) *ticket = 0u;
}

// Shared-memory layout of cp12_run; ra = number of float2 columns of the
// 8-row scatter buffer.
struct Cp12Smem {
  static constexpr size_t kB = 0;                                   // 8 x kRS float2
  static constexpr size_t kTw = kB + sizeof(float2) * 8 * wdit::kRS;
  static constexpr size_t kA = kTw + sizeof(float2) * wdit::w12::kTwLen;
  static size_t bytes(int ra) { return kA + sizeof(float2) * 8 * size_t(ra); }
};

// Ranks [r0, r1) of sketch d for P = 8192 on the warp-DIT engine of
// wdit::w12 (256 threads): per transform the Count Sketch goes into an 8-row
// scatter buffer, warp w runs the 512-point FFT of row w, one block barrier,
// then each thread transforms its two columns and unpacks them in registers
// (TWICE the spectrum values, so the inverse scales by 2^-N).  The mode
// product and the rank sum stay in registers; the next column is scattered
// between the barriers by half the warps before step 2 and half after.  CPT
// and `groups` as for cp_run; RMAX = number of 32-entry blocks per
// scatter-buffer row (ra <= 32 RMAX).  Every thread of the 256-thread block
// calls it; it returns with no barrier pending.
template <int CPT, int RMAX, class Prob>
__device__ __forceinline__ void cp12_run(const Prob &a, int d, int64_t r0, int64_t r1,
                                         unsigned groups, unsigned char *smem_raw,
                                         const float2 *__restrict__ tw, int *is_last) {
  namespace W = wdit::w12;
  constexpr int NT = W::kNT, M = W::kM, HALF = M / 2;
  float2 *B = reinterpret_cast<float2 *>(smem_raw + Cp12Smem::kB);
  float2 *tws = reinterpret_cast<float2 *>(smem_raw + Cp12Smem::kTw);
  float2 *A2 = reinterpret_cast<float2 *>(smem_raw + Cp12Smem::kA);
  float *A = reinterpret_cast<float *>(A2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = a.modes();
  const int sb = a.sb;
  const int ra = (sb + 15) >> 4;
  const int ua = W::ua_of(tid), ub = W::ub_of(tid);

  float pv[CPT];
  int ph[CPT];
  auto fetch = [&](int64_t r, int n) {
    const int64_t In = a.dim(n);
    const float *col = a.column(n, r);
    const int32_t *hn = a.hashes(d, n);
    const int8_t *sn = a.signs(d, n);
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int64_t i = tid + int64_t(c) * NT;
      ph[c] = -1;
      pv[c] = 0.f;
      if (i < In) {
        const float v = a.ld(col + i);
        pv[c] = a.ld(sn + i) < 0 ? -v : v;
        ph[c] = a.ld(hn + i);
      }
    }
  };
  auto scatter = [&](int64_t r, int n) {
#pragma unroll
    for (int c = 0; c < CPT; ++c)
      if (unsigned(ph[c]) < unsigned(sb)) atomicAdd(A + W::a_index(ph[c], ra), pv[c]);
    const int64_t In = a.dim(n);
    if (In > int64_t(CPT) * NT) {
      const float *col = a.column(n, r);
      const int32_t *hn = a.hashes(d, n);
      const int8_t *sn = a.signs(d, n);
      for (int64_t i = int64_t(CPT) * NT + tid; i < In; i += NT) {
        const int hb = a.ld(hn + i);
        const float v = a.ld(col + i);
        if (unsigned(hb) < unsigned(sb))
          atomicAdd(A + W::a_index(hb, ra), a.ld(sn + i) < 0 ? -v : v);
      }
    }
  };
  fetch(r0, 0);
  W::fill_twiddles(tws, tw);
  for (int e = tid; e < 8 * ra; e += NT) A2[e] = make_float2(0.f, 0.f);
  __syncthreads();
  scatter(r0, 0);
  __syncthreads();

  float2 pa[8], pb[8], acca[8], accb[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acca[j] = accb[j] = make_float2(0.f, 0.f);
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
      __syncthreads();
      const bool early = tid < NT / 2;
      if (more && early) scatter(rn, nn);
      float2 va[8], vb[8];
      W::step2(B, tws, va, vb);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (n == 0) {
          pa[j] = va[j];
          pb[j] = vb[j];
        } else {
          pa[j] = cmul(pa[j], va[j]);
          pb[j] = slot_mul(pb[j], vb[j], tid == 0 && j == 0);
        }
      }
      if (n == N - 1) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          acca[j] = cadd(acca[j], pa[j]);
          accb[j] = cadd(accb[j], pb[j]);
        }
      }
      if (more && !early) scatter(rn, nn);
      __syncthreads();
    }
  }

  // publish the partial spectrum: bins ua + 512 j and ub + 512 j (thread 0:
  // ub = 0, whose j = 0 value packs the real bins 0 and M)
  float2 *Gd = a.spectrum() + d * int64_t(M + 2);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    atomicAdd(&Gd[ua + 512 * j], acca[j]);
    if (tid == 0 && j == 0) {
      atomicAdd(&Gd[0].x, accb[0].x);
      atomicAdd(&Gd[M].x, accb[0].y);
    } else {
      atomicAdd(&Gd[ub + 512 * j], accb[j]);
    }
  }
  __threadfence();
  __syncthreads();
  unsigned *ticket = a.ticket(d);
  if (tid == 0) *is_last = (atomicAdd(ticket, 1u) == groups - 1);
  __syncthreads();
  if (!*is_last) return;
  __threadfence();

  // last group for sketch d: the conj-packed sequence of the summed spectrum,
  // row-swizzled into B, a forward complex FFT in place, conj and scaling
  {
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
        Wv[k] = __ldg(&tw[q << (kLogTwN - 13)]);      // W_P^q, P = 8192
      }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int q = k * NT + tid;
      float2 cq, cm;
      pack_pair_conj_values_w(q, Av[k], Bv[k], Wv[k], cq, cm);
      B[W::row_pos_swz(q)] = cq;
      B[W::row_pos_swz(q ? M - q : HALF)] = cm;
    }
  }
  __syncthreads();
  wdit::step1_row<16, true, true>(B + warp * wdit::kRS, 512, B + warp * wdit::kRS, tws, warp);
  __syncthreads();
  float2 va[8], vb[8];
  W::step2_complex(B, tws, va, vb);                  // Z[ua + 512 q1], Z[ub + 512 q1]
  // 1/M of the inverse and 2^-N for the doubled unpack of every mode
  const float sc = 1.0f / (float(M) * float(1 << N));
  float *od = a.sketch(d);
  const int64_t Jt = a.length();
#pragma unroll
  for (int q1 = 0; q1 < 8; ++q1) {
    const int64_t ma = ua + 512 * q1, mb = ub + 512 * q1;
    if (2 * ma < Jt) od[2 * ma] = va[q1].x * sc;
    if (2 * ma + 1 < Jt) od[2 * ma + 1] = -va[q1].y * sc;
    if (2 * mb < Jt) od[2 * mb] = vb[q1].x * sc;
    if (2 * mb + 1 < Jt) od[2 * mb + 1] = -vb[q1].y * sc;
  }
  if (tid == 0) *ticket = 0u;
}

}  // namespace fcs
