// fcs_fft.cuh -- the block FFT used by the sketch kernels: a forward real FFT
// of length P = 2M whose input is a sparse Count Sketch column and whose
// output half spectrum lands directly in per-thread registers.
//
// Pass plan for the length-M complex FFT (Stockham auto-sort, radices 16 and a
// tail whose last radix is <= 8):
//     M = 16^a * 2^b  ->  [16]*a + [2^b]           (b = 1..3)
//     M = 16^a        ->  [16]*(a-1) + [8, 2]
//     M = 8           ->  [4, 2]
// * The first pass reads the real scatter buffer (z[m] = x[2m] + i x[2m+1])
//   and skips the zero padding beyond the longest hash range.
// * Middle passes run in place in padded shared memory with twiddles from a
//   small shared table holding, for each k < Ns, the powers W^k, W^2k, W^4k,
//   W^8k of W = exp(-2 pi i / (Ns R)); other powers are products of those
//   (at most three roundings).
// * The last pass assigns each thread "slots" of two butterflies (j, Ns - j)
//   (slot 0 pairs butterflies 0 and Ns/2), whose outputs are closed under
//   q -> M - q.  The real-FFT unpack
//       E = (Z[q] + conj Z[M-q]) / 2,  O = (Z[q] - conj Z[M-q]) / (2i),
//       X[q] = E + W_P^q O,  X[M-q] = conj(E - W_P^q O)
//   then needs no data exchange, so the half spectrum X[0..M] of the real
//   input stays in registers (X[0] and X[M], both real, share one float2).
#pragma once

#include "fcs_internal.cuh"

namespace fcs {

__host__ __device__ constexpr int plan_npass(int L) { return L == 3 ? 2 : L / 4 + 1; }

// log2 of the radix of pass p
__host__ __device__ constexpr int plan_lr(int L, int p) {
  if (L == 3) return p == 0 ? 2 : 1;
  if (L % 4 == 0) return p < L / 4 - 1 ? 4 : (p == L / 4 - 1 ? 3 : 1);
  return p < L / 4 ? 4 : L % 4;
}

// log2 of Ns (product of the radices before pass p)
__host__ __device__ constexpr int plan_lns(int L, int p) {
  int s = 0;
  for (int q = 0; q < p; ++q) s += plan_lr(L, q);
  return s;
}

// offset (float2) of pass p's twiddle powers in the shared table; middle
// passes 1 .. npass-2 only
__host__ __device__ constexpr int plan_twoff(int L, int p) {
  int o = 0;
  for (int q = 1; q < p; ++q) o += plan_lr(L, q) << plan_lns(L, q);
  return o;
}
__host__ __device__ constexpr int plan_twlen(int L) { return plan_twoff(L, plan_npass(L) - 1); }

// Compile-time facts about the fused last pass of a length-2^L FFT run by NT
// threads.
template <int L, int NT>
struct LastPass {
  static constexpr int M = 1 << L;
  static constexpr int NP = plan_npass(L);
  static constexpr int LRL = plan_lr(L, NP - 1);
  static constexpr int RL = 1 << LRL;
  static constexpr int NS = M / RL;
  static constexpr int SLOTS = NS / 2;
  static constexpr int EPS = (SLOTS + NT - 1) / NT;    // slots per thread
  static constexpr int NV = EPS * 2 * RL;              // spectrum values per thread
};

// Fill the shared twiddle table of the middle passes from the global table
// tw[k] = exp(-2 pi i k / kTwN).
template <int L, int NT>
__device__ __forceinline__ void fill_twiddles(float2 *tws, const float2 *__restrict__ tw) {
  constexpr int NP = plan_npass(L);
#pragma unroll
  for (int p = 1; p < NP - 1; ++p) {
    const int lr = plan_lr(L, p), lns = plan_lns(L, p);
    const int n = lr << lns;
    float2 *dst = tws + plan_twoff(L, p);
    for (int e = threadIdx.x; e < n; e += NT) {
      const int b = e >> lns, k = e & ((1 << lns) - 1);
      dst[e] = __ldg(&tw[(k << b) << (kLogTwN - lns - lr)]);
    }
  }
}

// v[r] *= w^r for r = 1 .. R-1, with w^(2^b) given in wp[b].
template <int LR>
__device__ __forceinline__ void twiddle_powers(float2 *v, const float2 *wp) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int r = 1; r < R; ++r) {
    float2 w = make_float2(1.f, 0.f);
    bool first = true;
#pragma unroll
    for (int b = 0; b < LR; ++b) {
      if ((r >> b) & 1) {
        w = first ? wp[b] : cmul(w, wp[b]);
        first = false;
      }
    }
    v[r] = cmul(v[r], w);
  }
}

// First pass: radix 2^LR0 butterflies over z[m] = A[2m] + i A[2m+1] where
// the real buffer A holds `sb` floats (sb even; entries past it are zero),
// written to B in Stockham order.  No twiddles (Ns = 1).
template <int L, int NT>
__device__ __forceinline__ void fft_first_pass(const float *A, int sb, float2 *B) {
  constexpr int M = 1 << L;
  constexpr int LR = plan_lr(L, 0);
  constexpr int R = 1 << LR;
  constexpr int NB = M / R;
  constexpr int PER = (NB + NT - 1) / NT;
  const float2 *A2 = reinterpret_cast<const float2 *>(A);
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = threadIdx.x + b * NT;
    if (NB % NT == 0 || j < NB) {
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * NB;
        v[r] = (2 * m < sb) ? A2[m] : make_float2(0.f, 0.f);
      }
      Dft<R>::run(v);
      if constexpr (R == 16) {
        float2 *o = B + j * 17;              // pad(16 j + r) = 17 j + r
#pragma unroll
        for (int r = 0; r < R; ++r) o[r] = v[r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) B[pad(j * R + r)] = v[r];
      }
    }
  }
}

// Middle pass p (in place on B): load, barrier, twiddle + DFT, store, barrier.
template <int L, int NT, int P>
__device__ __forceinline__ void fft_middle_pass(float2 *B, const float2 *tws) {
  constexpr int M = 1 << L;
  constexpr int LR = plan_lr(L, P);
  constexpr int R = 1 << LR;
  constexpr int LNS = plan_lns(L, P);
  constexpr int NS = 1 << LNS;
  constexpr int NB = M / R;
  constexpr int PER = (NB + NT - 1) / NT;
  const float2 *tp = tws + plan_twoff(L, P);
  // NB and NS are multiples of 16 here, so pad(x + r*S) = pad(x) + r*(S + S/16)
  static_assert(NB % 16 == 0 && NS % 16 == 0, "middle pass strides");
  constexpr int SNB = NB + NB / 16, SNS = NS + NS / 16;
  float2 v[PER][R];
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = threadIdx.x + b * NT;
    if (NB % NT == 0 || j < NB) {
      const float2 *src = B + pad(j);
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = src[r * SNB];
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = threadIdx.x + b * NT;
    if (NB % NT == 0 || j < NB) {
      const int k = j & (NS - 1);
      float2 wp[LR];
#pragma unroll
      for (int q = 0; q < LR; ++q) wp[q] = tp[q * NS + k];
      twiddle_powers<LR>(v[b], wp);
      Dft<R>::run(v[b]);
      float2 *dst = B + pad((j - k) * R + k);
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * SNS] = v[b][r];
    }
  }
  __syncthreads();
}

template <int L, int NT, int P>
__device__ __forceinline__ void fft_middle_passes(float2 *B, const float2 *tws) {
  if constexpr (P < plan_npass(L) - 1) {
    fft_middle_pass<L, NT, P>(B, tws);
    fft_middle_passes<L, NT, P + 1>(B, tws);
  }
}

// exp(-i pi m / 32) from the 64-point constant table (m in [0, 32]).
__device__ __forceinline__ float2 unit64(int j) {
  return make_float2(cos64(j), -sin64(j));
}

// Real-FFT unpack of one pair (q, M-q) with w = W_P^q:
__device__ __forceinline__ void unpack2(float2 za, float2 zb, float2 w, float2 &xa,
                                        float2 &xb) {
  const float2 e = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
  const float2 dd = make_float2(za.x - zb.x, za.y + zb.y);
  const float2 o = make_float2(0.5f * dd.y, -0.5f * dd.x);
  const float2 t = cmul(w, o);
  xa = cadd(e, t);
  xb = cconj(csub(e, t));
}

// The twiddles of the fused last pass depend only on the thread's slots, not
// on the data: a kernel that runs many transforms loads them into registers
// once (LastPassTw::load) instead of from the global table in every last pass.
// Both twiddle sources give W_M^(u 2^b) (w0) and W_P^u (wP), P = 2M, for the
// slot u = threadIdx.x + e NT (u != 0, a live slot).
template <int L, int NT>
struct LastPassTw {
  using LPs = LastPass<L, NT>;
  float2 c0[LPs::EPS][LPs::LRL];
  float2 cP[LPs::EPS];
  __device__ __forceinline__ void load(const float2 *__restrict__ tw) {
#pragma unroll
    for (int e = 0; e < LPs::EPS; ++e) {
      const int u = threadIdx.x + e * NT;
      const bool live = u != 0 && (LPs::SLOTS % NT == 0 || u < LPs::SLOTS);
#pragma unroll
      for (int b = 0; b < LPs::LRL; ++b)
        c0[e][b] = live ? __ldg(&tw[(u << b) << (kLogTwN - L)]) : make_float2(1.f, 0.f);
      cP[e] = live ? __ldg(&tw[u << (kLogTwN - L - 1)]) : make_float2(1.f, 0.f);
    }
  }
  __device__ __forceinline__ float2 w0(int e, int b, int) const { return c0[e][b]; }
  __device__ __forceinline__ float2 wP(int e, int) const { return cP[e]; }
};

// The same twiddles parked in shared memory, [e][b or LRL for W_P][thread]:
// each thread writes and reads only its own column (no barrier needed), so a
// kernel short of registers still avoids global loads in every last pass.
template <int L, int NT>
struct LastPassTwShared {
  using LPs = LastPass<L, NT>;
  static constexpr int kLen = LPs::EPS * (LPs::LRL + 1) * NT;   // float2 entries
  const float2 *s;
  __device__ __forceinline__ static void fill(float2 *dst, const float2 *__restrict__ tw) {
    LastPassTw<L, NT> t;
    t.load(tw);
#pragma unroll
    for (int e = 0; e < LPs::EPS; ++e) {
#pragma unroll
      for (int b = 0; b < LPs::LRL; ++b) dst[(e * (LPs::LRL + 1) + b) * NT + threadIdx.x] = t.c0[e][b];
      dst[(e * (LPs::LRL + 1) + LPs::LRL) * NT + threadIdx.x] = t.cP[e];
    }
  }
  __device__ __forceinline__ float2 w0(int e, int b, int) const {
    return s[(e * (LPs::LRL + 1) + b) * NT + threadIdx.x];
  }
  __device__ __forceinline__ float2 wP(int e, int) const {
    return s[(e * (LPs::LRL + 1) + LPs::LRL) * NT + threadIdx.x];
  }
};

// The global table read inside the last pass (no registers held across it).
template <int L>
struct LastPassTwGlobal {
  const float2 *__restrict__ tw;
  __device__ __forceinline__ float2 w0(int, int b, int u) const {
    return __ldg(&tw[(u << b) << (kLogTwN - L)]);
  }
  __device__ __forceinline__ float2 wP(int, int u) const {
    return __ldg(&tw[u << (kLogTwN - L - 1)]);
  }
};

// Fused last pass + real unpack.  X[e][b][r] receives the half-spectrum value
// at index q(e, b, r) = j_b + r NS with j_0 = u, j_1 = (u ? NS - u : NS / 2),
// u = threadIdx.x + e NT (inactive slots leave zeros); q = 0 holds the packed
// pair (X[0], X[M]).
template <int L, int NT, class TW>
__device__ __forceinline__ void fft_last_pass_unpack(const float2 *B, const TW &ltw,
                                                     float2 (*X)[2][LastPass<L, NT>::RL]) {
  using LPs = LastPass<L, NT>;
  constexpr int RL = LPs::RL, LRL = LPs::LRL, NS = LPs::NS;
#pragma unroll
  for (int e = 0; e < LPs::EPS; ++e) {
    const int u = threadIdx.x + e * NT;
    float2(&z0)[RL] = X[e][0];
    float2(&z1)[RL] = X[e][1];
    if (LPs::SLOTS % NT != 0 && u >= LPs::SLOTS) {
#pragma unroll
      for (int r = 0; r < RL; ++r) z0[r] = z1[r] = make_float2(0.f, 0.f);
      continue;
    }
    const int j1 = u ? NS - u : NS / 2;
    if constexpr (NS % 16 == 0) {
      constexpr int SNS = NS + NS / 16;
      const float2 *s0 = B + pad(u), *s1 = B + pad(j1);
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        z0[r] = s0[r * SNS];
        z1[r] = s1[r * SNS];
      }
    } else {
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        z0[r] = B[pad(u + r * NS)];
        z1[r] = B[pad(j1 + r * NS)];
      }
    }
    if (u != 0) {
      // butterfly u: powers of W_M^u; butterfly NS-u: powers of
      // W_M^(NS-u) = exp(-2 pi i / RL) conj(W_M^u)
      float2 wp0[LRL], wp1[LRL];
#pragma unroll
      for (int b = 0; b < LRL; ++b) {
        wp0[b] = ltw.w0(e, b, u);
        // exp(-2 pi i 2^b / RL) = unit64(64 * 2^b / RL)
        wp1[b] = cmul(unit64((64 >> LRL) << b), cconj(wp0[b]));
      }
      twiddle_powers<LRL>(z0, wp0);
      twiddle_powers<LRL>(z1, wp1);
    } else {
      // butterfly NS/2: powers of W_M^(NS/2) = exp(-i pi / RL)
      float2 wp1[LRL];
#pragma unroll
      for (int b = 0; b < LRL; ++b) wp1[b] = unit64((32 >> LRL) << b);
      twiddle_powers<LRL>(z1, wp1);
    }
    Dft<RL>::run(z0);
    Dft<RL>::run(z1);
    float2 x0[RL], x1[RL];
    if (u != 0) {
      const float2 wP = ltw.wP(e, u);                             // W_P^u
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        // q = u + r NS; W_P^q = W_P^u exp(-i pi r / RL); partner in z1[RL-1-r]
        const float2 w = r == 0 ? wP : cmul(wP, unit64((32 >> LRL) * r));
        unpack2(z0[r], z1[RL - 1 - r], w, x0[r], x1[RL - 1 - r]);
      }
    } else {
      // butterfly 0: q = r NS; q = 0 packed reals, q = M/2 self-paired
      x0[0] = make_float2(z0[0].x + z0[0].y, z0[0].x - z0[0].y);
      x0[RL / 2] = cconj(z0[RL / 2]);
#pragma unroll
      for (int r = 1; r < RL / 2; ++r)
        unpack2(z0[r], z0[RL - r], unit64((32 >> LRL) * r), x0[r], x0[RL - r]);
      // butterfly NS/2: q = NS/2 + r NS, partner NS/2 + (RL-1-r) NS,
      // W_P^q = exp(-i pi (2r+1) / (2 RL))
#pragma unroll
      for (int r = 0; r < RL / 2; ++r)
        unpack2(z1[r], z1[RL - 1 - r], unit64((16 >> LRL) * (2 * r + 1)), x1[r],
                x1[RL - 1 - r]);
    }
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      z0[r] = x0[r];
      z1[r] = x1[r];
    }
  }
}

// Index q of register value X[e][b][r] (see fft_last_pass_unpack).
template <int L, int NT>
__device__ __forceinline__ int last_pass_index(int e, int b, int r) {
  using LPs = LastPass<L, NT>;
  const int u = threadIdx.x + e * NT;
  const int j = b == 0 ? u : (u ? LPs::NS - u : LPs::NS / 2);
  return j + r * LPs::NS;
}

// Forward real FFT of the compact real buffer A (sb floats, everything past
// them zero) into slot registers X.  Starts and ends with a barrier; A is
// cleared (float4 stores; sb a multiple of 4) once the first pass has read it.
template <int L, int NT, class TW>
__device__ __forceinline__ void rfft_to_slots(float *A, int sb, float2 *B, const float2 *tws,
                                              const TW &ltw,
                                              float2 (*X)[2][LastPass<L, NT>::RL]) {
  __syncthreads();
  fft_first_pass<L, NT>(A, sb, B);
  __syncthreads();
  for (int e = threadIdx.x; e < sb / 4; e += NT)
    reinterpret_cast<float4 *>(A)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  fft_middle_passes<L, NT, 1>(B, tws);
  fft_last_pass_unpack<L, NT>(B, ltw, X);
  __syncthreads();
}

// Same, reading the last-pass twiddles from the global table (for kernels
// whose register budget cannot keep them).
template <int L, int NT>
__device__ __forceinline__ void rfft_to_slots(float *A, int sb, float2 *B, const float2 *tws,
                                              const float2 *__restrict__ tw,
                                              float2 (*X)[2][LastPass<L, NT>::RL]) {
  rfft_to_slots<L, NT>(A, sb, B, tws, LastPassTwGlobal<L>{tw}, X);
}

// Write slot values X (a half spectrum) into B as the conjugated packed
// sequence conj(Z) of pack_pair_conj, so that a forward complex FFT of B,
// conjugated and scaled by 1/M, yields the real inverse transform.  Every
// pair (q, M-q) lives in one thread.  The caller synchronises afterwards.
template <int L, int NT>
__device__ __forceinline__ void slots_to_conj_packed(float2 *B,
                                                     const float2 (*X)[2][LastPass<L, NT>::RL],
                                                     const float2 *__restrict__ tw) {
  using LPs = LastPass<L, NT>;
  constexpr int M = 1 << L;
  constexpr int RL = LPs::RL, NS = LPs::NS;
#pragma unroll
  for (int e = 0; e < LPs::EPS; ++e) {
    const int u = threadIdx.x + e * NT;
    if (LPs::SLOTS % NT != 0 && u >= LPs::SLOTS) continue;
    if (u != 0) {
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int a = u + r * NS;                  // partner M - a is X[e][1][RL-1-r]
        if (a < M / 2)
          pack_pair_conj<L>(B, a, X[e][0][r], X[e][1][RL - 1 - r], tw);
        else
          pack_pair_conj<L>(B, M - a, X[e][1][RL - 1 - r], X[e][0][r], tw);
      }
    } else {
      pack_pair_conj<L>(B, 0, X[e][0][0], X[e][0][RL / 2], tw);
#pragma unroll
      for (int r = 1; r < RL / 2; ++r)
        pack_pair_conj<L>(B, r * NS, X[e][0][r], X[e][0][RL - r], tw);
#pragma unroll
      for (int r = 0; r < RL / 2; ++r)
        pack_pair_conj<L>(B, NS / 2 + r * NS, X[e][1][r], X[e][1][RL - 1 - r], tw);
    }
  }
}

// Shared-memory layout for kernels built on rfft_to_slots: B (padded FFT
// buffer) | twiddle table | last-pass twiddles (LastPassTwShared) | A
// (compact real input of sb floats).
template <int L>
struct FftSmem {
  static constexpr size_t up16(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t kB = 0;
  static constexpr size_t kTw = up16(sizeof(float2) * padded_len(1 << L));
  static constexpr size_t kLp = up16(kTw + sizeof(float2) * plan_twlen(L));
  static constexpr size_t kA =
      up16(kLp + sizeof(float2) * LastPassTwShared<L, fft_threads(L)>::kLen);
  static size_t bytes(int sb) { return kA + sizeof(float) * size_t(sb); }
};

// ---------------------------------------------------------------- warp-DIT engine
// A second forward real FFT for the largest size, P = 16384 (M = 8192), with
// one block barrier per transform instead of one per pass.  Decimation in
// time splits z into the 16 sub-sequences z_w[m2] = z[16 m2 + w]:
//   Z[k + 512 q1] = sum_w W16^(w q1) W_M^(w k) Y_w[k],   Y_w = FFT_512(z_w).
// Step 1 (warp-local): warp w computes Y_w, 16 values per lane, as
//   Y_w[ka + 16 kb] = sum_l W32^(l kb) W512^(l ka) sum_r W16^(r ka) z_w[l + 32 r]:
//   a radix-16 DFT over r in registers (input-pruned: rows r >= RMAX of the
//   scatter buffer are empty), the twiddle W512^(l ka), a transpose through
//   a warp-private stretch of B (__syncwarp only), then the 16 32-point DFTs
//   over l split between the two half-warps (half e takes the outputs
//   kb = 2 kk + e after one radix-2 step); Y_w goes to row w of B.
// Step 2 (after one block barrier): thread t owns column q2(t) of B, applies
//   W_M^(w q2) and the radix-16 DFT over w, which leaves Z[q2 + 512 q1] in its
//   registers.  Lane l and lane l ^ 16 hold q2 = u and 512 - u, so every
//   real-FFT unpack pair (q, M - q) spans the two lanes: each lane finishes
//   the pairs of its q1 < 8, receiving 8 values from its neighbour (q2 = 0
//   and q2 = 256 pair with themselves).
// The input is the real scatter buffer seen as z[m] = x[2m] + i x[2m+1],
// stored row-wise: z[m] at float2 index (m mod 16) ra + m / 16, ra >= sb/32.
namespace wdit {

constexpr int kL = 13;
constexpr int kM = 1 << kL;
constexpr int kNT = 512;
constexpr int kRS = 576;     // row stride of B (float2); B also serves the padded block FFT
constexpr int kTR = 18;      // row stride of the step-1 transpose (float2, even: 16-byte pairs)
constexpr int kTw2 = 16 * 32;               // start of the step-2 part of the table
constexpr int kTwLen = kTw2 + 5 * kNT;      // per-CTA twiddle table (float2)
static_assert(16 * kRS >= padded_len(kM), "B doubles as the padded block-FFT buffer");
static_assert(31 * kTR + 16 <= kRS, "transpose fits in one row of B");

// Float index of real sample h in the row-wise scatter buffer.
__device__ __forceinline__ int a_index(int h, int ra) {
  const int m = h >> 1;
  return 2 * ((m & 15) * ra + (m >> 4)) + (h & 1);
}

// Column of B owned by thread t in step 2: u = 16 (t / 32) + t mod 16 and
// half-warp e = (t / 16) mod 2 give q2 = u (e = 0) or 512 - u (e = 1; 256
// for u = 0).
__device__ __forceinline__ int q2_of(int t) {
  const int u = ((t >> 5) << 4) | (t & 15);
  return ((t >> 4) & 1) == 0 ? u : (u == 0 ? 256 : 512 - u);
}
// Column of the unpack partner (itself for q2 = 0 and 256).
__device__ __forceinline__ int q2_partner(int q2) {
  return (q2 & 255) == 0 ? q2 : 512 - q2;
}
// Spectrum index held in v[j] after step 2 by a thread owning column q2.
__device__ __forceinline__ int spectrum_index(int q2, int j) {
  return (j < 8 ? q2 : q2_partner(q2)) + 512 * j;
}

// Per-CTA twiddle table: W512^(l ka) at ka*32 + l (ka < 16, l < 32); then
// for thread t, W_M^(q2(t) 2^b) at kTw2 + b*512 + t (b < 4) and W_P^q2(t) at
// kTw2 + 4*512 + t.  Filled from the global table tw[k] = exp(-2 pi i k / 2^15).
// All loads are issued before the first store (one memory round trip).
// Called by all kNT threads.
__device__ __forceinline__ void fill_twiddles(float2 *tws, const float2 *__restrict__ tw) {
  constexpr int PER = kTwLen / kNT;
  static_assert(kTwLen % kNT == 0, "twiddle table fill");
  float2 v[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int e = threadIdx.x + k * kNT;
    if (e < kTw2) {
      const int ka = e >> 5, l = e & 31;
      v[k] = __ldg(&tw[(l * ka) << (kLogTwN - 9)]);
    } else {
      const int b = (e - kTw2) >> 9, q2 = q2_of((e - kTw2) & (kNT - 1));
      v[k] = b < 4 ? __ldg(&tw[(q2 << b) << (kLogTwN - kL)])
                   : __ldg(&tw[q2 << (kLogTwN - kL - 1)]);
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) tws[threadIdx.x + k * kNT] = v[k];
}

// Position of z[m] in a full-height row-wise buffer (ra = 512) whose rows
// are XOR-swizzled: row w holds z[16 m2 + w] at column m2 ^ w, so that 16
// consecutive m (16 rows, one column) land in distinct banks.  Read back by
// step1<16, true>.
__device__ __forceinline__ int row_pos_swz(int m) {
  const int w = m & 15;
  return w * 512 + ((m >> 4) ^ w);
}

// DFT of size R whose inputs v[NZ..R-1] are zero (input-pruned radix-2
// decimation in time; entries at or past NZ are not read).
template <int R, int NZ>
struct DftNZ {
  static __device__ __forceinline__ void run(float2 *v) {
    if constexpr (NZ >= R) {
      Dft<R>::run(v);
    } else if constexpr (NZ <= 0) {
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = make_float2(0.f, 0.f);
    } else if constexpr (NZ == 1) {
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = v[0];
    } else {
      float2 e[R / 2], o[R / 2];
#pragma unroll
      for (int k = 0; k < R / 2; ++k) {
        e[k] = v[2 * k];
        o[k] = v[2 * k + 1];
      }
      DftNZ<R / 2, (NZ + 1) / 2>::run(e);
      DftNZ<R / 2, NZ / 2>::run(o);
      DftCombine<R>::run(v, e, o);
    }
  }
};

// Step 1.  Reads (and clears) row w of the scatter buffer A2 (ra <= 32 RMAX
// float2), writes Y_w[k] to B[w kRS + k].  No block barrier inside.
// With SWZ the rows are XOR-swizzled as written by row_pos_swz (ra = 512).
template <int RMAX, bool SWZ = false>
__device__ __forceinline__ void step1(float2 *A2, int ra, float2 *B, const float2 *tws) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int lc = SWZ ? (l ^ w) : l;                 // column of m2 = l + 32 r, minus 32 r
  float2 v[16];
  float2 *row = A2 + w * ra;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int m2 = l + 32 * r;
    v[r] = (r < RMAX && m2 < ra) ? row[lc + 32 * r] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    const int m2 = l + 32 * r;
    if (m2 < ra) row[lc + 32 * r] = make_float2(0.f, 0.f);
  }
  DftNZ<16, RMAX>::run(v);
#pragma unroll
  for (int ka = 1; ka < 16; ++ka) v[ka] = cmul(v[ka], tws[ka * 32 + l]);   // W512^(l ka)
  float2 *T = B + w * kRS;
#pragma unroll
  for (int ka = 0; ka < 16; ka += 2)
    *reinterpret_cast<float4 *>(T + l * kTR + ka) =
        make_float4(v[ka].x, v[ka].y, v[ka + 1].x, v[ka + 1].y);
  __syncwarp();
  const int j = l & 15;
  const bool odd = l >= 16;
  const float sg = odd ? -1.f : 1.f;
#pragma unroll
  for (int lp = 0; lp < 16; ++lp) {
    const float2 a = T[lp * kTR + j], b = T[(lp + 16) * kTR + j];
    float2 g = make_float2(fmaf(sg, b.x, a.x), fmaf(sg, b.y, a.y));      // a + (-1)^e b
    if (lp > 0) {
      const float2 w = unit64(2 * lp);                                  // W32^(lp e)
      g = cmul(g, make_float2(odd ? w.x : 1.f, odd ? w.y : 0.f));
    }
    v[lp] = g;
  }
  Dft<16>::run(v);                                  // v[kk] = Y_w[j + 16 e + 32 kk]
  __syncwarp();
  const int k0 = j + (odd ? 16 : 0);
#pragma unroll
  for (int kk = 0; kk < 16; ++kk) T[k0 + 32 * kk] = v[kk];
}

// Step 2 up to the complex spectrum: v[q1] = Z[q2 + 512 q1], q2 = q2_of(threadIdx.x).
// RS: row stride of B (float2).
template <int RS = kRS>
__device__ __forceinline__ void step2_complex(const float2 *B, const float2 *tws,
                                              float2 (&v)[16]) {
  const int t = threadIdx.x;
  const int q2 = q2_of(t);
#pragma unroll
  for (int w = 0; w < 16; ++w) v[w] = B[w * RS + q2];
  {
    float2 wp[4];                                   // W_M^(q2 2^b)
#pragma unroll
    for (int b = 0; b < 4; ++b) wp[b] = tws[kTw2 + b * kNT + t];
    twiddle_powers<4>(v, wp);
  }
  Dft<16>::run(v);
}

// Twice the real-FFT unpack of one pair: with w = W_P^q,
// 2 X[q] = 2E + w 2O and 2 X[M - q] = conj(2E - w 2O).
__device__ __forceinline__ void unpack2_twice(float2 za, float2 zb, float2 w, float2 &xa,
                                              float2 &xb) {
  const float2 e = make_float2(za.x + zb.x, za.y - zb.y);
  const float2 o = make_float2(za.y + zb.y, zb.x - za.x);
  const float2 t = cmul(w, o);
  xa = cadd(e, t);
  xb = cconj(csub(e, t));
}

// Step 2.  Leaves in v[j] TWICE the half-spectrum value X[spectrum_index(q2, j)]
// of the real input, q2 = q2_of(threadIdx.x) (the factor 2 saves the halvings
// of the unpack; callers divide it out at the end); for thread 0, v[0] packs
// the two real bins (2 X[0], 2 X[M]).  `stash` is 16 float2 of shared scratch
// used by thread 0.  Every lane of every warp must call it (it shuffles).
template <int RS = kRS>
__device__ __forceinline__ void step2(const float2 *B, const float2 *tws, float2 *stash,
                                      float2 (&v)[16]) {
  const int t = threadIdx.x;
  step2_complex<RS>(B, tws, v);                     // v[q1] = Z[q2 + 512 q1]
  if (t == 0) {
#pragma unroll
    for (int q1 = 0; q1 < 16; ++q1) stash[q1] = v[q1];
  }
  const int lane = t & 31;
  const bool self = t < 32 && (lane & 15) == 0;     // q2 = 0 or 256
  const int src = self ? lane : (lane ^ 16);
  const float2 wP = tws[kTw2 + 4 * kNT + t];        // W_P^q2
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    // Z[M - (q2 + 512 i)] = Z[q2p + 512 (15 - i)] is the partner's v[15 - i]
    float2 zm;
    zm.x = __shfl_sync(0xffffffffu, v[15 - i].x, src);
    zm.y = __shfl_sync(0xffffffffu, v[15 - i].y, src);
    // W_P^(q2 + 512 i) = W_P^q2 exp(-2 pi i i / 32)
    const float2 wq = i == 0 ? wP : cmul(wP, unit64(2 * i));
    unpack2_twice(v[i], zm, wq, v[i], v[15 - i]);  // 2 X[q], 2 X[M - q]
  }
  if (t == 0) {
    // q2 = 0: Z[512 q1] pairs with Z[512 (16 - q1)]; q1 = 0 and 8 pair with themselves
    const float2 z0 = stash[0], z8 = stash[8];
    v[0] = make_float2(2.f * (z0.x + z0.y), 2.f * (z0.x - z0.y));
    v[8] = make_float2(2.f * z8.x, -2.f * z8.y);
#pragma unroll
    for (int q1 = 1; q1 < 8; ++q1)
      unpack2_twice(stash[q1], stash[16 - q1], unit64(2 * q1), v[q1], v[16 - q1]);
  }
}

// Step 1 for row w: the 512-point FFT of in_row (ra float2 entries; with SWZ
// column c of row w sits at c ^ w) into out_row (kRS float2, also the
// transpose scratch).  INPLACE: in_row == out_row, so the warp synchronises
// after reading its input and nothing is cleared; otherwise the entries read
// are cleared.  No block barrier inside.
template <int RMAX, bool SWZ, bool INPLACE>
__device__ __forceinline__ void step1_row(float2 *in_row, int ra, float2 *out_row,
                                          const float2 *tws, int w) {
  const int l = threadIdx.x & 31;
  const int lc = SWZ ? (l ^ w) : l;
  float2 v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int m2 = l + 32 * r;
    v[r] = (r < RMAX && m2 < ra) ? in_row[lc + 32 * r] : make_float2(0.f, 0.f);
  }
  if (INPLACE) {
    __syncwarp();
  } else {
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const int m2 = l + 32 * r;
      if (m2 < ra) in_row[lc + 32 * r] = make_float2(0.f, 0.f);
    }
  }
  DftNZ<16, RMAX>::run(v);
#pragma unroll
  for (int ka = 1; ka < 16; ++ka) v[ka] = cmul(v[ka], tws[ka * 32 + l]);   // W512^(l ka)
  float2 *T = out_row;
#pragma unroll
  for (int ka = 0; ka < 16; ka += 2)
    *reinterpret_cast<float4 *>(T + l * kTR + ka) =
        make_float4(v[ka].x, v[ka].y, v[ka + 1].x, v[ka + 1].y);
  __syncwarp();
  const int j = l & 15;
  const bool odd = l >= 16;
  const float sg = odd ? -1.f : 1.f;
#pragma unroll
  for (int lp = 0; lp < 16; ++lp) {
    const float2 a = T[lp * kTR + j], b = T[(lp + 16) * kTR + j];
    float2 g = make_float2(fmaf(sg, b.x, a.x), fmaf(sg, b.y, a.y));
    if (lp > 0) {
      const float2 wv = unit64(2 * lp);
      g = cmul(g, make_float2(odd ? wv.x : 1.f, odd ? wv.y : 0.f));
    }
    v[lp] = g;
  }
  Dft<16>::run(v);
  __syncwarp();
  const int k0 = j + (odd ? 16 : 0);
#pragma unroll
  for (int kk = 0; kk < 16; ++kk) T[k0 + 32 * kk] = v[kk];
}

// ---------------------------------------------------------------- M = 2^14
// The same decomposition for M = 16384 (P = 32768): z[32 m2 + w] for 32
// sub-sequences w of 512 points.  Step 1 runs the 512-point FFT of row w
// exactly as above (each of the 16 warps takes rows w and w + 16); step 2
// gives thread t column q2 = q2_of(t) of the 32 x 512 result, twiddles it by
// W_M^(w q2) and takes a 32-point DFT over w, so that v[q1] = Z[q2 + 512 q1];
// the real-FFT unpack pairs (q, M - q) again span lanes l and l ^ 16.
namespace w15 {

constexpr int kRows = 32;
constexpr int kM = 1 << 14;
constexpr int kTw2 = 16 * 32;               // after the step-1 table W512^(l ka)
constexpr int kTwLen = kTw2 + 6 * kNT;      // W_M^(q2 2^b), b < 5; W_P^q2

// Float index of real sample h in the 32-row scatter buffer (row m mod 32,
// column m / 32 for m = h / 2; rows of ra float2).
__device__ __forceinline__ int a_index(int h, int ra) {
  const int m = h >> 1;
  return 2 * ((m & 31) * ra + (m >> 5)) + (h & 1);
}

// Position of z[m] in a 32-row buffer of row stride kRS whose rows are
// XOR-swizzled (row w holds z[32 m2 + w] at column m2 ^ w); read back by
// step1_row<16, true, true>.
__device__ __forceinline__ int row_pos_swz(int m) {
  const int w = m & 31;
  return w * kRS + ((m >> 5) ^ w);
}

// Per-CTA twiddle table: the step-1 part as in wdit::fill_twiddles, then for
// thread t W_M^(q2(t) 2^b) at kTw2 + b*512 + t (b < 5) and W_P^q2(t) at
// kTw2 + 5*512 + t, from tw[k] = exp(-2 pi i k / 2^15).  Called by all kNT
// threads; every load is issued before the first store.
__device__ __forceinline__ void fill_twiddles(float2 *tws, const float2 *__restrict__ tw) {
  constexpr int PER = kTwLen / kNT;
  static_assert(kTwLen % kNT == 0, "twiddle table fill");
  float2 v[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int e = threadIdx.x + k * kNT;
    if (e < kTw2) {
      const int ka = e >> 5, l = e & 31;
      v[k] = __ldg(&tw[(l * ka) << (kLogTwN - 9)]);
    } else {
      const int b = (e - kTw2) >> 9, q2 = q2_of((e - kTw2) & (kNT - 1));
      v[k] = b < 5 ? __ldg(&tw[(q2 << b) << (kLogTwN - 14)]) : __ldg(&tw[q2]);
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) tws[threadIdx.x + k * kNT] = v[k];
}

// Step 2 up to the complex spectrum: v[q1] = Z[q2 + 512 q1], q2 = q2_of(t).
__device__ __forceinline__ void step2_complex(const float2 *B, const float2 *tws,
                                              float2 (&v)[32]) {
  const int t = threadIdx.x;
  const int q2 = q2_of(t);
#pragma unroll
  for (int w = 0; w < 32; ++w) v[w] = B[w * kRS + q2];
  {
    float2 wp[5];                                   // W_M^(q2 2^b)
#pragma unroll
    for (int b = 0; b < 5; ++b) wp[b] = tws[kTw2 + b * kNT + t];
    twiddle_powers<5>(v, wp);
  }
  Dft<32>::run(v);
}

// Step 2 with the real-FFT unpack: v[j] = TWICE the half-spectrum value
// X[(j < 16 ? q2 : q2_partner(q2)) + 512 j]; thread 0 holds X[512 j], with
// v[0] packing the two real bins (2 X[0], 2 X[M]).  `stash` is 32 float2 of
// shared scratch for thread 0.  Every lane of every warp must call it.
__device__ __forceinline__ void step2(const float2 *B, const float2 *tws, float2 *stash,
                                      float2 (&v)[32]) {
  const int t = threadIdx.x;
  step2_complex(B, tws, v);
  if (t == 0) {
#pragma unroll
    for (int q1 = 0; q1 < 32; ++q1) stash[q1] = v[q1];
  }
  const int lane = t & 31;
  const bool self = t < 32 && (lane & 15) == 0;     // q2 = 0 or 256
  const int src = self ? lane : (lane ^ 16);
  const float2 wP = tws[kTw2 + 5 * kNT + t];        // W_P^q2, P = 32768
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    // Z[M - (q2 + 512 i)] = Z[q2p + 512 (31 - i)] is the partner's v[31 - i]
    float2 zm;
    zm.x = __shfl_sync(0xffffffffu, v[31 - i].x, src);
    zm.y = __shfl_sync(0xffffffffu, v[31 - i].y, src);
    // W_P^(q2 + 512 i) = W_P^q2 exp(-2 pi i i / 64)
    const float2 wq = i == 0 ? wP : cmul(wP, unit64(i));
    unpack2_twice(v[i], zm, wq, v[i], v[31 - i]);
  }
  if (t == 0) {
    // q2 = 0: Z[512 q1] pairs with Z[512 (32 - q1)]; q1 = 0 and 16 pair with themselves
    const float2 z0 = stash[0], z16 = stash[16];
    v[0] = make_float2(2.f * (z0.x + z0.y), 2.f * (z0.x - z0.y));
    v[16] = make_float2(2.f * z16.x, -2.f * z16.y);
#pragma unroll
    for (int q1 = 1; q1 < 16; ++q1)
      unpack2_twice(stash[q1], stash[32 - q1], unit64(q1), v[q1], v[32 - q1]);
  }
}

}  // namespace w15

// ---------------------------------------------------------------- M = 2^12
// M = 4096 (P = 8192) on 256 threads: z[8 m2 + w] for 8 sub-sequences of
// 512 points, warp w running step 1 on row w (step1_row).  In step 2 thread t
// takes the two columns ua(t) and ub(t) = 512 - ua(t) (t = 0: columns 256
// and 0), twiddles each by W_M^(w q2), takes two 8-point DFTs, and does the
// real-FFT unpack inside the thread: bin ua + 512 q1 pairs with
// ub + 512 (7 - q1), so no data crosses lanes.
namespace w12 {

constexpr int kRows = 8;
constexpr int kM = 1 << 12;
constexpr int kNT = 256;
constexpr int kTw2 = 16 * 32;               // after the step-1 table W512^(l ka)
constexpr int kTwLen = kTw2 + 7 * kNT;      // W_M^(ua 2^b), W_M^(ub 2^b) (b < 3), W_P^ua

__device__ __forceinline__ int ua_of(int t) { return t ? t : 256; }
__device__ __forceinline__ int ub_of(int t) { return t ? 512 - t : 0; }

// Float index of real sample h in the 8-row scatter buffer (row m mod 8,
// column m / 8 for m = h / 2; rows of ra float2).
__device__ __forceinline__ int a_index(int h, int ra) {
  const int m = h >> 1;
  return 2 * ((m & 7) * ra + (m >> 3)) + (h & 1);
}

// Position of z[m] in an 8-row buffer of row stride kRS, rows XOR-swizzled
// (row w holds z[8 m2 + w] at column m2 ^ w), read back by
// step1_row<16, true, true>.
__device__ __forceinline__ int row_pos_swz(int m) {
  const int w = m & 7;
  return w * kRS + ((m >> 3) ^ w);
}

// Per-CTA twiddle table: the step-1 part (W512^(l ka) at ka*32 + l), then for
// thread t W_M^(ua 2^b) at kTw2 + b*256 + t, W_M^(ub 2^b) at
// kTw2 + (3 + b)*256 + t (b < 3) and W_P^ua at kTw2 + 6*256 + t, from
// tw[k] = exp(-2 pi i k / 2^15).  Every load is issued before the first store.
__device__ __forceinline__ void fill_twiddles(float2 *tws, const float2 *__restrict__ tw) {
  constexpr int PER = kTwLen / kNT;
  static_assert(kTwLen % kNT == 0, "twiddle table fill");
  float2 v[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int e = threadIdx.x + k * kNT;
    if (e < kTw2) {
      const int ka = e >> 5, l = e & 31;
      v[k] = __ldg(&tw[(l * ka) << (kLogTwN - 9)]);
    } else {
      const int b = (e - kTw2) >> 8, t = (e - kTw2) & (kNT - 1);
      const int ua = ua_of(t), ub = ub_of(t);
      v[k] = b < 3   ? __ldg(&tw[(ua << b) << (kLogTwN - 12)])
             : b < 6 ? __ldg(&tw[(ub << (b - 3)) << (kLogTwN - 12)])
                     : __ldg(&tw[ua << (kLogTwN - 13)]);
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) tws[threadIdx.x + k * kNT] = v[k];
}

// Step 2 up to the complex spectrum: va[q1] = Z[ua + 512 q1],
// vb[q1] = Z[ub + 512 q1].
__device__ __forceinline__ void step2_complex(const float2 *B, const float2 *tws, float2 (&va)[8],
                                              float2 (&vb)[8]) {
  const int t = threadIdx.x;
  const int ua = ua_of(t), ub = ub_of(t);
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    va[w] = B[w * kRS + ua];
    vb[w] = B[w * kRS + ub];
  }
  float2 wa[3], wb[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    wa[b] = tws[kTw2 + b * kNT + t];
    wb[b] = tws[kTw2 + (3 + b) * kNT + t];
  }
  twiddle_powers<3>(va, wa);
  twiddle_powers<3>(vb, wb);
  Dft<8>::run(va);
  Dft<8>::run(vb);
}

// Step 2 with the real-FFT unpack: TWICE the half-spectrum values,
// va[q1] = 2 X[ua + 512 q1], vb[q1] = 2 X[ub + 512 q1]; for thread 0 (ub = 0)
// vb[0] packs the two real bins (2 X[0], 2 X[M]).
__device__ __forceinline__ void step2(const float2 *B, const float2 *tws, float2 (&va)[8],
                                      float2 (&vb)[8]) {
  const int t = threadIdx.x;
  step2_complex(B, tws, va, vb);
  if (t != 0) {
    const float2 wP = tws[kTw2 + 6 * kNT + t];      // W_P^ua, P = 8192
#pragma unroll
    for (int q1 = 0; q1 < 8; ++q1) {
      // W_P^(ua + 512 q1) = W_P^ua exp(-2 pi i q1 / 16); partner ub + 512 (7 - q1)
      const float2 wq = q1 == 0 ? wP : cmul(wP, unit64(4 * q1));
      unpack2_twice(va[q1], vb[7 - q1], wq, va[q1], vb[7 - q1]);
    }
  } else {
    // column 256 pairs with itself: 256 + 512 q1 <-> 256 + 512 (7 - q1)
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1)
      unpack2_twice(va[q1], va[7 - q1], unit64(2 + 4 * q1), va[q1], va[7 - q1]);
    // column 0: 512 q1 <-> 512 (8 - q1); q1 = 0 and 4 pair with themselves
    const float2 z0 = vb[0], z4 = vb[4];
    vb[0] = make_float2(2.f * (z0.x + z0.y), 2.f * (z0.x - z0.y));
    vb[4] = make_float2(2.f * z4.x, -2.f * z4.y);
#pragma unroll
    for (int q1 = 1; q1 < 4; ++q1) unpack2_twice(vb[q1], vb[8 - q1], unit64(4 * q1), vb[q1], vb[8 - q1]);
  }
}

}  // namespace w12

}  // namespace wdit

}  // namespace fcs
