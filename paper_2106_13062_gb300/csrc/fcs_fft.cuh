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

// Fused last pass + real unpack.  X[e][b][r] receives the half-spectrum value
// at index q(e, b, r) = j_b + r NS with j_0 = u, j_1 = (u ? NS - u : NS / 2),
// u = threadIdx.x + e NT (inactive slots leave zeros); q = 0 holds the packed
// pair (X[0], X[M]).
template <int L, int NT>
__device__ __forceinline__ void fft_last_pass_unpack(const float2 *B,
                                                     const float2 *__restrict__ tw,
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
        wp0[b] = __ldg(&tw[(u << b) << (kLogTwN - L)]);
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
      const float2 wP = __ldg(&tw[u << (kLogTwN - L - 1)]);       // W_P^u
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
template <int L, int NT>
__device__ __forceinline__ void rfft_to_slots(float *A, int sb, float2 *B, const float2 *tws,
                                              const float2 *__restrict__ tw,
                                              float2 (*X)[2][LastPass<L, NT>::RL]) {
  __syncthreads();
  fft_first_pass<L, NT>(A, sb, B);
  __syncthreads();
  for (int e = threadIdx.x; e < sb / 4; e += NT)
    reinterpret_cast<float4 *>(A)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  fft_middle_passes<L, NT, 1>(B, tws);
  fft_last_pass_unpack<L, NT>(B, tw, X);
  __syncthreads();
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
// buffer) | twiddle table | A (compact real input of sb floats).
template <int L>
struct FftSmem {
  static constexpr size_t up16(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t kB = 0;
  static constexpr size_t kTw = up16(sizeof(float2) * padded_len(1 << L));
  static constexpr size_t kA = up16(kTw + sizeof(float2) * plan_twlen(L));
  static size_t bytes(int sb) { return kA + sizeof(float) * size_t(sb); }
};

}  // namespace fcs
