// fcs_internal.cuh -- shared host/device pieces of libfcs (not part of the ABI).
//
// Device building blocks:
//   * complex helpers on float2,
//   * in-register DFTs of size 2..32 (radix-2 decimation in time, constant
//     twiddles folded at compile time),
//   * a block-wide complex FFT of length M = 2^LOG2M held in shared memory in
//     natural order, computed by Stockham auto-sort passes of radix 16 (and
//     one smaller remainder pass), with twiddles read from a FP64-derived
//     table,
//   * the real-FFT pack/unpack of a length-P real signal through a length
//     M = P/2 complex FFT,
//   * small fixed-size median networks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/fcs.h"

// ---------------------------------------------------------------- context
struct fcs_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = (size_t)-1;
  int sm_count = 0;
  float2 *twiddle = nullptr;     // kTwN entries: exp(-2 pi i k / kTwN)
  void *ws = nullptr;            // workspace, grown on demand
  size_t ws_bytes = 0;
  size_t plan_bytes = 0;         // device bytes held by live batch plans
  struct fcs_batch_state *batch = nullptr;   // autotune cache (fcs_batch.cu)
  struct fcs_spec_cache *spec_cache = nullptr;   // sketch spectra (fcs_contract.cu)
  bool cache_spectra = false;                    // fcs_cache_spectra
  float *raw = nullptr;          // per-sketch estimates of long contractions
  size_t raw_bytes = 0;
  void *algo = nullptr;          // scratch of fcs_rtpm / fcs_als
  size_t algo_bytes = 0;
  cudaEvent_t switch_ev = nullptr;   // orders a new stream after the old one
  void *stage = nullptr;             // device staging of fcs_sketch_cp_host
  size_t stage_bytes = 0;
  std::string err;
};

namespace fcs {

constexpr int kLogTwN = 15;            // twiddle table resolution 2^15
constexpr int kTwN = 1 << kLogTwN;
constexpr int kMaxN = 8;
constexpr int kMaxD = 16;
constexpr int kMaxLog2P = 14;          // FFT length P <= 16384 in one CTA
constexpr int kMaxLog2PBig = 20;       // longer transforms through global memory
constexpr int kMinLog2P = 4;

int set_error(fcs_ctx *ctx, int code, const char *fmt, ...);
void batch_state_destroy(fcs_ctx *ctx);
// Spectrum cache of fcs_contract: drop the entries whose key lies in
// [p, p + bytes) (after the work that still reads them), or all of them.
void spec_cache_invalidate(fcs_ctx *ctx, const void *p, size_t bytes);
void spec_cache_destroy(fcs_ctx *ctx);
int check_cuda(fcs_ctx *ctx, cudaError_t e, const char *what);
// Grow a context-owned device buffer (*buf, *have bytes) to at least `bytes`
// (rounded up to 256; contents are not kept), ordered on the context's
// stream: the old buffer is released once the work queued before the call
// has run, and the new one is ready for the work queued after it, with no
// host wait and no device synchronisation.  Refused (FCS_EINVAL) while the
// stream is being captured: make the same call once before capturing.
int grow_buffer(fcs_ctx *ctx, void **buf, size_t *have, size_t bytes, const char *what);
// Grow the workspace to at least `bytes` (contents are not preserved).
int ensure_workspace(fcs_ctx *ctx, size_t bytes, void **out);
// Grow ctx->raw to at least `bytes` (counted against the budget with the workspace).
int ensure_raw(fcs_ctx *ctx, size_t bytes);


// RAII guard that makes ctx->device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool switched = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      switched = cudaSetDevice(dev) == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (switched) cudaSetDevice(prev);
  }
};

inline int ilog2_ceil(int64_t x) {
  int l = 0;
  while ((int64_t(1) << l) < x) ++l;
  return l;
}

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return make_float2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) {
  return make_float2(a.x * s, a.y * s);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulconj(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// Padded shared-memory index: one float2 of padding after every 16, so that
// the stride-16 writes of a first radix-16 pass hit distinct banks.
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int m) { return m + (m >> 4); }

// cos(2 pi j / 64) for j = 0..16 (quarter wave).
__host__ __device__ constexpr float cos64_q(int j) {
  constexpr float t[17] = {
      1.0f, 0.99518472667219693f, 0.98078528040323043f, 0.95694033573220882f,
      0.92387953251128674f, 0.88192126434835505f, 0.83146961230254524f,
      0.77301045336273699f, 0.70710678118654757f, 0.63439328416364549f,
      0.55557023301960229f, 0.47139673682599781f, 0.38268343236508984f,
      0.29028467725446233f, 0.19509032201612833f, 0.09801714032956077f, 0.0f};
  return t[j];
}
// cos and sin of 2 pi j / 64 for j in [0, 32] (half wave suffices here).
__host__ __device__ constexpr float cos64(int j) {
  return j <= 16 ? cos64_q(j) : -cos64_q(32 - j);
}
__host__ __device__ constexpr float sin64(int j) {
  return j <= 16 ? cos64_q(16 - j) : cos64_q(j - 16);
}

// tan(2 pi j / 64) for j = 0..8.
__host__ __device__ constexpr float tan64_q(int j) {
  constexpr float t[9] = {0.0f,
                          0.09849140335716425f,
                          0.198912367379658f,
                          0.3033466836073424f,
                          0.41421356237309503f,
                          0.5345111359507916f,
                          0.6681786379192989f,
                          0.8206787908286602f,
                          1.0f};
  return t[j];
}

// Radix-2 butterfly a' = a + W b, b' = a - W b with W = exp(-2 pi i J / 64),
// 0 < J < 32, J != 16, in six FMAs: with c = cos, s = sin of 2 pi J / 64,
//   W b = c (b.x + (s/c) b.y, b.y - (s/c) b.x)   when |c| >= |s|,
//   W b = s ((c/s) b.x + b.y, (c/s) b.y - b.x)   otherwise,
// so the ratio is a tangent of magnitude <= 1.
template <int J>
__device__ __forceinline__ void bfly_tw(float2 &a, float2 &b) {
  static_assert(J > 0 && J < 32 && J != 16, "twiddle index");
  float f, ux, uy;
  if constexpr (J <= 8 || J >= 24) {
    constexpr float t = J <= 8 ? tan64_q(J) : -tan64_q(32 - J);     // s / c
    f = cos64(J);
    ux = fmaf(t, b.y, b.x);
    uy = fmaf(-t, b.x, b.y);
  } else {
    constexpr float k = J <= 16 ? tan64_q(16 - J) : -tan64_q(J - 16);   // c / s
    f = sin64(J);
    ux = fmaf(k, b.x, b.y);
    uy = fmaf(k, b.y, -b.x);
  }
  const float2 a0 = a;
  a = make_float2(fmaf(f, ux, a0.x), fmaf(f, uy, a0.y));
  b = make_float2(fmaf(-f, ux, a0.x), fmaf(-f, uy, a0.y));
}

// Last radix-2 stage of an R-point DFT from the half-size DFTs e (even
// inputs) and o (odd inputs): v[k] = e[k] + W_R^k o[k], v[k + R/2] =
// e[k] - W_R^k o[k], unrolled over k by template recursion.
template <int R, int K = 0>
struct DftCombine {
  static __device__ __forceinline__ void run(float2 *v, const float2 *e, const float2 *o) {
    if constexpr (K < R / 2) {
      float2 a = e[K], b = o[K];
      if constexpr (K == 0) {
        v[K] = cadd(a, b);
        v[K + R / 2] = csub(a, b);
      } else if constexpr (4 * K == R) {                 // W = -i
        const float2 t = make_float2(b.y, -b.x);
        v[K] = cadd(a, t);
        v[K + R / 2] = csub(a, t);
      } else {
        bfly_tw<K * (64 / R)>(a, b);
        v[K] = a;
        v[K + R / 2] = b;
      }
      DftCombine<R, K + 1>::run(v, e, o);
    }
  }
};

// In-register forward DFT of size R (R a power of two, R <= 32), natural
// order in and out: X[k] = sum_n x[n] exp(-2 pi i n k / R).
template <int R>
struct Dft {
  static __device__ __forceinline__ void run(float2 *v) {
    float2 e[R / 2], o[R / 2];
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      e[k] = v[2 * k];
      o[k] = v[2 * k + 1];
    }
    Dft<R / 2>::run(e);
    Dft<R / 2>::run(o);
    DftCombine<R>::run(v, e, o);
  }
};
template <>
struct Dft<1> {
  static __device__ __forceinline__ void run(float2 *) {}
};

// One Stockham auto-sort pass of radix R over a length-M sequence in padded
// shared memory (in place: every thread loads its butterflies, the block
// synchronises, then stores).  Ns = product of the radices already applied.
// Butterfly j reads x[j + r M/R], multiplies by exp(-2 pi i r (j mod Ns) /
// (Ns R)), takes the R-point DFT and writes output r to
// (j / Ns) Ns R + (j mod Ns) + r Ns.
template <int M, int NT, int R>
__device__ __forceinline__ void stockham_pass(float2 *buf, int Ns, int log2NsR,
                                              const float2 *__restrict__ tw) {
  constexpr int NB = M / R;
  constexpr int PER = (NB + NT - 1) / NT;
  constexpr int LR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
  static_assert((1 << LR) == R, "radix 2, 4, 8 or 16");
  float2 v[PER][R];
  // W^(k 2^e), e < log2 R: loaded with the data, before the barrier; the
  // other powers are products of at most log2 R of them
  float2 wp[PER][LR];
  const int tid = threadIdx.x;
  const int shift = kLogTwN - log2NsR;
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = tid + b * NT;
    if (NB % NT == 0 || j < NB) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = buf[pad(j + r * NB)];
      const int k = j & (Ns - 1);
#pragma unroll
      for (int e = 0; e < LR; ++e)
        wp[b][e] = Ns > 1 ? __ldg(&tw[(k << e) << shift]) : make_float2(1.f, 0.f);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = tid + b * NT;
    if (NB % NT == 0 || j < NB) {
      const int k = j & (Ns - 1);
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = make_float2(1.f, 0.f);
          bool first = true;
#pragma unroll
          for (int e = 0; e < LR; ++e) {
            if ((r >> e) & 1) {
              w = first ? wp[b][e] : cmul(w, wp[b][e]);
              first = false;
            }
          }
          v[b][r] = cmul(v[b][r], w);
        }
      }
      Dft<R>::run(v[b]);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[pad(base + r * Ns)] = v[b][r];
    }
  }
  __syncthreads();
}

// Block-wide forward complex FFT of length M = 2^LOG2M, natural order in and
// out, in padded shared memory.  All NT threads of the block must call it;
// the caller synchronises before (data written) -- the function ends synced.
template <int LOG2M, int NT>
__device__ __forceinline__ void block_fft(float2 *buf, const float2 *__restrict__ tw) {
  constexpr int M = 1 << LOG2M;
  constexpr int N16 = LOG2M / 4;       // radix-16 passes
  constexpr int REM = LOG2M % 4;       // remainder pass radix 2^REM, last
  int Ns = 1, l = 0;
  if constexpr (N16 > 0) {
#pragma unroll
    for (int p = 0; p < N16; ++p) {
      stockham_pass<M, NT, 16>(buf, Ns, l + 4, tw);
      Ns <<= 4;
      l += 4;
    }
  }
  if constexpr (REM == 1) stockham_pass<M, NT, 2>(buf, Ns, l + 1, tw);
  if constexpr (REM == 2) stockham_pass<M, NT, 4>(buf, Ns, l + 2, tw);
  if constexpr (REM == 3) stockham_pass<M, NT, 8>(buf, Ns, l + 3, tw);
}

// ---------------------------------------------------------------- real FFT
// A real signal x of length P = 2M is held as the complex sequence
// z[m] = x[2m] + i x[2m+1] (so the real buffer and the complex buffer are the
// same memory, up to padding).  After Z = FFT_M(z), the half spectrum
// X[0..M] of x is recovered pairwise:  for 0 < q < M/2,
//   E = (Z[q] + conj Z[M-q]) / 2,  O = (Z[q] - conj Z[M-q]) / (2i),
//   X[q] = E + W^q O,  X[M-q] = conj(E - W^q O),   W = exp(-2 pi i / P);
// q = 0 gives the two real bins X[0] = Re Z0 + Im Z0, X[M] = Re Z0 - Im Z0
// (packed as one float2 "slot A"), and X[M/2] = conj Z[M/2] ("slot B").
// Slot A of pair q is X[q] (or the packed reals), slot B is X[M-q] (or X[M/2]).

// Offset (in floats) of real sample p inside the padded complex buffer.
__device__ __forceinline__ int real_off(int p) { return 2 * pad(p >> 1) + (p & 1); }

template <int LOG2M>
__device__ __forceinline__ void unpack_pair(const float2 *buf, int q,
                                            const float2 *__restrict__ tw,
                                            float2 &A, float2 &B) {
  constexpr int M = 1 << LOG2M;
  if (q == 0) {
    const float2 z0 = buf[pad(0)];
    A = make_float2(z0.x + z0.y, z0.x - z0.y);
    B = cconj(buf[pad(M / 2)]);
  } else {
    const float2 zq = buf[pad(q)];
    const float2 zm = buf[pad(M - q)];
    const float2 e = make_float2(0.5f * (zq.x + zm.x), 0.5f * (zq.y - zm.y));
    // o = (zq - conj zm) / (2i)
    const float2 dd = make_float2(zq.x - zm.x, zq.y + zm.y);
    const float2 o = make_float2(0.5f * dd.y, -0.5f * dd.x);
    const float2 w = __ldg(&tw[q << (kLogTwN - LOG2M - 1)]);
    const float2 t = cmul(w, o);
    A = cadd(e, t);
    B = cconj(csub(e, t));
  }
}

// Inverse of unpack_pair: from the half spectrum slots (A, B) of pair q,
// write conj(Z[q]) and conj(Z[M-q]) into buf so that a forward FFT followed
// by conj and 1/M scaling yields z (hence x).  With
//   E = (X[q] + conj X[M-q]) / 2,  O = (X[q] - conj X[M-q]) conj(W^q) / 2,
//   Z[q] = E + i O,  Z[M-q] = conj(E) + i conj(O).
// The two values pack_pair_conj writes for pair q: cq goes to position q and
// cm to position M - q (for q = 0: positions 0 and M/2).
// w = W_P^q (unused for q = 0).
__device__ __forceinline__ void pack_pair_conj_values_w(int q, float2 A, float2 B, float2 w,
                                                        float2 &cq, float2 &cm) {
  if (q == 0) {
    const float e = 0.5f * (A.x + A.y), o = 0.5f * (A.x - A.y);
    cq = make_float2(e, -o);                   // conj(e + i o)
    cm = B;                                    // Z[M/2] = conj(X[M/2]); conj again
  } else {
    const float2 e = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
    const float2 dd = make_float2(0.5f * (A.x - B.x), 0.5f * (A.y + B.y));
    const float2 o = cmulconj(dd, w);
    // Z[q] = e + i o = (e.x - o.y, e.y + o.x);  Z[M-q] = conj(e) + i conj(o)
    cq = make_float2(e.x - o.y, -(e.y + o.x));
    cm = make_float2(e.x + o.y, -(o.x - e.y));
  }
}

template <int LOG2M>
__device__ __forceinline__ void pack_pair_conj_values(int q, float2 A, float2 B,
                                                      const float2 *__restrict__ tw,
                                                      float2 &cq, float2 &cm) {
  const float2 w = q ? __ldg(&tw[q << (kLogTwN - LOG2M - 1)]) : make_float2(1.f, 0.f);
  pack_pair_conj_values_w(q, A, B, w, cq, cm);
}

template <int LOG2M>
__device__ __forceinline__ void pack_pair_conj(float2 *buf, int q, float2 A, float2 B,
                                               const float2 *__restrict__ tw) {
  constexpr int M = 1 << LOG2M;
  float2 cq, cm;
  pack_pair_conj_values<LOG2M>(q, A, B, tw, cq, cm);
  buf[pad(q)] = cq;
  buf[pad(q ? M - q : M / 2)] = cm;
}

// Product of two slot values; slot A of pair 0 packs two reals.
__device__ __forceinline__ float2 slot_mul(float2 a, float2 b, bool packed_reals) {
  return packed_reals ? make_float2(a.x * b.x, a.y * b.y) : cmul(a, b);
}
// a * conj(b) for slots.
__device__ __forceinline__ float2 slot_mulconj(float2 a, float2 b, bool packed_reals) {
  return packed_reals ? make_float2(a.x * b.x, a.y * b.y) : cmulconj(a, b);
}

// ---------------------------------------------------------------- median
// Median of D values held in registers (sorted in place by a fixed
// insertion network; even D -> mean of the two middle values).
template <int D>
__device__ __forceinline__ float median_inplace(float *v) {
#pragma unroll
  for (int i = 1; i < D; ++i) {
#pragma unroll
    for (int j = i; j > 0; --j) {
      const float a = v[j - 1], b = v[j];
      v[j - 1] = fminf(a, b);
      v[j] = fmaxf(a, b);
    }
  }
  if (D & 1) return v[D / 2];
  return 0.5f * (v[D / 2 - 1] + v[D / 2]);
}

// Batcher's odd-even merge sorting network for D values (comparators listed
// at compile time as (a << 6) | b, applied by template recursion so every
// index is a constant and the values stay in registers).
template <int D>
struct SortNet {
  static constexpr int count() {
    int c = 0;
    for (int p = 1; p < D; p <<= 1)
      for (int k = p; k >= 1; k >>= 1)
        for (int j = k % p; j + k < D; j += 2 * k)
          for (int i = 0; i < k && i < D - j - k; ++i)
            if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) ++c;
    return c;
  }
  static constexpr int kN = count();
  struct Arr {
    int v[kN > 0 ? kN : 1];
  };
  static constexpr Arr make() {
    Arr r{};
    int c = 0;
    for (int p = 1; p < D; p <<= 1)
      for (int k = p; k >= 1; k >>= 1)
        for (int j = k % p; j + k < D; j += 2 * k)
          for (int i = 0; i < k && i < D - j - k; ++i)
            if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) r.v[c++] = ((i + j) << 6) | (i + j + k);
    return r;
  }
  static constexpr Arr net = make();
};

template <int D, int C>
__device__ __forceinline__ void sort_net_apply(float *v) {
  if constexpr (C < SortNet<D>::kN) {
    constexpr int e = SortNet<D>::net.v[C];
    const float x = v[e >> 6], y = v[e & 63];
    v[e >> 6] = fminf(x, y);
    v[e & 63] = fmaxf(x, y);
    sort_net_apply<D, C + 1>(v);
  }
}

// Median by the sorting network (even D: mean of the two middle values).
template <int D>
__device__ __forceinline__ float median_net(float *v) {
  sort_net_apply<D, 0>(v);
  if (D & 1) return v[D / 2];
  return 0.5f * (v[D / 2 - 1] + v[D / 2]);
}

// ---------------------------------------------------------------- launch helpers
// Runtime LOG2M -> compile-time dispatch for 3 <= LOG2M <= 13.
#define FCS_DISPATCH_LOG2M(log2m, BODY)                      \
  switch (log2m) {                                           \
    case 3: { constexpr int L = 3; BODY; } break;            \
    case 4: { constexpr int L = 4; BODY; } break;            \
    case 5: { constexpr int L = 5; BODY; } break;            \
    case 6: { constexpr int L = 6; BODY; } break;            \
    case 7: { constexpr int L = 7; BODY; } break;            \
    case 8: { constexpr int L = 8; BODY; } break;            \
    case 9: { constexpr int L = 9; BODY; } break;            \
    case 10: { constexpr int L = 10; BODY; } break;          \
    case 11: { constexpr int L = 11; BODY; } break;          \
    case 12: { constexpr int L = 12; BODY; } break;          \
    case 13: { constexpr int L = 13; BODY; } break;          \
    default: break;                                          \
  }

// Threads used for a length-M complex FFT: one radix-16 butterfly each,
// at least one warp.
__host__ __device__ constexpr int fft_threads(int log2m) {
  return (log2m - 4) > 5 ? (1 << (log2m - 4)) : 32;
}

// Hash-table geometry shared by the sketch kernels.
struct Modes {
  int N;
  int64_t I[kMaxN];
  int64_t off[kMaxN];   // offset of mode n inside one sketch's table row
  int32_t J[kMaxN];
  int64_t ldh;          // elements between sketch rows of h / s
  int64_t Jt;
};

int make_modes(fcs_ctx *ctx, int N, const int64_t *host_I, const int32_t *host_J,
               int64_t ldh, Modes *m);
// make_modes without a context: the message goes to err (n bytes, may be NULL).
int make_modes_msg(char *err, size_t n, int N, const int64_t *host_I,
                   const int32_t *host_J, int64_t ldh, Modes *m);

// FFT-based calls for kMaxLog2P < log2p <= kMaxLog2PBig (fcs_big.cu); the
// callers have validated the arguments.
// ext_ws: caller-owned device buffer of ext_bytes (a batch plan's), or NULL
// for the context workspace.  stage 0 issues everything.  A batch plan splits
// the P = 2^15 warp-DIT route in two: stage 1 issues only the clearing of its
// accumulator (*split = true when the route applies; otherwise nothing is
// issued), stage 2 only its kernel, launched as a programmatic dependent of
// the kernel before it in the stream (it waits for that grid at its end).
int big_sketch_cp(fcs_ctx *ctx, const Modes &m, int64_t R, int D, const float *const *host_U,
                  const int64_t *host_ldU, const float *lambda, const int32_t *h,
                  const int8_t *s, float *out, int log2p, void *ext_ws = nullptr,
                  size_t ext_bytes = 0, int stage = 0, bool *split = nullptr);
// Device bytes big_sketch_cp uses when its buffer holds at most `cap` bytes.
size_t big_sketch_cp_bytes(const Modes &m, int64_t R, int D, int log2p, size_t cap, int nsm);
int big_contract(fcs_ctx *ctx, const Modes &m, int kind, int free_mode, int D,
                 const float *fcsT, int64_t B, const float *const *vec, const int32_t *h,
                 const int8_t *s, float2 *spec, bool need_spec, cudaEvent_t spec_ready,
                 float *raw, int log2p);
int big_outer(fcs_ctx *ctx, int64_t nbatch, int64_t L, int D, int64_t La, int64_t Lb,
              const float *fa, const float *fb, float *out, int log2p);

}  // namespace fcs
