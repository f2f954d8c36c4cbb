// fcs_hash.cuh -- one entry of the per-mode hash pairs {h_n, s_n} of Def. 4,
// shared by fcs_make_hashes (its own launch) and the CP route's prep launch
// (fcs_sketch_cp_seeded), so both write the same tables for a seed.
//
// Family (the paper only requires 2-wise independence): Carter-Wegman
// multiply-mod-prime over p = 2^61 - 1 with coefficients from SplitMix64
// (Steele, Lea & Flood 2014), four draws (a_h, b_h, a_s, b_s) per (d, n) in
// d-major, n-minor order.  SplitMix64 is counter-based -- draw k is
// mix(seed + (k+1) * golden_gamma) -- so every thread derives its own
// coefficients without any sequential state.
#pragma once

#include "fcs_internal.cuh"

namespace fcs {

constexpr uint64_t kP61 = (uint64_t(1) << 61) - 1;

__device__ __forceinline__ uint64_t splitmix_draw(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// (a*i + b) mod (2^61-1) for a, b < 2^61 and i < 2^32: the 128-bit value is
// folded with 2^61 = 1 (mod p).
__device__ __forceinline__ uint64_t mulmod_p61(uint64_t a, uint64_t i, uint64_t b) {
  uint64_t lo = a * i;
  uint64_t hi = __umul64hi(a, i);
  lo += b;
  hi += (lo < b) ? 1 : 0;
  const uint64_t t0 = lo & kP61;
  const uint64_t t1 = ((lo >> 61) | (hi << 3)) & kP61;
  const uint64_t t2 = hi >> 58;
  uint64_t s = t0 + t1 + t2;          // < 3 * 2^61
  s = (s & kP61) + (s >> 61);
  if (s >= kP61) s -= kP61;
  return s;
}

struct HashArgs {
  uint64_t seed;
  int N, D;
  int64_t total;                 // sum_n I_n (the tables' row length)
  int64_t off[kMaxN + 1];        // prefix sums of I_n
  int32_t J[kMaxN];
};

// Entry e (global position in [0, total)) of sketch d: h[d*total + e] and
// s[d*total + e].
__device__ __forceinline__ void hash_entry(const HashArgs &a, int d, int64_t e,
                                           int32_t *__restrict__ h, int8_t *__restrict__ s) {
  int n = 0;
#pragma unroll
  for (int m = 1; m < kMaxN; ++m)
    if (m < a.N && e >= a.off[m]) n = m;
  const uint64_t i = uint64_t(e - a.off[n]);
  const uint64_t k = uint64_t(4) * (uint64_t(d) * a.N + n);
  const uint64_t ah = 1 + splitmix_draw(a.seed, k) % (kP61 - 1);
  const uint64_t bh = splitmix_draw(a.seed, k + 1) % kP61;
  const uint64_t as = 1 + splitmix_draw(a.seed, k + 2) % (kP61 - 1);
  const uint64_t bs = splitmix_draw(a.seed, k + 3) % kP61;
  const uint64_t vh = mulmod_p61(ah, i, bh);
  const uint64_t vs = mulmod_p61(as, i, bs);
  h[d * a.total + e] = int32_t(vh % uint64_t(a.J[n]));
  s[d * a.total + e] = int8_t(1 - 2 * int(vs & 1));
}

// Host side: the arguments for N modes (validated by the caller: I_n <= 2^32).
inline HashArgs hash_args(uint64_t seed, int N, int D, const int64_t *host_I,
                          const int32_t *host_J) {
  HashArgs a{};
  a.seed = seed;
  a.N = N;
  a.D = D;
  int64_t t = 0;
  for (int n = 0; n < N; ++n) {
    a.off[n] = t;
    t += host_I[n];
  }
  for (int n = N; n <= kMaxN; ++n) a.off[n] = t;
  a.total = t;
  for (int n = 0; n < kMaxN; ++n) a.J[n] = n < N ? host_J[n] : 1;
  return a;
}

}  // namespace fcs
