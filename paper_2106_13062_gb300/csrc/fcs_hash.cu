// fcs_hash.cu -- fcs_make_hashes: the per-mode hash pairs {h_n, s_n} of
// Def. 4 for D independent sketches.
//
// Family (the paper only requires 2-wise independence): Carter-Wegman
// multiply-mod-prime over p = 2^61 - 1 with coefficients from SplitMix64
// (Steele, Lea & Flood 2014), four draws (a_h, b_h, a_s, b_s) per (d, n) in
// d-major, n-minor order.  SplitMix64 is counter-based -- draw k is
// mix(seed + (k+1) * golden_gamma) -- so every thread derives its own
// coefficients without any sequential state.
#include "fcs_internal.cuh"

namespace fcs {
namespace {

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
  int64_t total;                 // sum_n I_n
  int64_t off[kMaxN + 1];        // prefix sums of I_n
  int32_t J[kMaxN];
};

// One thread per table entry (d, global position e in [0, total)).
__global__ void make_hashes_kernel(HashArgs a, int32_t *__restrict__ h,
                                   int8_t *__restrict__ s) {
  const int d = blockIdx.y;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < a.total;
       e += int64_t(gridDim.x) * blockDim.x) {
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
}

}  // namespace
}  // namespace fcs

using namespace fcs;

extern "C" int fcs_make_hashes(fcs_ctx *ctx, uint64_t seed, int N, const int64_t *host_I,
                               const int32_t *host_J, int D, int32_t *h, int8_t *s) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  Modes m;
  int rc = make_modes(ctx, N, host_I, host_J, 0, &m);
  if (rc) return rc;
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (!h || !s) return set_error(ctx, FCS_EINVAL, "h or s is NULL");
  for (int n = 0; n < N; ++n)
    if (host_I[n] > (int64_t(1) << 32))
      return set_error(ctx, FCS_EINVAL, "I[%d] too large for the hash family", n);
  HashArgs a{};
  a.seed = seed;
  a.N = N;
  a.D = D;
  a.total = m.ldh;
  for (int n = 0; n <= kMaxN; ++n) a.off[n] = n < N ? m.off[n] : m.ldh;
  for (int n = 0; n < kMaxN; ++n) a.J[n] = n < N ? host_J[n] : 1;
  DeviceGuard g(ctx->device);
  const int threads = 256;
  int64_t blocks = (a.total + threads - 1) / threads;
  if (blocks > 65535) blocks = 65535;
  make_hashes_kernel<<<dim3(unsigned(blocks), unsigned(D)), threads, 0, ctx->stream>>>(a, h, s);
  return check_cuda(ctx, cudaGetLastError(), "make_hashes_kernel");
}
