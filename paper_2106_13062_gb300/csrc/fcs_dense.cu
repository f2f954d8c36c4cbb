// fcs_dense.cu -- fcs_sketch_dense: FCS of a general tensor, eq. (FCS_asyn):
//   FCS_d(T)[sum_n h_n(i_n)] += prod_n s_n(i_n) T(i_1, ..., i_N)
// for every entry and every sketch d.  H and S are never materialised; the
// per-mode tables are staged in shared memory (h and the sign packed into one
// int32), and each CTA accumulates all D sketches in shared-memory bins before
// adding them to the output once.
//
// Fast path (last mode contiguous, 16-byte aligned rows): one warp handles
// 128 consecutive entries of a row with one float4 load per lane; the partial
// hash of the leading modes is computed once per row and sketch.
#include "fcs_internal.cuh"

#include <cfloat>
#include <type_traits>

namespace fcs {
namespace {

struct DenseArgs {
  Modes m;
  int D;
  const float *T;
  int64_t stride[kMaxN];
  const int32_t *h;
  const int8_t *s;
  float *out;
  int64_t tbs, obs;     // batch strides (elements)
  int64_t rows;         // prod_{n < N-1} I_n
  int64_t L;            // I_{N-1}
  int64_t cpr;          // chunks per row (vector path) / entries per warp unit
  int64_t units;        // work units per batch item
  int tot;              // sum I_n
  // row-chunk kernel: offset of leading mode n in the staged compact table
  // (the modes may be permuted so that a unit-stride mode comes last; the
  // table entry of mode n, index i stays at h[d*ldh + m.off[n] + i])
  int64_t coff[kMaxN];
};

__global__ void zero_out_kernel(float *out, int64_t len, int64_t obs) {
  float *o = out + blockIdx.y * obs;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < len;
       e += int64_t(gridDim.x) * blockDim.x)
    o[e] = 0.f;
}

// Packed table entry: (h << 1) | (s < 0).
__device__ __forceinline__ int32_t packed_entry(const DenseArgs &a, int d, int e) {
  const int64_t g = d * a.m.ldh + e;
  return (a.h[g] << 1) | (a.s[g] < 0 ? 1 : 0);
}

template <bool VEC, bool SMEM>
__global__ void __launch_bounds__(1024) dense_kernel(DenseArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int D = a.D, tot = a.tot, N = a.m.N;
  const int64_t Jt = a.m.Jt;
  int32_t *tab = reinterpret_cast<int32_t *>(smem);
  float *bins = reinterpret_cast<float *>(tab + (SMEM ? D * tot : 0));
  const int b = blockIdx.y;
  float *outb = a.out + b * a.obs;
  if (SMEM) {
    for (int e = threadIdx.x; e < D * tot; e += blockDim.x) {
      const int d = e / tot;
      tab[e] = packed_entry(a, d, e - d * tot);
    }
    for (int64_t e = threadIdx.x; e < D * Jt; e += blockDim.x) bins[e] = 0.f;
    __syncthreads();
  }
  auto entry = [&](int d, int64_t e) -> int32_t {
    return SMEM ? tab[d * tot + e] : packed_entry(a, d, int(e));
  };
  // a hash value outside [0, J_n) in any mode drops the entry for sketch d
  auto valid = [&](int32_t t, int n) { return unsigned(t >> 1) < unsigned(a.m.J[n]); };
  auto add = [&](int d, int64_t bin, float v) {
    if (bin < 0 || bin >= Jt) return;
    if (SMEM)
      atomicAdd(&bins[d * Jt + bin], v);
    else
      atomicAdd(&outb[d * Jt + bin], v);
  };
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const float *Tb = a.T + b * a.tbs;

  for (int64_t u = gw; u < a.units; u += nw) {
    if (VEC) {
      const int64_t row = u / a.cpr;
      const int64_t c = u - row * a.cpr;
      int64_t idx[kMaxN];
      int64_t rr = row, addr = 0;
      for (int n = N - 2; n >= 0; --n) {
        idx[n] = rr % a.m.I[n];
        rr /= a.m.I[n];
        addr += idx[n] * a.stride[n];
      }
      const int64_t il = c * 128 + lane * 4;
      const bool active = il < a.L;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (active) v = __ldcs(reinterpret_cast<const float4 *>(Tb + addr + il));
      const float vv[4] = {v.x, v.y, v.z, v.w};
      for (int d = 0; d < D; ++d) {
        int base = 0, neg = 0;
        bool ok = true;
        for (int n = 0; n < N - 1; ++n) {
          const int32_t t = entry(d, a.m.off[n] + idx[n]);
          base += t >> 1;
          neg ^= t & 1;
          ok = ok && valid(t, n);
        }
        if (active && ok) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int32_t t = entry(d, a.m.off[N - 1] + il + k);
            const float x = ((neg ^ t) & 1) ? -vv[k] : vv[k];
            if (valid(t, N - 1)) add(d, base + (t >> 1), x);
          }
        }
      }
    } else {
      // generic strides: 32 consecutive logical (C-order) entries per unit
      const int64_t e = u * 32 + lane;
      const int64_t numel = a.rows * a.L;
      if (e < numel) {
        int64_t idx[kMaxN];
        int64_t rr = e, addr = 0;
        for (int n = N - 1; n >= 0; --n) {
          idx[n] = rr % a.m.I[n];
          rr /= a.m.I[n];
          addr += idx[n] * a.stride[n];
        }
        const float x = Tb[addr];
        for (int d = 0; d < D; ++d) {
          int bin = 0, neg = 0;
          bool ok = true;
          for (int n = 0; n < N; ++n) {
            const int32_t t = entry(d, a.m.off[n] + idx[n]);
            bin += t >> 1;
            neg ^= t & 1;
            ok = ok && valid(t, n);
          }
          if (ok) add(d, bin, neg ? -x : x);
        }
      }
    }
  }
  if (SMEM) {
    __syncthreads();
    for (int64_t e = threadIdx.x; e < D * Jt; e += blockDim.x) {
      const float v = bins[e];
      if (v != 0.f) atomicAdd(&outb[e], v);
    }
  }
}

// Row-chunk kernel (contiguous last mode, J_{N-1} < 2^15): warp w owns a
// fixed chunk of 256 consecutive last-mode indices (two float4 per lane) and
// walks the rows i_1..i_{N-1} of its batch item.  Because the chunk never
// changes, the lane's eight last-mode bin offsets (16-bit) and signs (one
// mask word) per sketch are read from shared memory as two words per row and
// sketch; the leading modes' partial hash and sign are the same for the whole
// warp, read once per row and sketch.  The next row's values are prefetched
// while the current row is scattered.
//
// Accumulation is exact integer fixed point: shared-memory FP32 atomics are a
// compare-and-swap loop (about 6x slower than a 32-bit integer atomic add), so
// every entry x is rounded once to xi = rint(x / q) with a power-of-two step
// q = 2^(E-25) per CTA, where 2^E bounds the magnitudes of a sample (the first
// row of every warp), and the D signed copies of xi are added with int32
// atomics.  Integer sums do not depend on the order of the adds.  Three cases
// leave the fast path, each exactly:
//  * outliers (|x| >= ~2^30 q, NaN, Inf) are added in FP32 straight into the
//    output sketch with global atomics;
//  * a bin whose int32 sum wraps adds the carry, +-2^32 q (a power of two),
//    to the output the same way, so bins are effectively 64-bit.  Every add
//    returns the bin's old value; an add of |xi| < 2^30 to a bin below 2^30
//    in magnitude cannot wrap, so only adds that saw a larger old value are
//    examined for a wrap;
//  * if the rounding error of the CTA, whose expected L2 norm is
//    q sqrt(n/12) for n rounded entries, exceeds 1e-7 of the CTA's
//    ||x||_2 (data with a large dynamic range), the CTA re-reads its rows and
//    adds the exact remainders x - q xi with FP32 shared atomics.
// A CTA whose sample is all zeros or outside 2^-100..2^100 accumulates in FP32.
// The bins are flushed to the output as FP32 (q xi_sum, one rounding).
// Hash values outside [0, J_n) are skipped; a CTA that finds one in its
// tables takes the checked (slower) scatter for every row.
// NL = number of leading modes (N - 1) when known at compile time, -1 for the
// general case (N - 1 <= kMaxN - 1, checked at run time).
template <int NT, int NL>
__global__ void __launch_bounds__(NT) dense_rows_kernel(DenseArgs a, int totL, int cpr,
                                                        int64_t warps_used, int DC) {
  constexpr int NLMAX = NL >= 0 ? NL : kMaxN - 1;
  auto leading = [&](int n) { return n < NLMAX && (NL >= 0 || n < a.m.N - 1); };
  // this CTA handles sketches d0 .. d0 + nd - 1 (nd <= DC); d below is local
  const int d0 = blockIdx.z * DC;
  const int nd = min(DC, a.D - d0);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned int s_max;            // sample max |x|, FP32 bits
  __shared__ float s_sumsq;
  __shared__ unsigned long long s_nfx;
  __shared__ int s_bad;                     // some hash value outside [0, J_n)
  const int N = a.m.N;
  const int64_t Jt = a.m.Jt;
  uint32_t *ltab = reinterpret_cast<uint32_t *>(smem);     // [nd][cpr][32][4] last mode
  uint32_t *lsg = ltab + DC * cpr * 128;                  // [nd][cpr][32] sign masks
  int32_t *tab = reinterpret_cast<int32_t *>(lsg + DC * cpr * 32);   // [nd][totL] leading
  int32_t *ibins = tab + DC * totL;                        // [nd][Jt] int32 (or FP32)
  float *fbins = reinterpret_cast<float *>(ibins);
  if (threadIdx.x == 0) {
    s_max = 0u;
    s_sumsq = 0.f;
    s_nfx = 0ull;
    s_bad = 0;
  }
  __syncthreads();
  {
    int bad = 0;
    for (int e = threadIdx.x; e < nd * totL; e += NT) {
      const int d = e / totL;
      const int k = e - d * totL;
      int n = 0;
#pragma unroll
      for (int m = 1; m < kMaxN - 1; ++m)
        if (m < N - 1 && k >= a.coff[m]) n = m;
      const int32_t t = packed_entry(a, d0 + d, int(a.m.off[n] + (k - a.coff[n])));
      bad |= int(unsigned(t >> 1) >= unsigned(a.m.J[n]));
      tab[e] = t;
    }
    if (bad) s_bad = 1;
  }
  for (int64_t e = threadIdx.x; e < nd * Jt; e += NT) ibins[e] = 0;

  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * int64_t(NT) + threadIdx.x) >> 5;
  const int c = int(gw % cpr);
  const int64_t rstride = warps_used / cpr;
  const int64_t i0 = int64_t(c) * 256 + lane * 4;      // segment s starts at i0 + 128 s
  const bool act0 = i0 < a.L, act1 = i0 + 128 < a.L;
  // last-mode tables in shared memory, one 16-byte word per (sketch, chunk,
  // lane): eight 16-bit entries (offset in bits 0..14, sign in bit 15) for
  // the lane's elements e = 0..7, last-mode index i0 + (e / 4) * 128 + e % 4;
  // the eight signs are also gathered into one mask word per (sketch, chunk,
  // lane) in lsg.
  // Absent elements (past the end of the mode) get a distinct in-range
  // offset and value 0, so they add nothing and never collide.
  {
    const int64_t offl = a.m.off[N - 1];
    const uint32_t JL = uint32_t(a.m.J[N - 1]);
    int bad = 0;
    for (int k = threadIdx.x; k < nd * cpr * 32 * 8; k += NT) {
      const int e = k & 7, ln = (k >> 3) & 31;
      const int cc = (k >> 8) % cpr, d = (k >> 8) / cpr;
      const int64_t i = int64_t(cc) * 256 + ln * 4 + (e >> 2) * 128 + (e & 3);
      uint32_t t16 = uint32_t(ln) % JL;
      if (i < a.L) {
        const int32_t t = packed_entry(a, d0 + d, int(offl + i));
        const uint32_t hv = uint32_t(t >> 1);
        bad |= int(hv >= JL);
        t16 = (hv < JL ? hv : 0u) | (uint32_t(t & 1) << 15);   // sign kept for lsg
      }
      reinterpret_cast<uint16_t *>(ltab)[k] = uint16_t(t16);
    }
    if (bad) s_bad = 1;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nd * cpr * 32; k += NT) {
    const uint16_t *t = reinterpret_cast<const uint16_t *>(ltab) + k * 8;
    uint32_t m = 0;
    for (int e = 0; e < 8; ++e) m |= uint32_t(t[e] >> 15) << e;
    lsg[k] = m;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nd * cpr * 32 * 8; k += NT)
    reinterpret_cast<uint16_t *>(ltab)[k] &= uint16_t(0x7fff);

  const int b = blockIdx.y;
  const float *Tb = a.T + b * a.tbs;
  float *outb = a.out + b * a.obs;
  // rows < 2^31 and I_n < 2^31 here, so 32-bit division suffices
  auto row_addr = [&](int64_t row, int *idx) {
    uint32_t rr = uint32_t(row);
    int64_t addr = 0;
#pragma unroll
    for (int n = NLMAX - 1; n >= 0; --n) {
      if (leading(n)) {
        const uint32_t In = uint32_t(a.m.I[n]);
        const uint32_t q = rr / In;
        idx[n] = int(rr - q * In);
        rr = q;
        addr += idx[n] * a.stride[n];
      }
    }
    return addr;
  };
  // rows advance by rstride: its mixed-radix digits over the leading modes
  // let the next row's indices follow by digit-wise addition with carries
  int rsd[kMaxN];
  {
    uint32_t rr = uint32_t(warps_used / cpr);
#pragma unroll
    for (int n = NLMAX - 1; n >= 0; --n) {
      rsd[n] = 0;
      if (leading(n)) {
        const uint32_t In = uint32_t(a.m.I[n]);
        rsd[n] = int(rr % In);
        rr /= In;
      }
    }
  }
  auto next_row = [&](const int *idx, int *nidx) {
    int carry = 0;
    int64_t addr = 0;
#pragma unroll
    for (int n = NLMAX - 1; n >= 0; --n) {
      if (leading(n)) {
        const int In = int(a.m.I[n]);
        const int v = idx[n] + rsd[n] + carry;
        carry = v >= In;
        nidx[n] = carry ? v - In : v;
        addr += nidx[n] * a.stride[n];
      }
    }
    return addr;
  };
  auto load = [&](int64_t addr, float4 &x0, float4 &x1) {
    x0 = act0 ? __ldcs(reinterpret_cast<const float4 *>(Tb + addr + i0))
              : make_float4(0.f, 0.f, 0.f, 0.f);
    x1 = act1 ? __ldcs(reinterpret_cast<const float4 *>(Tb + addr + i0 + 128))
              : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  const bool working = gw < warps_used;
  const int64_t row0 = gw / cpr;

  // ---- scale from the sample: the first row of every warp
  {
    float m = 0.f;
    if (working && row0 < a.rows) {
      int idx[kMaxN];
      float4 x0, x1;
      load(row_addr(row0, idx), x0, x1);
      const float v[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (fabsf(v[e]) <= FLT_MAX) m = fmaxf(m, fabsf(v[e]));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && m > 0.f) atomicMax(&s_max, __float_as_uint(m));
  }
  __syncthreads();
  const bool tables_ok = s_bad == 0;
  int E = 0;
  const float smax = __uint_as_float(s_max);
  frexpf(smax, &E);                        // smax < 2^E
  const bool fx = smax > 0.f && E > -100 && E < 100;
  const float q = fx ? ldexpf(1.f, E - 25) : 1.f;        // fixed-point step
  const float inv_q = fx ? ldexpf(1.f, 25 - E) : 1.f;
  const float carry = fx ? ldexpf(1.f, E + 7) : 0.f;     // 2^32 q

  // Fast scatter of one row into sketch d: eight int32 adds issued back to
  // back, then one test of their old values (bit 31 of old + 2^30 is set iff
  // |old| >= 2^30); only then are the adds checked for a wrap.  LNEG is the
  // leading modes' sign, uniform across the warp.  The lane's table and bin
  // pointers for sketch d are passed in (stepped once per sketch).
  const uint4 *ltab_l = reinterpret_cast<const uint4 *>(ltab) + c * 32 + lane;
  const uint32_t *lsg_l = lsg + c * 32 + lane;
  const int lstep = cpr * 32;
  auto scatter_fast = [&](auto lneg_c, int d, int base, const int *xi, const uint4 *tp,
                          const uint32_t *sp, int32_t *bins_d) {
    constexpr bool LNEG = decltype(lneg_c)::value;
    const uint4 tw = *tp;
    const uint32_t w[4] = {tw.x, tw.y, tw.z, tw.w};
    const uint32_t sg = *sp;
    int32_t *bb = bins_d + base;
    int val[8], old[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const uint32_t off = (e & 1) ? (w[e >> 1] >> 16) : (w[e >> 1] & 0xffffu);
      const bool sneg = ((sg >> e) & 1u) != 0;
      val[e] = (sneg != LNEG) ? -xi[e] : xi[e];
      old[e] = atomicAdd(bb + off, val[e]);
    }
    // bit 31 of old + 2^30 is set iff |old| >= 2^30
    int flag = 0;
#pragma unroll
    for (int e = 0; e < 8; e += 2)
      flag |= int(unsigned(old[e]) + 0x40000000u) | int(unsigned(old[e + 1]) + 0x40000000u);
    if (flag < 0) {                                    // rare: a large bin
      float *od = outb + (d0 + d) * Jt + base;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const uint32_t off = (e & 1) ? (w[e >> 1] >> 16) : (w[e >> 1] & 0xffffu);
        const int nw = int(unsigned(old[e]) + unsigned(val[e]));
        if (((old[e] ^ nw) & (val[e] ^ nw)) < 0)
          atomicAdd(od + off, val[e] > 0 ? carry : -carry);
      }
    }
  };

  // mode 0: fixed point (+ outliers, carries); 1: FP32 remainders x - q xi
  // of the fixed-point entries; 2: plain FP32 accumulation.
  float sumsq = 0.f;
  unsigned nfx = 0;
  auto run_rows = [&](auto mode_c) {
    constexpr int MODE = decltype(mode_c)::value;
    int64_t row = row0;
    int idx[kMaxN], nidx[kMaxN];
#pragma unroll
    for (int n = 0; n < kMaxN; ++n) idx[n] = nidx[n] = 0;
    float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
    if (working && row < a.rows) load(row_addr(row, nidx), n0, n1);
    for (; working && row < a.rows; row += rstride) {
#pragma unroll
      for (int n = 0; n < kMaxN; ++n) idx[n] = nidx[n];
      const float v[8] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
      if (row + rstride < a.rows) load(next_row(idx, nidx), n0, n1);
      int xi[8];
      float rv[8];
      // one sum of squares per row decides the fast path: below 2^60 every
      // |u| < 2^30 and nothing is NaN or Inf
      float srow = 0.f;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float u = v[e] * inv_q;
        xi[e] = __float2int_rn(u);
        srow = fmaf(u, u, srow);
      }
      const bool fast_row =
          MODE == 0 && tables_ok && __all_sync(0xffffffffu, srow < 1.152921504606846976e18f);
      unsigned fastm = 0xffu;      // bit e: entry e goes through the integer path
      if (MODE == 0) {
        sumsq += srow;             // in units of q^2
        nfx += 8u;
      }
      if (!fast_row) {
        fastm = 0u;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float u = v[e] * inv_q;
          const bool fast = fabsf(u) < 1073741760.f;     // 2^30 - 2^6; false for NaN
          if (!fast) xi[e] = 0;
          fastm |= unsigned(fast) << e;
          rv[e] = MODE == 1 ? (fast ? fmaf(-q, __int2float_rn(xi[e]), v[e]) : 0.f) : v[e];
        }
      }
      if (fast_row) {
        const int32_t *tabn[kMaxN];
#pragma unroll
        for (int n = 0; n < NLMAX; ++n)
          if (leading(n)) tabn[n] = tab + int(a.coff[n] + idx[n]);
        const uint4 *tp = ltab_l;
        const uint32_t *sp = lsg_l;
        int32_t *bins_d = ibins;
#pragma unroll 1
        for (int d = 0; d < nd; ++d) {
          int base = 0, neg = 0;
#pragma unroll
          for (int n = 0; n < NLMAX; ++n) {
            if (leading(n)) {
              const int32_t t = *tabn[n];
              tabn[n] += totL;
              base += t >> 1;
              neg ^= t & 1;
            }
          }
          if (neg)
            scatter_fast(std::true_type(), d, base, xi, tp, sp, bins_d);
          else
            scatter_fast(std::false_type(), d, base, xi, tp, sp, bins_d);
          tp += lstep;
          sp += lstep;
          bins_d += Jt;
        }
        continue;
      }
      // checked scatter (bad hash values, outliers, FP32 modes): the tables
      // are re-read from global memory and every index is checked
#pragma unroll 1
      for (int d = 0; d < nd; ++d) {
        int base = 0, neg = 0;
        bool row_ok = true;
#pragma unroll
        for (int n = 0; n < NLMAX; ++n) {
          if (leading(n)) {
            const int32_t t = tab[d * totL + int(a.coff[n] + idx[n])];
            base += t >> 1;
            neg ^= t & 1;
            row_ok = row_ok && unsigned(t >> 1) < unsigned(a.m.J[n]);
          }
        }
        if (!row_ok) continue;
        int32_t *bi = ibins + d * Jt + base;
        float *bf = fbins + d * Jt + base;
        float *od = outb + (d0 + d) * Jt + base;
        const uint32_t JL = uint32_t(a.m.J[N - 1]);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          if (!((e < 4) ? act0 : act1)) continue;
          const int64_t il = i0 + (e >> 2) * 128 + (e & 3);
          const int32_t t = packed_entry(a, d0 + d, int(a.m.off[N - 1] + il));
          const uint32_t off = uint32_t(t >> 1);
          if (off >= JL) continue;
          const bool sneg = ((t & 1) != 0) != (neg != 0);
          if (MODE == 0) {
            if ((fastm >> e) & 1u) {
              const int val = sneg ? -xi[e] : xi[e];
              const int old = atomicAdd(bi + off, val);
              const int nw = int(unsigned(old) + unsigned(val));
              if (((old ^ nw) & (val ^ nw)) < 0) atomicAdd(od + off, val > 0 ? carry : -carry);
            } else {
              atomicAdd(od + off, sneg ? -v[e] : v[e]);   // outlier, exact FP32
            }
          } else if (MODE == 2 || ((fastm >> e) & 1u)) {
            atomicAdd(bf + off, sneg ? -rv[e] : rv[e]);
          }
        }
      }
    }
  };
  // Add the CTA's bins (value(e) for local bin e) to the output: 16-byte
  // vector reductions over the aligned middle, scalar atomics at the ends.
  auto flush = [&](auto value) {
    float *dst = outb + d0 * Jt;
    const int64_t n = nd * Jt;
    int64_t head = int64_t((16 - (reinterpret_cast<uintptr_t>(dst) & 15)) & 15) / 4;
    if (head > n) head = n;
    const int64_t body = head + ((n - head) & ~int64_t(3));
    for (int64_t e = threadIdx.x; e < head; e += NT) {
      const float x = value(e);
      if (x != 0.f) atomicAdd(dst + e, x);
    }
    for (int64_t e = head + 4 * int64_t(threadIdx.x); e < body; e += 4 * int64_t(NT)) {
      const float x0 = value(e), x1 = value(e + 1), x2 = value(e + 2), x3 = value(e + 3);
      if (x0 != 0.f || x1 != 0.f || x2 != 0.f || x3 != 0.f)
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + e), "f"(x0),
                     "f"(x1), "f"(x2), "f"(x3)
                     : "memory");
    }
    for (int64_t e = body + threadIdx.x; e < n; e += NT) {
      const float x = value(e);
      if (x != 0.f) atomicAdd(dst + e, x);
    }
  };
  auto flush_float = [&]() { flush([&](int64_t e) { return fbins[e]; }); };

  if (!fx) {                          // this CTA accumulates in FP32
    run_rows(std::integral_constant<int, 2>());
    __syncthreads();
    flush_float();
    return;
  }
  run_rows(std::integral_constant<int, 0>());
  // CTA totals for the rounding-error test
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    sumsq += __shfl_xor_sync(0xffffffffu, sumsq, o);
    nfx += __shfl_xor_sync(0xffffffffu, nfx, o);
  }
  if (lane == 0) {
    atomicAdd(&s_sumsq, sumsq);
    atomicAdd(&s_nfx, (unsigned long long)nfx);
  }
  __syncthreads();
  flush([&](int64_t e) { return __int2float_rn(ibins[e]) * q; });
  // expected squared rounding error n q^2 / 12 against (1e-7 ||x||)^2, in
  // units of q^2 (the test is uniform across the CTA)
  if (!(float(s_nfx) * (1.f / 12.f) > 1e-14f * s_sumsq)) return;
  __syncthreads();
  for (int64_t e = threadIdx.x; e < nd * Jt; e += NT) fbins[e] = 0.f;
  __syncthreads();
  run_rows(std::integral_constant<int, 1>());
  __syncthreads();
  flush_float();
}

}  // namespace
}  // namespace fcs

using namespace fcs;

extern "C" int fcs_sketch_dense(fcs_ctx *ctx, int N, const int64_t *host_I,
                                const int64_t *host_stride, const int32_t *host_J, int D,
                                const float *T, const int32_t *h, const int8_t *s,
                                int64_t ldh, float *out, int64_t nbatch,
                                int64_t T_batch_stride, int64_t out_batch_stride) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  DenseArgs a{};
  int rc = make_modes(ctx, N, host_I, host_J, ldh, &a.m);
  if (rc) return rc;
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (!T || !h || !s || !out) return set_error(ctx, FCS_EINVAL, "NULL device pointer");
  if (nbatch < 1 || nbatch > 65535)
    return set_error(ctx, FCS_EINVAL, "nbatch=%lld outside [1,65535]", (long long)nbatch);
  a.D = D;
  a.T = T;
  a.h = h;
  a.s = s;
  a.out = out;
  a.tbs = nbatch > 1 ? T_batch_stride : 0;
  a.obs = nbatch > 1 ? out_batch_stride : 0;
  const int64_t Jt = a.m.Jt;
  if (nbatch > 1 && (a.obs < D * Jt || a.tbs < 0))
    return set_error(ctx, FCS_EINVAL, "batch strides overlap");
  int64_t tot = 0;
  for (int n = 0; n < N; ++n) tot += host_I[n];
  if (tot > (int64_t(1) << 30)) return set_error(ctx, FCS_EUNSUPPORTED, "tables too large");
  a.tot = int(tot);
  // default C-order strides
  int64_t st = 1;
  for (int n = N - 1; n >= 0; --n) {
    a.stride[n] = host_stride ? host_stride[n] : st;
    st *= host_I[n];
  }
  // FCS does not depend on the order of the modes (bin and sign are a sum and
  // a product over them): when the last mode is not the contiguous one but
  // another is, that mode is moved last so the row-chunk kernel applies.
  // Only the per-mode geometry moves; the hash tables stay where they are.
  if (a.stride[N - 1] != 1) {
    int k = -1;
    for (int n = N - 2; n >= 0 && k < 0; --n)
      if (a.stride[n] == 1 && a.m.I[n] >= 4) k = n;
    if (k >= 0) {
      const int64_t Ik = a.m.I[k], ok = a.m.off[k], sk = a.stride[k];
      const int32_t Jk = a.m.J[k];
      for (int n = k; n < N - 1; ++n) {
        a.m.I[n] = a.m.I[n + 1];
        a.m.J[n] = a.m.J[n + 1];
        a.m.off[n] = a.m.off[n + 1];
        a.stride[n] = a.stride[n + 1];
      }
      a.m.I[N - 1] = Ik;
      a.m.J[N - 1] = Jk;
      a.m.off[N - 1] = ok;
      a.stride[N - 1] = sk;
    }
  }
  {
    int64_t c = 0;
    for (int n = 0; n < kMaxN; ++n) {
      a.coff[n] = c;
      if (n < N - 1) c += a.m.I[n];
    }
  }
  a.L = a.m.I[N - 1];
  a.rows = 1;
  for (int n = 0; n < N - 1; ++n) a.rows *= a.m.I[n];

  bool vec = a.stride[N - 1] == 1 && a.L % 4 == 0 &&
             (reinterpret_cast<uintptr_t>(T) & 15) == 0 && (a.tbs % 4) == 0;
  for (int n = 0; n < N - 1; ++n) vec = vec && (a.stride[n] % 4 == 0);
  if (vec) {
    a.cpr = (a.L + 127) / 128;
    a.units = a.rows * a.cpr;
  } else {
    a.cpr = 0;
    a.units = (a.rows * a.L + 31) / 32;
  }
  const size_t smem = size_t(D) * (size_t(tot) + size_t(Jt)) * 4;
  const bool use_smem = smem <= 200 * 1024;

  DeviceGuard g(ctx->device);
  spec_cache_invalidate(ctx, out, sizeof(float) * size_t((nbatch - 1) * a.obs + D * Jt));
  // zero the output sketches
  {
    int64_t len = D * Jt;
    int blocks = int((len + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    zero_out_kernel<<<dim3(blocks, unsigned(nbatch)), 256, 0, ctx->stream>>>(out, len, a.obs);
    rc = check_cuda(ctx, cudaGetLastError(), "zero_out_kernel");
    if (rc) return rc;
  }
  const int threads = 1024;
  auto launch = [&](auto kern) -> int {
    const size_t sm = use_smem ? smem : 0;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(sm));
      if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(dense)");
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sm);
    if (per_sm < 1) per_sm = 1;
    int64_t want = int64_t(ctx->sm_count) * per_sm;         // CTAs in flight
    int64_t per_item = want / nbatch;   // one wave
    const int64_t need = (a.units * 32 + threads - 1) / threads;
    if (per_item > need) per_item = need;
    if (per_item < 1) per_item = 1;
    kern<<<dim3(unsigned(per_item), unsigned(nbatch)), threads, sm, ctx->stream>>>(a);
    return check_cuda(ctx, cudaGetLastError(), "dense_kernel");
  };
  // row-chunk kernel: contiguous last mode, 15-bit last-mode offsets.  The D
  // sketches are split into the fewest groups (one per blockIdx.z) whose
  // bins and tables fit in shared memory; each group reads T once.
  int64_t totL = tot - a.m.I[N - 1];
  const int cpr_rows = int((a.m.I[N - 1] + 255) / 256);
  auto rows_smem = [&](int dc) {
    return size_t(dc) * (size_t(totL) + size_t(Jt)) * 4 + size_t(dc) * size_t(cpr_rows) * 640;
  };
  int ngroups = 1;
  while (ngroups < D && rows_smem((D + ngroups - 1) / ngroups) > 200 * 1024) ++ngroups;
  const int DC = (D + ngroups - 1) / ngroups;
  const size_t smem_rows = rows_smem(DC);
  if (vec && a.m.J[N - 1] <= 32767 && smem_rows <= 200 * 1024 && a.rows < (int64_t(1) << 31)) {
    const int cpr = cpr_rows;
    auto launch_rows = [&](auto kern, int nt) -> int {
      if (smem_rows > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem_rows));
        if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(dense_rows)");
      }
      int per_sm = 1;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem_rows);
      if (per_sm < 1) per_sm = 1;
      // CTAs per (batch item, sketch group): one wave in total (a partial
      // second wave would double the time of the CTAs in it)
      const int64_t slots = int64_t(nbatch) * ngroups;
      int64_t per_item = (int64_t(ctx->sm_count) * per_sm) / slots;
      // no more warps than (rows x chunks) work units
      const int64_t need_warps = a.rows * cpr;
      const int64_t need = (need_warps * 32 + nt - 1) / nt;
      if (per_item > need) per_item = need;
      if (per_item < 1) per_item = 1;
      int64_t warps = per_item * (nt / 32);
      int64_t used = (warps / cpr) * cpr;
      if (used < cpr) {          // fewer warps than chunks: add CTAs
        per_item = (int64_t(cpr) * 32 + nt - 1) / nt;
        used = cpr;
      }
      kern<<<dim3(unsigned(per_item), unsigned(nbatch), unsigned(ngroups)), nt, smem_rows,
             ctx->stream>>>(a, int(totL), cpr, used, DC);
      return check_cuda(ctx, cudaGetLastError(), "dense_rows_kernel");
    };
    switch (N - 1) {
      case 0: return launch_rows(dense_rows_kernel<768, 0>, 768);
      case 1: return launch_rows(dense_rows_kernel<768, 1>, 768);
      case 2: return launch_rows(dense_rows_kernel<768, 2>, 768);
      case 3: return launch_rows(dense_rows_kernel<768, 3>, 768);
      default: return launch_rows(dense_rows_kernel<768, -1>, 768);
    }
  }
  if (vec)
    return use_smem ? launch(dense_kernel<true, true>) : launch(dense_kernel<true, false>);
  return use_smem ? launch(dense_kernel<false, true>) : launch(dense_kernel<false, false>);
}
