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
  auto add = [&](int d, int64_t bin, float v) {
    if (bin < 0 || bin >= Jt) return;     // hash value outside [0, J_n): skip
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
        for (int n = 0; n < N - 1; ++n) {
          const int32_t t = entry(d, a.m.off[n] + idx[n]);
          base += t >> 1;
          neg ^= t & 1;
        }
        if (active) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int32_t t = entry(d, a.m.off[N - 1] + il + k);
            const float x = ((neg ^ t) & 1) ? -vv[k] : vv[k];
            add(d, base + (t >> 1), x);
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
          for (int n = 0; n < N; ++n) {
            const int32_t t = entry(d, a.m.off[n] + idx[n]);
            bin += t >> 1;
            neg ^= t & 1;
          }
          add(d, bin, neg ? -x : x);
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
// changes, the lane's last-mode hash/sign entries for all D sketches stay in
// registers (16-bit packed pairs) for the whole kernel; only the leading
// modes' entries are read from shared memory, once per row and sketch.  The
// next row's values are prefetched while the current row is scattered.
template <int D, int NT>
__global__ void __launch_bounds__(NT) dense_rows_kernel(DenseArgs a, int totL, int cpr,
                                                        int64_t warps_used) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.m.N;
  const int64_t Jt = a.m.Jt;
  int32_t *tab = reinterpret_cast<int32_t *>(smem);       // [D][totL] leading modes
  float *bins = reinterpret_cast<float *>(tab + D * totL);  // [D][Jt]
  for (int e = threadIdx.x; e < D * totL; e += NT) {
    const int d = e / totL;
    tab[e] = packed_entry(a, d, e - d * totL);
  }
  for (int64_t e = threadIdx.x; e < D * Jt; e += NT) bins[e] = 0.f;

  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * int64_t(NT) + threadIdx.x) >> 5;
  const int c = int(gw % cpr);
  const int64_t rstride = warps_used / cpr;
  const int64_t i0 = int64_t(c) * 256 + lane * 4;      // segment s starts at i0 + 128 s
  const bool act0 = i0 < a.L, act1 = i0 + 128 < a.L;
  // last-mode entries: word[d][m] packs elements 2m (low) and 2m+1 (high)
  uint32_t tl[D][4];
  {
    const int64_t offl = a.m.off[N - 1];
#pragma unroll
    for (int d = 0; d < D; ++d)
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        uint32_t w = 0;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int e = 2 * m + q;                      // element: segment e/4, lane slot e%4
          const int64_t i = i0 + (e >> 2) * 128 + (e & 3);
          if (i < a.L) w |= uint32_t(packed_entry(a, d, int(offl + i)) & 0xffff) << (16 * q);
        }
        tl[d][m] = w;
      }
  }
  __syncthreads();

  const int b = blockIdx.y;
  const float *Tb = a.T + b * a.tbs;
  float *outb = a.out + b * a.obs;
  // rows < 2^31 and I_n < 2^31 here, so 32-bit division suffices
  auto row_addr = [&](int64_t row, int *idx) {
    uint32_t rr = uint32_t(row);
    int64_t addr = 0;
#pragma unroll
    for (int n = kMaxN - 2; n >= 0; --n) {
      if (n < N - 1) {
        const uint32_t In = uint32_t(a.m.I[n]);
        const uint32_t q = rr / In;
        idx[n] = int(rr - q * In);
        rr = q;
        addr += idx[n] * a.stride[n];
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

  int64_t row = gw / cpr;
  const bool working = gw < warps_used;
  int idx[kMaxN], nidx[kMaxN];
#pragma unroll
  for (int n = 0; n < kMaxN; ++n) idx[n] = nidx[n] = 0;
  float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
  if (working && row < a.rows) load(row_addr(row, nidx), n0, n1);
  for (; working && row < a.rows; row += rstride) {
#pragma unroll
    for (int n = 0; n < kMaxN; ++n) idx[n] = nidx[n];
    const float v[8] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
    if (row + rstride < a.rows) load(row_addr(row + rstride, nidx), n0, n1);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      int base = 0, neg = 0;
#pragma unroll
      for (int n = 0; n < kMaxN - 1; ++n) {
        if (n < N - 1) {
          const int32_t t = tab[d * totL + int(a.m.off[n] + idx[n])];
          base += t >> 1;
          neg ^= t & 1;
        }
      }
      float *bd = bins + d * Jt;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        if ((e < 4) ? act0 : act1) {
          const uint32_t t = (tl[d][e >> 1] >> (16 * (e & 1))) & 0xffffu;
          const int bin = base + int(t >> 1);
          const float x = ((uint32_t(neg) ^ t) & 1u) ? -v[e] : v[e];
          if (unsigned(bin) < unsigned(Jt)) atomicAdd(bd + bin, x);
        }
      }
    }
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < D * Jt; e += NT) {
    const float x = bins[e];
    if (x != 0.f) atomicAdd(&outb[e], x);
  }
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
  a.L = host_I[N - 1];
  a.rows = 1;
  for (int n = 0; n < N - 1; ++n) a.rows *= host_I[n];

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
    int64_t per_item = (want + nbatch - 1) / nbatch;
    const int64_t need = (a.units * 32 + threads - 1) / threads;
    if (per_item > need) per_item = need;
    if (per_item < 1) per_item = 1;
    kern<<<dim3(unsigned(per_item), unsigned(nbatch)), threads, sm, ctx->stream>>>(a);
    return check_cuda(ctx, cudaGetLastError(), "dense_kernel");
  };
  // row-chunk kernel: contiguous last mode, 16-bit last-mode entries
  int64_t totL = tot - host_I[N - 1];
  const size_t smem_rows = size_t(D) * (size_t(totL) + size_t(Jt)) * 4;
  if (vec && host_J[N - 1] <= 32767 && smem_rows <= 200 * 1024 && a.rows < (int64_t(1) << 31)) {
    const int cpr = int((a.L + 255) / 256);
    auto launch_rows = [&](auto kern, int nt) -> int {
      if (smem_rows > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem_rows));
        if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(dense_rows)");
      }
      int per_sm = 1;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem_rows);
      if (per_sm < 1) per_sm = 1;
      int64_t per_item = (int64_t(ctx->sm_count) * per_sm + nbatch - 1) / nbatch;
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
      kern<<<dim3(unsigned(per_item), unsigned(nbatch)), nt, smem_rows, ctx->stream>>>(
          a, int(totL), cpr, used);
      return check_cuda(ctx, cudaGetLastError(), "dense_rows_kernel");
    };
    switch (D) {
#define FCS_DR_CASE(K)                                          \
  case K: {                                                     \
    constexpr int kNT = (K <= 4) ? 1024 : 512;                  \
    return launch_rows(dense_rows_kernel<K, kNT>, kNT);         \
  }
      FCS_DR_CASE(1) FCS_DR_CASE(2) FCS_DR_CASE(3) FCS_DR_CASE(4) FCS_DR_CASE(5)
      FCS_DR_CASE(6) FCS_DR_CASE(7) FCS_DR_CASE(8) FCS_DR_CASE(9) FCS_DR_CASE(10)
      FCS_DR_CASE(11) FCS_DR_CASE(12) FCS_DR_CASE(13) FCS_DR_CASE(14) FCS_DR_CASE(15)
      FCS_DR_CASE(16)
#undef FCS_DR_CASE
      default:
        break;
    }
  }
  if (vec)
    return use_smem ? launch(dense_kernel<true, true>) : launch(dense_kernel<true, false>);
  return use_smem ? launch(dense_kernel<false, true>) : launch(dense_kernel<false, false>);
}
