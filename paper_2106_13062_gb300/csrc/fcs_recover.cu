// fcs_recover.cu -- fcs_recover: entry estimates from sketches, the
// decompressing rule of the Kronecker / tensor-contraction compression
// subsections:
//   raw_d[q] = prod_n s_n(i_n) * sketch_d[ sum_n h_n(i_n) ],  out[q] = median_d.
// One thread per sample: N index loads, D table lookups per mode (tables
// staged in shared memory, h and the sign packed into one int32), D gathers
// from the sketches (L1/L2 resident), and the median in registers.
#include "fcs_internal.cuh"

namespace fcs {
namespace {

struct RecoverArgs {
  Modes m;
  const float *sketch;
  const int32_t *h;
  const int8_t *s;
  const int32_t *idx;
  float *out;
  float *raw;
  int64_t M;
  int64_t sbs, ibs, obs;   // batch strides
  int64_t nbatch;
  int tot;
};

template <int D, bool SMEM>
__global__ void __launch_bounds__(256) recover_kernel(RecoverArgs a) {
  extern __shared__ __align__(16) int32_t tab[];
  const int N = a.m.N, tot = a.tot;
  if (SMEM) {
    for (int e = threadIdx.x; e < D * tot; e += blockDim.x) {
      const int d = e / tot;
      const int64_t g = d * a.m.ldh + (e - d * tot);
      tab[e] = (a.h[g] << 1) | (a.s[g] < 0 ? 1 : 0);
    }
    __syncthreads();
  }
  const int64_t b = blockIdx.y;
  const float *sk = a.sketch + b * a.sbs;
  const int32_t *idx = a.idx + b * a.ibs;
  float *out = a.out + b * a.obs;
  const int64_t Jt = a.m.Jt;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < a.M;
       q += int64_t(gridDim.x) * blockDim.x) {
    int bin[D], neg[D];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < D; ++d) bin[d] = neg[d] = 0;
    for (int n = 0; n < N; ++n) {
      int64_t i = __ldcs(idx + q * N + n);
      if (i < 0 || i >= a.m.I[n]) {      // index outside the tensor: NaN result
        ok = false;
        i = 0;
      }
      const int64_t e = a.m.off[n] + i;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int32_t t =
            SMEM ? tab[d * tot + e]
                 : ((__ldg(a.h + d * a.m.ldh + e) << 1) | (__ldg(a.s + d * a.m.ldh + e) < 0));
        bin[d] += t >> 1;
        neg[d] ^= t & 1;
      }
    }
    float v[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const bool in = ok && unsigned(bin[d]) < unsigned(Jt);
      const float x = in ? __ldg(sk + d * Jt + bin[d]) : __int_as_float(0x7fc00000);
      v[d] = neg[d] ? -x : x;
      if (a.raw) a.raw[d * a.M + q] = v[d];
    }
    __stcs(out + q, median_inplace<D>(v));
  }
}

// Shared-memory variant: the batch item's D sketches and its hash tables are
// staged in shared memory first, so the D gathers and N*D table lookups of
// each sample hit shared memory instead of L1/L2.  Tables are packed as
// 16-bit (h << 1) | (s < 0) in index-major order (the D entries of one index
// are adjacent and read as 32-bit words).
template <int D>
__global__ void __launch_bounds__(512) recover_smem_kernel(RecoverArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int W = (D + 1) / 2;                   // 32-bit words per index row
  const int N = a.m.N, tot = a.tot;
  const int64_t Jt = a.m.Jt;
  float *sk = reinterpret_cast<float *>(smem);                                 // [D][Jt]
  uint32_t *tab = reinterpret_cast<uint32_t *>(smem + ((size_t(D) * Jt * 4 + 15) & ~size_t(15)));
  const int64_t b = blockIdx.y;
  const float *skg = a.sketch + b * a.sbs;
  for (int64_t e = threadIdx.x; e < D * Jt; e += blockDim.x) sk[e] = __ldg(skg + e);
  for (int e = threadIdx.x; e < tot * W; e += blockDim.x) {
    const int i = e / W, w = e - i * W;
    uint32_t v = 0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int d = 2 * w + q;
      if (d < D) {
        const int64_t g = d * a.m.ldh + i;
        v |= uint32_t(((a.h[g] << 1) | (a.s[g] < 0 ? 1 : 0)) & 0xffff) << (16 * q);
      }
    }
    tab[e] = v;
  }
  __syncthreads();
  const int32_t *idx = a.idx + b * a.ibs;
  float *out = a.out + b * a.obs;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < a.M;
       q += int64_t(gridDim.x) * blockDim.x) {
    int bin[D], neg[D];
#pragma unroll
    for (int d = 0; d < D; ++d) bin[d] = neg[d] = 0;
    bool ok = true;
    for (int n = 0; n < N; ++n) {
      int i = __ldcs(idx + q * N + n);
      if (i < 0 || i >= a.m.I[n]) {
        ok = false;
        i = 0;
      }
      const uint32_t *row = tab + (int(a.m.off[n]) + i) * W;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const uint32_t v = row[w];
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2) {
          const int d = 2 * w + q2;
          if (d < D) {
            const uint32_t t = (v >> (16 * q2)) & 0xffffu;
            bin[d] += int(t >> 1);
            neg[d] ^= int(t & 1u);
          }
        }
      }
    }
    float v[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const bool in = ok && unsigned(bin[d]) < unsigned(Jt);
      const float x = in ? sk[d * Jt + bin[d]] : __int_as_float(0x7fc00000);
      v[d] = neg[d] ? -x : x;
      if (a.raw) a.raw[d * a.M + q] = v[d];
    }
    __stcs(out + q, median_inplace<D>(v));
  }
}

// SIMD-table variant (Jt < 8192, N <= 7): each table entry is the 16-bit
// e = (h << 3) | (s < 0), two sketches per 32-bit word.  Summing the N modes'
// words with plain 32-bit adds gives, in each half, 8 * sum_n h + (number of
// negative signs): the sum stays below 2^16, so halves never carry into each
// other; the bin is the half >> 3 and the sign parity its low bit.  The
// sketches sit in shared memory; two samples per thread per iteration.
template <int D, bool RAW, bool IDX4>
__global__ void __launch_bounds__(1024) recover_simd_kernel(RecoverArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int W = (D + 1) / 2;
  const int N = a.m.N, tot = a.tot;
  const int Jt = int(a.m.Jt);
  float *sk = reinterpret_cast<float *>(smem);
  uint32_t *tab = reinterpret_cast<uint32_t *>(smem + ((size_t(D) * Jt * 4 + 15) & ~size_t(15)));
  // the tables are the same for every batch item: staged once
  for (int e = threadIdx.x; e < tot * W; e += blockDim.x) {
    const int i = e / W, w = e - i * W;
    uint32_t v = 0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int d = 2 * w + q;
      if (d < D) {
        const int64_t g = d * a.m.ldh + i;
        v |= uint32_t((a.h[g] << 3) | (a.s[g] < 0 ? 1 : 0)) << (16 * q);
      }
    }
    tab[e] = v;
  }
  const int32_t *idx = a.idx;
  float *out = a.out;
  const uint32_t M = uint32_t(a.M);
  int off[kMaxN], In[kMaxN];
#pragma unroll
  for (int n = 0; n < kMaxN; ++n) {
    off[n] = int(a.m.off[n]);
    In[n] = int(a.m.I[n]);
  }
  auto load = [&](uint32_t q, int *iv) {
    if (IDX4) {
      const int4 t = __ldcs(reinterpret_cast<const int4 *>(idx) + q);
      iv[0] = t.x; iv[1] = t.y; iv[2] = t.z; iv[3] = t.w;
    } else {
#pragma unroll
      for (int n = 0; n < kMaxN; ++n)
        if (n < N) iv[n] = __ldcs(idx + size_t(q) * N + n);
    }
  };
  auto one = [&](uint32_t q, const int *iv) {
    uint32_t acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = 0u;
    bool ok = true;
#pragma unroll
    for (int n = 0; n < kMaxN; ++n) {
      if (IDX4 ? n < 4 : n < N) {
        int i = iv[n];
        if (unsigned(i) >= unsigned(In[n])) {
          ok = false;
          i = 0;
        }
        const uint32_t *row = tab + (off[n] + i) * W;
#pragma unroll
        for (int w = 0; w < W; ++w) acc[w] += row[w];
      }
    }
    float v[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const uint32_t half = (acc[d >> 1] >> (16 * (d & 1))) & 0xffffu;
      const int bin = int(half >> 3);
      const float x = (ok && bin < Jt) ? sk[d * Jt + bin] : __int_as_float(0x7fc00000);
      v[d] = (half & 1u) ? -x : x;
      if (RAW) a.raw[size_t(d) * M + q] = v[d];
    }
    __stcs(out + q, median_net<D>(v));
  };
  // CTA k takes the k-th equal share of the flattened (item, sample) range,
  // so one wave of CTAs covers every item; the sketches of each item the
  // share touches (at most a few) are staged in turn.
  const int64_t S = a.nbatch * a.M;
  const int64_t lo = S * blockIdx.x / gridDim.x, hi = S * (blockIdx.x + 1) / gridDim.x;
  constexpr int U = 4;
  const uint32_t stride = blockDim.x;
  for (int64_t pos = lo; pos < hi;) {
    const int64_t b = pos / a.M;
    const int64_t end = min(hi, (b + 1) * a.M);
    __syncthreads();                         // readers of the previous sketches are done
    const float *skg = a.sketch + b * a.sbs;
    for (int e = threadIdx.x; e < D * Jt; e += blockDim.x) sk[e] = __ldg(skg + e);
    __syncthreads();
    idx = a.idx + b * a.ibs;
    out = a.out + b * a.obs;
    const uint32_t q1 = uint32_t(end - b * a.M);
    uint32_t q = uint32_t(pos - b * a.M) + threadIdx.x;
    // four samples per iteration: all index loads are issued before any use
    for (; q + (U - 1) * stride < q1; q += U * stride) {
      int iv[U][kMaxN];
#pragma unroll
      for (int u = 0; u < U; ++u) load(q + u * stride, iv[u]);
#pragma unroll
      for (int u = 0; u < U; ++u) one(q + u * stride, iv[u]);
    }
    for (; q < q1; q += stride) {
      int iv[kMaxN];
      load(q, iv);
      one(q, iv);
    }
    pos = end;
  }
}

template <int D>
int launch_recover(fcs_ctx *ctx, RecoverArgs &a, int64_t nbatch) {
  {
    // staged variant when sketches and 16-bit tables fit in shared memory
    bool j16 = true;
    for (int n = 0; n < a.m.N; ++n) j16 = j16 && a.m.J[n] <= 32767;
    const size_t sm2 = ((size_t(D) * a.m.Jt * 4 + 15) & ~size_t(15)) +
                       size_t(a.tot) * ((D + 1) / 2) * 4;
    if (a.m.Jt < 8192 && a.m.N <= 7 && sm2 <= 220 * 1024 && a.M < (int64_t(1) << 31)) {
      const bool idx4 = a.m.N == 4 && (reinterpret_cast<uintptr_t>(a.idx) & 15) == 0 &&
                        (a.ibs % 4) == 0;
      auto pick = [&](auto kern) -> int {
        if (sm2 > 48 * 1024) {
          cudaError_t e =
              cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm2));
          if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(recover_simd)");
        }
        int per_sm = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 1024, sm2);
        if (per_sm < 1) per_sm = 1;
        // one wave of CTAs over all items' samples (a few thousand per CTA)
        int64_t grid = int64_t(ctx->sm_count) * per_sm;
        const int64_t need = (nbatch * a.M + 4095) / 4096;
        if (grid > need) grid = need;
        if (grid < 1) grid = 1;
        kern<<<unsigned(grid), 1024, sm2, ctx->stream>>>(a);
        return check_cuda(ctx, cudaGetLastError(), "recover_simd_kernel");
      };
      if (a.raw) return idx4 ? pick(recover_simd_kernel<D, true, true>)
                             : pick(recover_simd_kernel<D, true, false>);
      return idx4 ? pick(recover_simd_kernel<D, false, true>)
                  : pick(recover_simd_kernel<D, false, false>);
    }
    if (j16 && sm2 <= 220 * 1024 && a.tot < (1 << 30)) {
      auto kern = recover_smem_kernel<D>;
      if (sm2 > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm2));
        if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(recover_smem)");
      }
      int per_sm = 1;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, sm2);
      if (per_sm < 1) per_sm = 1;
      int64_t per_item = (int64_t(ctx->sm_count) * per_sm) / nbatch;   // one wave
      const int64_t need = (a.M + 511) / 512;
      if (per_item > need) per_item = need;
      if (per_item < 1) per_item = 1;
      kern<<<dim3(unsigned(per_item), unsigned(nbatch)), 512, sm2, ctx->stream>>>(a);
      return check_cuda(ctx, cudaGetLastError(), "recover_smem_kernel");
    }
  }
  const size_t smem = size_t(D) * a.tot * sizeof(int32_t);
  const bool use_smem = smem <= 96 * 1024;
  auto kern = use_smem ? recover_kernel<D, true> : recover_kernel<D, false>;
  const size_t sm = use_smem ? smem : 0;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(recover)");
  }
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm);
  if (per_sm < 1) per_sm = 1;
  int64_t want = int64_t(ctx->sm_count) * per_sm;
  int64_t per_item = want / nbatch;   // one wave
  const int64_t need = (a.M + 255) / 256;
  if (per_item > need) per_item = need;
  if (per_item < 1) per_item = 1;
  kern<<<dim3(unsigned(per_item), unsigned(nbatch)), 256, sm, ctx->stream>>>(a);
  return check_cuda(ctx, cudaGetLastError(), "recover_kernel");
}

}  // namespace
}  // namespace fcs

using namespace fcs;

extern "C" int fcs_recover(fcs_ctx *ctx, int N, const int64_t *host_I, const int32_t *host_J,
                           int D, const float *sketch, const int32_t *h, const int8_t *s,
                           int64_t ldh, int64_t M, const int32_t *idx, float *out,
                           float *out_raw, int64_t nbatch, int64_t sketch_batch_stride,
                           int64_t idx_batch_stride, int64_t out_batch_stride) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  RecoverArgs a{};
  int rc = make_modes(ctx, N, host_I, host_J, ldh, &a.m);
  if (rc) return rc;
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (M < 0) return set_error(ctx, FCS_EINVAL, "M=%lld < 0", (long long)M);
  if (nbatch < 1 || nbatch > 65535)
    return set_error(ctx, FCS_EINVAL, "nbatch=%lld outside [1,65535]", (long long)nbatch);
  if (nbatch > 1 && out_raw)
    return set_error(ctx, FCS_EINVAL, "out_raw must be NULL when nbatch > 1");
  if (M == 0) return FCS_OK;
  if (!sketch || !h || !s || !idx || !out) return set_error(ctx, FCS_EINVAL, "NULL pointer");
  int64_t tot = 0;
  for (int n = 0; n < N; ++n) tot += host_I[n];
  a.tot = int(tot);
  a.sketch = sketch;
  a.h = h;
  a.s = s;
  a.idx = idx;
  a.out = out;
  a.raw = out_raw;
  a.M = M;
  a.sbs = nbatch > 1 ? sketch_batch_stride : 0;
  a.ibs = nbatch > 1 ? idx_batch_stride : 0;
  a.obs = nbatch > 1 ? out_batch_stride : 0;
  a.nbatch = nbatch;
  DeviceGuard g(ctx->device);
  switch (D) {
#define FCS_REC_CASE(K) \
  case K: return launch_recover<K>(ctx, a, nbatch);
    FCS_REC_CASE(1) FCS_REC_CASE(2) FCS_REC_CASE(3) FCS_REC_CASE(4) FCS_REC_CASE(5)
    FCS_REC_CASE(6) FCS_REC_CASE(7) FCS_REC_CASE(8) FCS_REC_CASE(9) FCS_REC_CASE(10)
    FCS_REC_CASE(11) FCS_REC_CASE(12) FCS_REC_CASE(13) FCS_REC_CASE(14) FCS_REC_CASE(15)
    FCS_REC_CASE(16)
#undef FCS_REC_CASE
    default:
      break;
  }
  return set_error(ctx, FCS_EINVAL, "D=%d outside [1,16]", D);
}
