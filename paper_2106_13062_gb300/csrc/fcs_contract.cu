// fcs_contract.cu -- fcs_contract: the sketched contractions of Sec. 4.1.
//
//  ALL  (eq. T_uvw):  e_d = <FCS_d(T), FCS_d(v_1 o ... o v_N)>
//       = (1/P) Re sum_{k<P} conj(F(FCS_d T))[k] prod_n F(CS_n v_n)[k]
//       (Parseval; FCS_d of the rank-1 tensor is the product of the per-mode
//       spectra by eq. FCS_syn with R = 1).
//  FREE (eq. T_Ivw, free mode m; also the ALS columns of Sec. 4.1.2):
//       z_d = IFFT(F(FCS_d T) prod_{n != m} conj F(CS_n v_n)),
//       est_d[i] = s_m(i) z_d[h_m(i)]   (exact for P >= Jt: the circular
//       correlation never wraps at the lags h_m(i) < J_m).
//  Then the median over the D sketches (Sec. 4 opening).
//
// Kernels: (1) the half spectra of the D sketches of T; (2) one CTA per
// (batch item, sketch) that builds each needed Count Sketch in shared memory,
// transforms it and folds it into the per-thread spectrum product, then either
// reduces the Parseval sum or runs the inverse FFT and gathers; (3) the median.
//
// With fcs_cache_spectra enabled, the spectra of (1) are kept in a
// per-context cache keyed by the sketch pointer and shape, so repeated
// contractions against one sketch (the RTPM and ALS loops) transform it
// once.  fcs_forget drops an entry; the library's own sketch calls drop the
// entries of the buffers they overwrite.
#include <vector>

#include "fcs_fft.cuh"

struct fcs_spec_cache {
  struct Entry {
    const float *key;
    int64_t Jt;
    int D;
    int log2m;
    float2 *spec;
    size_t bytes;
    cudaEvent_t ready;   // spectrum written
    cudaEvent_t used;    // last contraction that read it
    uint64_t tick;
    bool stale;          // key's contents may have changed: recompute on next use
  };
  std::vector<Entry> e;
  size_t bytes = 0;
  uint64_t tick = 0;
};

namespace fcs {
namespace {

constexpr int kSpecCacheEntries = 16;
constexpr size_t kSpecCacheMaxBytes = size_t(512) << 20;

void spec_entry_free(fcs_spec_cache::Entry &x) {
  cudaEventSynchronize(x.used);
  cudaEventDestroy(x.ready);
  cudaEventDestroy(x.used);
  cudaFree(x.spec);
}

void spec_cache_erase(fcs_spec_cache *c, size_t i) {
  spec_entry_free(c->e[i]);
  c->bytes -= c->e[i].bytes;
  c->e.erase(c->e.begin() + i);
}

// Entry for (key, Jt, D, log2m): an existing one (hit = true) or a new one
// whose spectrum the caller must compute; nullptr when it cannot be cached.
fcs_spec_cache::Entry *spec_cache_get(fcs_ctx *ctx, const float *key, int64_t Jt, int D,
                                      int log2m, bool *hit) {
  *hit = false;
  if (!ctx->cache_spectra) return nullptr;
  if (!ctx->spec_cache) ctx->spec_cache = new (std::nothrow) fcs_spec_cache();
  fcs_spec_cache *c = ctx->spec_cache;
  if (!c) return nullptr;
  ++c->tick;
  for (auto &x : c->e) {
    if (x.key == key && x.Jt == Jt && x.D == D && x.log2m == log2m) {
      x.tick = c->tick;
      if (x.stale) {
        // recompute into the same memory once its last readers are done
        if (cudaStreamWaitEvent(ctx->stream, x.used, 0) != cudaSuccess) {
          cudaGetLastError();
          return nullptr;
        }
        x.stale = false;
        return &x;
      }
      *hit = true;
      return &x;
    }
  }
  const size_t bytes = sizeof(float2) * size_t(D) * ((size_t(1) << log2m) + 1);
  const size_t cap = ctx->budget / 2 < kSpecCacheMaxBytes ? ctx->budget / 2 : kSpecCacheMaxBytes;
  if (bytes > cap) return nullptr;
  while (!c->e.empty() && (c->bytes + bytes > cap || int(c->e.size()) >= kSpecCacheEntries)) {
    size_t lru = 0;
    for (size_t i = 1; i < c->e.size(); ++i)
      if (c->e[i].tick < c->e[lru].tick) lru = i;
    spec_cache_erase(c, lru);
  }
  fcs_spec_cache::Entry x{key, Jt, D, log2m, nullptr, bytes, nullptr, nullptr, c->tick, false};
  if (cudaMalloc(&x.spec, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (cudaEventCreateWithFlags(&x.ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&x.used, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (x.ready) cudaEventDestroy(x.ready);
    cudaFree(x.spec);
    return nullptr;
  }
  c->e.push_back(x);
  c->bytes += bytes;
  return &c->e.back();
}

struct ContractArgs {
  Modes m;
  int D;
  int kind;
  int free_mode;
  int64_t B;
  const float *fcsT;      // [D][Jt]
  const float *vec[kMaxN];
  const int32_t *h;
  const int8_t *s;
  float2 *spec;           // [D][M+1]
  float *raw;             // [B][D] or [B][D][I_m]
  float *raw_all;         // kBoth: the T(v_1..v_N) estimates [B][D]
  float *out;             // [B] or [B][I_m]
  int sb;                 // compact count-sketch buffer (floats, multiple of 4)
};

// Half spectrum of each of the D sketches of T, natural order [D][M+1]: the
// sketch is read into the compact real buffer and transformed by the block
// real FFT whose last pass leaves the spectrum in registers.
template <int LOG2M, int NT>
__global__ void __launch_bounds__(NT) spectrum_kernel(const float *__restrict__ x, int64_t len,
                                                      int64_t ld, int sb,
                                                      float2 *__restrict__ spec,
                                                      const float2 *__restrict__ tw) {
  using LPs = LastPass<LOG2M, NT>;
  using Lay = FftSmem<LOG2M>;
  constexpr int M = 1 << LOG2M;
  constexpr int RL = LPs::RL, EPS = LPs::EPS;
  extern __shared__ __align__(16) unsigned char smem[];
  float2 *B = reinterpret_cast<float2 *>(smem + Lay::kB);
  float2 *tws = reinterpret_cast<float2 *>(smem + Lay::kTw);
  float *A = reinterpret_cast<float *>(smem + Lay::kA);
  const float *xd = x + blockIdx.x * ld;
  fill_twiddles<LOG2M, NT>(tws, tw);
  float2 *lps = reinterpret_cast<float2 *>(smem + Lay::kLp);
  LastPassTwShared<LOG2M, NT>::fill(lps, tw);
  const LastPassTwShared<LOG2M, NT> ltw{lps};
  for (int j = threadIdx.x; j < sb; j += NT) A[j] = j < len ? __ldg(xd + j) : 0.f;
  float2 X[EPS][2][RL];
  rfft_to_slots<LOG2M, NT>(A, sb, B, tws, ltw, X);
  float2 *sd = spec + blockIdx.x * int64_t(M + 1);
#pragma unroll
  for (int e = 0; e < EPS; ++e) {
    if (LPs::SLOTS % NT != 0 && int(threadIdx.x) + e * NT >= LPs::SLOTS) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int q = last_pass_index<LOG2M, NT>(e, b, r);
        if (q == 0) {
          sd[0] = make_float2(X[e][b][r].x, 0.f);
          sd[M] = make_float2(X[e][b][r].y, 0.f);
        } else {
          sd[q] = X[e][b][r];
        }
      }
  }
}

// Internal kind: both contractions of one vector set from one set of
// transforms (fcs_contract_both).
constexpr int kBoth = 2;

template <int LOG2M, int NT>
__global__ void __launch_bounds__(NT) contract_kernel(ContractArgs a,
                                                      const float2 *__restrict__ tw) {
  using LPs = LastPass<LOG2M, NT>;
  using Lay = FftSmem<LOG2M>;
  constexpr int M = 1 << LOG2M;
  constexpr int RL = LPs::RL, EPS = LPs::EPS;
  extern __shared__ __align__(16) unsigned char smem[];
  float2 *B = reinterpret_cast<float2 *>(smem + Lay::kB);
  float2 *tws = reinterpret_cast<float2 *>(smem + Lay::kTw);
  float *A = reinterpret_cast<float *>(smem + Lay::kA);
  __shared__ float red[NT / 32];
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x;
  const int d = blockIdx.y;
  const bool all = a.kind == FCS_CONTRACT_ALL;
  const int sb = a.sb;
  const float2 *sd = a.spec + d * int64_t(M + 1);
  fill_twiddles<LOG2M, NT>(tws, tw);
  float2 *lps = reinterpret_cast<float2 *>(smem + Lay::kLp);
  LastPassTwShared<LOG2M, NT>::fill(lps, tw);
  const LastPassTwShared<LOG2M, NT> ltw{lps};
  for (int e = tid; e < sb / 4; e += NT)
    reinterpret_cast<float4 *>(A)[e] = make_float4(0.f, 0.f, 0.f, 0.f);

  // spectrum of FCS_d(T) in this thread's slots, and the running product
  float2 F[EPS][2][RL], p[EPS][2][RL], X[EPS][2][RL];
#pragma unroll
  for (int e = 0; e < EPS; ++e)
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const bool live = LPs::SLOTS % NT == 0 || tid + e * NT < LPs::SLOTS;
        const int q = live ? last_pass_index<LOG2M, NT>(e, bb, r) : 1;
        F[e][bb][r] = live ? (q == 0 ? make_float2(sd[0].x, sd[M].x) : sd[q])
                           : make_float2(0.f, 0.f);
        // multiplicative identity; the q = 0 slot packs two reals
        p[e][bb][r] = all ? make_float2(1.f, q == 0 ? 1.f : 0.f) : F[e][bb][r];
      }

  for (int n = 0; n < a.m.N; ++n) {
    if (!all && n == a.free_mode) continue;
    __syncthreads();
    const int32_t *hn = a.h + d * a.m.ldh + a.m.off[n];
    const int8_t *sn = a.s + d * a.m.ldh + a.m.off[n];
    const float *vn = a.vec[n] + b * a.m.I[n];
    for (int64_t i = tid; i < a.m.I[n]; i += NT) {
      float v = __ldg(vn + i);
      if (__ldg(sn + i) < 0) v = -v;
      const int hb = __ldg(hn + i);
      if (unsigned(hb) < unsigned(sb)) atomicAdd(A + hb, v);
    }
    rfft_to_slots<LOG2M, NT>(A, sb, B, tws, ltw, X);
#pragma unroll
    for (int e = 0; e < EPS; ++e)
#pragma unroll
      for (int bb = 0; bb < 2; ++bb)
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const bool packed = bb == 0 && r == 0 && tid + e * NT == 0;
          p[e][bb][r] = all ? slot_mul(p[e][bb][r], X[e][bb][r], packed)
                            : slot_mulconj(p[e][bb][r], X[e][bb][r], packed);
        }
  }

  if (all) {
    // sum_{k<P} conj(F_T[k]) Y[k]: the packed q = 0 slot holds the real bins
    // 0 and M (weight 1); every other bin q in (0, M) appears twice
    float part = 0.f;
#pragma unroll
    for (int e = 0; e < EPS; ++e) {
      if (LPs::SLOTS % NT != 0 && tid + e * NT >= LPs::SLOTS) continue;
#pragma unroll
      for (int bb = 0; bb < 2; ++bb)
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const bool packed = bb == 0 && r == 0 && tid + e * NT == 0;
          const float dot = F[e][bb][r].x * p[e][bb][r].x + F[e][bb][r].y * p[e][bb][r].y;
          part += packed ? dot : 2.f * dot;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int w = 0; w < NT / 32; ++w) t += red[w];
      a.raw[b * a.D + d] = t / float(2 * M);
    }
    return;
  }

  if (a.kind == kBoth) {
    // p = F_T prod_{n != m} conj(F_n), so conj(p) F_m = conj(F_T) prod_n F_n:
    // T(v_1..v_N) is the Parseval sum of Re(conj(p) F_m) over the free
    // mode's transform, taken before p goes into the inverse transform
    const int m = a.free_mode;
    __syncthreads();
    const int32_t *hn = a.h + d * a.m.ldh + a.m.off[m];
    const int8_t *sn = a.s + d * a.m.ldh + a.m.off[m];
    const float *vn = a.vec[m] + b * a.m.I[m];
    for (int64_t i = tid; i < a.m.I[m]; i += NT) {
      float v = __ldg(vn + i);
      if (__ldg(sn + i) < 0) v = -v;
      const int hb = __ldg(hn + i);
      if (unsigned(hb) < unsigned(sb)) atomicAdd(A + hb, v);
    }
    rfft_to_slots<LOG2M, NT>(A, sb, B, tws, ltw, X);
    float part = 0.f;
#pragma unroll
    for (int e = 0; e < EPS; ++e) {
      if (LPs::SLOTS % NT != 0 && tid + e * NT >= LPs::SLOTS) continue;
#pragma unroll
      for (int bb = 0; bb < 2; ++bb)
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const bool packed = bb == 0 && r == 0 && tid + e * NT == 0;
          const float dot = p[e][bb][r].x * X[e][bb][r].x + p[e][bb][r].y * X[e][bb][r].y;
          part += packed ? dot : 2.f * dot;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int w = 0; w < NT / 32; ++w) t += red[w];
      a.raw_all[b * a.D + d] = t / float(2 * M);
    }
  }

  // FREE: inverse transform of the product, then gather at h_m(i)
  slots_to_conj_packed<LOG2M, NT>(B, p, tw);
  __syncthreads();
  block_fft<LOG2M, NT>(B, tw);
  const int m = a.free_mode;
  const int32_t *hm = a.h + d * a.m.ldh + a.m.off[m];
  const int8_t *sm = a.s + d * a.m.ldh + a.m.off[m];
  const int64_t Im = a.m.I[m];
  float *rawbd = a.raw + (b * a.D + d) * Im;
  const float sc = 1.0f / float(M);
  const float *bufr = reinterpret_cast<const float *>(B);
  for (int64_t i = tid; i < Im; i += NT) {
    const int pz = __ldg(hm + i);
    const float v = unsigned(pz) < unsigned(2 * M) ? bufr[real_off(pz)] : __int_as_float(0x7fc00000);
    const float z = (pz & 1) ? -v * sc : v * sc;
    rawbd[i] = __ldg(sm + i) < 0 ? -z : z;
  }
}

template <int D>
__global__ void median_kernel(const float *__restrict__ raw, int64_t B, int64_t width,
                              float *__restrict__ out) {
  // raw [B][D][width] -> out [B][width]
  const int64_t total = B * width;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = t / width, i = t - b * width;
    float v[D];
#pragma unroll
    for (int d = 0; d < D; ++d) v[d] = raw[(b * D + d) * width + i];
    out[t] = median_inplace<D>(v);
  }
}

template <int LOG2M>
int launch_contract(fcs_ctx *ctx, ContractArgs &a, int64_t Jt, bool need_spec,
                    cudaEvent_t spec_ready) {
  constexpr int NT = fft_threads(LOG2M);
  const int sb_spec = int((Jt + 3) / 4 * 4);
  const size_t smem1 = FftSmem<LOG2M>::bytes(sb_spec);
  const size_t smem2 = FftSmem<LOG2M>::bytes(a.sb);
  auto k1 = spectrum_kernel<LOG2M, NT>;
  auto k2 = contract_kernel<LOG2M, NT>;
  cudaError_t e = cudaSuccess;
  if (smem1 > 48 * 1024)
    e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem1));
  if (e == cudaSuccess && smem2 > 48 * 1024)
    e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem2));
  if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(contract)");
  if (need_spec) {
    k1<<<a.D, NT, smem1, ctx->stream>>>(a.fcsT, Jt, Jt, sb_spec, a.spec, ctx->twiddle);
    int rc = check_cuda(ctx, cudaGetLastError(), "spectrum_kernel");
    if (rc) return rc;
    if (spec_ready) {
      rc = check_cuda(ctx, cudaEventRecord(spec_ready, ctx->stream), "cudaEventRecord");
      if (rc) return rc;
    }
  }
  k2<<<dim3(unsigned(a.B), unsigned(a.D)), NT, smem2, ctx->stream>>>(a, ctx->twiddle);
  return check_cuda(ctx, cudaGetLastError(), "contract_kernel");
}

int launch_median(fcs_ctx *ctx, int D, const float *raw, int64_t B, int64_t width,
                  float *out) {
  const int64_t total = B * width;
  int blocks = int((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  switch (D) {
#define FCS_MED_CASE(K) \
  case K: median_kernel<K><<<blocks, 256, 0, ctx->stream>>>(raw, B, width, out); break;
    FCS_MED_CASE(1) FCS_MED_CASE(2) FCS_MED_CASE(3) FCS_MED_CASE(4) FCS_MED_CASE(5)
    FCS_MED_CASE(6) FCS_MED_CASE(7) FCS_MED_CASE(8) FCS_MED_CASE(9) FCS_MED_CASE(10)
    FCS_MED_CASE(11) FCS_MED_CASE(12) FCS_MED_CASE(13) FCS_MED_CASE(14) FCS_MED_CASE(15)
    FCS_MED_CASE(16)
#undef FCS_MED_CASE
    default:
      return set_error(ctx, FCS_EINVAL, "D=%d outside [1,16]", D);
  }
  return check_cuda(ctx, cudaGetLastError(), "median_kernel");
}

}  // namespace

void spec_cache_invalidate(fcs_ctx *ctx, const void *p, size_t bytes) {
  fcs_spec_cache *c = ctx ? ctx->spec_cache : nullptr;
  if (!c) return;
  const char *lo = static_cast<const char *>(p);
  for (auto &x : c->e) {
    const char *k = reinterpret_cast<const char *>(x.key);
    if (k >= lo && k < lo + bytes) x.stale = true;
  }
}

void spec_cache_destroy(fcs_ctx *ctx) {
  fcs_spec_cache *c = ctx->spec_cache;
  if (!c) return;
  while (!c->e.empty()) spec_cache_erase(c, c->e.size() - 1);
  delete c;
  ctx->spec_cache = nullptr;
}

}  // namespace fcs

using namespace fcs;

extern "C" int fcs_cache_spectra(fcs_ctx *ctx, int enable) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  DeviceGuard g(ctx->device);
  if (!enable) spec_cache_destroy(ctx);
  ctx->cache_spectra = enable != 0;
  return FCS_OK;
}

extern "C" int fcs_forget(fcs_ctx *ctx, const void *ptr) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  fcs_spec_cache *c = ctx->spec_cache;
  if (!c || !ptr) return FCS_OK;
  for (auto &x : c->e)
    if (x.key == ptr) x.stale = true;        // recomputed on next use; no host wait
  return FCS_OK;
}

namespace {

// fcs_contract (kind ALL or FREE) and fcs_contract_both (kind kBoth: the FREE
// result in out_median / out_raw, the ALL result in out_all / out_all_raw).
int contract_call(fcs_ctx *ctx, int kind, int free_mode, int N, const int64_t *host_I,
                  const int32_t *host_J, int D, const float *fcsT, int64_t B,
                  const float *const *host_vecs, const int32_t *h, const int8_t *s,
                  int64_t ldh, float *out_median, float *out_raw, float *out_all,
                  float *out_all_raw) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  ContractArgs a{};
  int rc = make_modes(ctx, N, host_I, host_J, ldh, &a.m);
  if (rc) return rc;
  if (kind != FCS_CONTRACT_ALL && kind != FCS_CONTRACT_FREE && kind != kBoth)
    return set_error(ctx, FCS_EINVAL, "unknown contraction kind %d", kind);
  if (kind != FCS_CONTRACT_ALL && (free_mode < 0 || free_mode >= N))
    return set_error(ctx, FCS_EINVAL, "free_mode=%d outside [0,%d)", free_mode, N);
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (B < 1 || B > 65535) return set_error(ctx, FCS_EINVAL, "B=%lld outside [1,65535]", (long long)B);
  if (!fcsT || !host_vecs || !h || !s || !out_median || (kind == kBoth && !out_all))
    return set_error(ctx, FCS_EINVAL, "NULL pointer argument");
  for (int n = 0; n < N; ++n) {
    if (kind == FCS_CONTRACT_FREE && n == free_mode) {
      a.vec[n] = nullptr;
      continue;
    }
    if (!host_vecs[n]) return set_error(ctx, FCS_EINVAL, "vector %d is NULL", n);
    a.vec[n] = host_vecs[n];
  }
  const int log2p = ilog2_ceil(a.m.Jt) < kMinLog2P ? kMinLog2P : ilog2_ceil(a.m.Jt);
  if (log2p > kMaxLog2PBig)
    return set_error(ctx, FCS_EUNSUPPORTED, "Jt=%lld needs FFT length > %d",
                     (long long)a.m.Jt, 1 << kMaxLog2PBig);
  const int log2m = log2p - 1;
  const int64_t M = int64_t(1) << log2m;
  a.D = D;
  a.kind = kind;
  a.free_mode = free_mode;
  a.B = B;
  a.fcsT = fcsT;
  a.h = h;
  a.s = s;
  a.out = out_median;
  {
    int64_t jmax = 0;
    for (int n = 0; n < N; ++n) jmax = host_J[n] > jmax ? host_J[n] : jmax;
    a.sb = int((jmax + 3) / 4 * 4);
  }
  const int64_t width = kind == FCS_CONTRACT_ALL ? 1 : host_I[free_mode];
  const bool both = kind == kBoth;
  DeviceGuard g(ctx->device);
  bool hit = false;
  fcs_spec_cache::Entry *ent = spec_cache_get(ctx, fcsT, a.m.Jt, D, log2m, &hit);
  // the long-FFT path places its own spectrum buffer in the workspace; its
  // raw buffer must then come from a separate allocation owned by the context
  const bool big = log2p > kMaxLog2P;
  const size_t sbytes =
      (ent || big) ? 0 : (sizeof(float2) * size_t(D) * size_t(M + 1) + 255) & ~size_t(255);
  const size_t rbytes =
      out_raw ? 0 : (sizeof(float) * size_t(B) * D * size_t(width) + 255) & ~size_t(255);
  const size_t abytes = (both && !out_all_raw) ? sizeof(float) * size_t(B) * D : 0;
  if (big && rbytes + abytes) {
    rc = ensure_raw(ctx, rbytes + abytes);
    if (rc) return rc;
  }
  void *ws = nullptr;
  if (!big && sbytes + rbytes + abytes > 0) {
    rc = ensure_workspace(ctx, sbytes + rbytes + abytes, &ws);
    if (rc) return rc;
  }
  char *rbase = big ? reinterpret_cast<char *>(ctx->raw) : static_cast<char *>(ws) + sbytes;
  a.spec = ent ? ent->spec : static_cast<float2 *>(ws);
  a.raw = out_raw ? out_raw : reinterpret_cast<float *>(rbase);
  a.raw_all = !both ? nullptr
              : out_all_raw ? out_all_raw
                            : reinterpret_cast<float *>(rbase + rbytes);
  if (hit) {
    // the spectrum may have been written on another stream
    rc = check_cuda(ctx, cudaStreamWaitEvent(ctx->stream, ent->ready, 0), "cudaStreamWaitEvent");
    if (rc) return rc;
  }
  rc = FCS_EUNSUPPORTED;
  if (log2p > kMaxLog2P) {
    if (both) {
      // the long-FFT route runs the two contractions one after the other
      // (the second reuses the cached spectra when the cache is on)
      rc = big_contract(ctx, a.m, FCS_CONTRACT_ALL, free_mode, D, fcsT, B, a.vec, h, s,
                        ent ? ent->spec : nullptr, !hit, ent ? ent->ready : nullptr, a.raw_all,
                        log2p);
      if (!rc)
        rc = big_contract(ctx, a.m, FCS_CONTRACT_FREE, free_mode, D, fcsT, B, a.vec, h, s,
                          ent ? ent->spec : nullptr, ent == nullptr, nullptr, a.raw, log2p);
    } else {
      rc = big_contract(ctx, a.m, kind, free_mode, D, fcsT, B, a.vec, h, s,
                        ent ? ent->spec : nullptr, !hit, ent ? ent->ready : nullptr, a.raw,
                        log2p);
    }
  } else {
    FCS_DISPATCH_LOG2M(log2m, rc = launch_contract<L>(ctx, a, a.m.Jt, !hit,
                                                      ent ? ent->ready : nullptr));
  }
  if (rc) {
    if (ent && !hit) ent->stale = true;          // never computed
    return rc;
  }
  if (ent) {
    rc = check_cuda(ctx, cudaEventRecord(ent->used, ctx->stream), "cudaEventRecord");
    if (rc) return rc;
  }
  if (both) {
    rc = launch_median(ctx, D, a.raw_all, B, 1, out_all);
    if (rc) return rc;
  }
  return launch_median(ctx, D, a.raw, B, width, out_median);
}

}  // namespace

extern "C" int fcs_contract(fcs_ctx *ctx, int kind, int free_mode, int N,
                            const int64_t *host_I, const int32_t *host_J, int D,
                            const float *fcsT, int64_t B, const float *const *host_vecs,
                            const int32_t *h, const int8_t *s, int64_t ldh,
                            float *out_median, float *out_raw) {
  if (kind != FCS_CONTRACT_ALL && kind != FCS_CONTRACT_FREE) {
    if (!ctx) return FCS_EINVAL;
    ctx->err.clear();
    return set_error(ctx, FCS_EINVAL, "unknown contraction kind %d", kind);
  }
  return contract_call(ctx, kind, free_mode, N, host_I, host_J, D, fcsT, B, host_vecs, h, s, ldh,
                       out_median, out_raw, nullptr, nullptr);
}

extern "C" int fcs_contract_both(fcs_ctx *ctx, int free_mode, int N, const int64_t *host_I,
                                 const int32_t *host_J, int D, const float *fcsT, int64_t B,
                                 const float *const *host_vecs, const int32_t *h,
                                 const int8_t *s, int64_t ldh, float *out_all, float *out_free,
                                 float *out_all_raw, float *out_free_raw) {
  return contract_call(ctx, kBoth, free_mode, N, host_I, host_J, D, fcsT, B, host_vecs, h, s,
                       ldh, out_free, out_free_raw, out_all, out_all_raw);
}
