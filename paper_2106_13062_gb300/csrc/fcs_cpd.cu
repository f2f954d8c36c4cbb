// fcs_cpd.cu -- CP decompositions from sketches (CP decomposition subsection):
//
// fcs_rtpm: sketched robust tensor power method for a symmetric order-N
//   tensor.  For each of K components: L starting vectors, n_iter power
//   iterations u <- T(I,u,..,u) / ||T(I,u,..,u)|| (eq. T_Ivw, free mode 0),
//   eigenvalues T(u,..,u) (eq. T_uvw), the start with the largest eigenvalue
//   kept; then the sketch is deflated by linearity,
//       FCS(T) <- FCS(T) - lambda FCS(u o .. o u)   (eq. FCS_syn, R = 1).
// fcs_als: sketched CP-ALS for an order-N tensor: per sweep and mode m, the
//   columns T_(m)(..) = [T(.., I (mode m), ..)]_r with the other factors'
//   r-th columns (eq. T_Ivw with distinct vectors per mode), then
//       F_m^T <- G^{-1} M^T,   G = *_{n != m} F_n F_n^T   (Hadamard product),
//   by a Cholesky factorisation, and column normalisation (weights lambda).
//
// Both are host loops over the library's own calls (fcs_contract,
// fcs_sketch_cp) plus small kernels; every intermediate stays on the device
// and the loops never synchronise the host.  The sketch spectra are cached
// for the duration of the call (fcs_contract's cache), so the power
// iterations and sweeps transform each sketch once.
#include <algorithm>
#include <vector>

#include "fcs_internal.cuh"

namespace fcs {
namespace {

constexpr int kMaxRank = 32;

// Scratch for the decompositions, separate from the workspace that the
// calls below use.
int ensure_algo(fcs_ctx *ctx, size_t bytes) {
  return grow_buffer(ctx, &ctx->algo, &ctx->algo_bytes, bytes, "decomposition scratch");
}

__device__ __forceinline__ float block_sum(float v, float *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;
}

// Each row of V [rows][I] scaled to unit norm (one block per row).
__global__ void normalize_rows_kernel(float *V, int64_t I) {
  __shared__ float red[32];
  float *v = V + int64_t(blockIdx.x) * I;
  float ss = 0.f;
  for (int64_t i = threadIdx.x; i < I; i += blockDim.x) ss += v[i] * v[i];
  const float nrm = sqrtf(block_sum(ss, red));
  const float inv = nrm > 0.f ? 1.0f / nrm : 0.f;
  for (int64_t i = threadIdx.x; i < I; i += blockDim.x) v[i] *= inv;
}

// The start with the largest eigenvalue (first one on ties): u <- V[best],
// *lam_out <- lam[best].
__global__ void pick_best_kernel(const float *lam, int L, const float *V, int64_t I, float *u,
                                 float *lam_out) {
  __shared__ int best;
  if (threadIdx.x == 0) {
    int b = 0;
    for (int l = 1; l < L; ++l)
      if (lam[l] > lam[b]) b = l;
    best = b;
    *lam_out = lam[b];
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < I; i += blockDim.x) u[i] = V[int64_t(best) * I + i];
}

__global__ void subtract_kernel(float *S, const float *R, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    S[i] -= R[i];
}

struct AlsArgs {
  int N, m, R;
  int64_t I[kMaxN];
  float *F[kMaxN];       // [R][I_n] each
  float *Mt;             // [R][I_m]: in T_(m) columns (transposed), out the solution
  float *lambda;         // [R]
};

// One CTA: G = *_{n != m} F_n F_n^T, Cholesky G = L L^T, then for every
// column i of M^T the solve G x = M^T[:, i]; row norms give lambda and the
// normalised rows the new F_m.
__global__ void __launch_bounds__(1024) als_update_kernel(AlsArgs a) {
  __shared__ float G[kMaxRank][kMaxRank + 1];
  __shared__ float nrm[kMaxRank];
  const int R = a.R;
  for (int p = threadIdx.x; p < R * R; p += blockDim.x) {
    const int r = p / R, q = p % R;
    float g = 1.f;
    for (int n = 0; n < a.N; ++n) {
      if (n == a.m) continue;
      const float *fr = a.F[n] + int64_t(r) * a.I[n];
      const float *fq = a.F[n] + int64_t(q) * a.I[n];
      float dot = 0.f;
      for (int64_t i = 0; i < a.I[n]; ++i) dot = fmaf(fr[i], fq[i], dot);
      g *= dot;
    }
    G[r][q] = g;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // Cholesky in place (lower triangle); a non-positive pivot is lifted to a
    // tiny multiple of the largest diagonal entry
    float dmax = 0.f;
    for (int r = 0; r < R; ++r) dmax = fmaxf(dmax, G[r][r]);
    for (int j = 0; j < R; ++j) {
      float v = G[j][j];
      for (int k = 0; k < j; ++k) v -= G[j][k] * G[j][k];
      v = v > 1e-12f * dmax ? v : 1e-12f * dmax + 1e-30f;
      const float ljj = sqrtf(v);
      G[j][j] = ljj;
      for (int i = j + 1; i < R; ++i) {
        float w = G[i][j];
        for (int k = 0; k < j; ++k) w -= G[i][k] * G[j][k];
        G[i][j] = w / ljj;
      }
    }
  }
  __syncthreads();
  const int64_t Im = a.I[a.m];
  for (int64_t i = threadIdx.x; i < Im; i += blockDim.x) {
    float x[kMaxRank];
    for (int r = 0; r < R; ++r) x[r] = a.Mt[int64_t(r) * Im + i];
    for (int r = 0; r < R; ++r) {             // L y = b
      float v = x[r];
      for (int k = 0; k < r; ++k) v -= G[r][k] * x[k];
      x[r] = v / G[r][r];
    }
    for (int r = R - 1; r >= 0; --r) {        // L^T x = y
      float v = x[r];
      for (int k = r + 1; k < R; ++k) v -= G[k][r] * x[k];
      x[r] = v / G[r][r];
    }
    for (int r = 0; r < R; ++r) a.Mt[int64_t(r) * Im + i] = x[r];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = warp; r < R; r += blockDim.x >> 5) {
    float ss = 0.f;
    for (int64_t i = lane; i < Im; i += 32) {
      const float v = a.Mt[int64_t(r) * Im + i];
      ss += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) nrm[r] = sqrtf(ss);
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < int64_t(R) * Im; e += blockDim.x) {
    const int r = int(e / Im);
    const float w = nrm[r];
    a.F[a.m][e] = w > 0.f ? a.Mt[e] / w : 0.f;
  }
  if (threadIdx.x < R) a.lambda[threadIdx.x] = nrm[threadIdx.x];
}

// Turns the spectrum cache on for the duration of a call and restores it.
struct CacheScope {
  fcs_ctx *ctx;
  bool prev;
  std::vector<const void *> keys;
  explicit CacheScope(fcs_ctx *c) : ctx(c), prev(c->cache_spectra) { c->cache_spectra = true; }
  ~CacheScope() {
    for (const void *k : keys) fcs_forget(ctx, k);
    ctx->cache_spectra = prev;
  }
};

}  // namespace
}  // namespace fcs

using namespace fcs;

extern "C" int fcs_rtpm(fcs_ctx *ctx, int N, int64_t I, const int32_t *host_J, int D,
                        const float *fcsT, const int32_t *h, const int8_t *s, int64_t ldh,
                        int K, int L, int n_iter, const float *init, float *lambda, float *U) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  if (N < 2 || N > kMaxN) return set_error(ctx, FCS_EINVAL, "N=%d outside [2,%d]", N, kMaxN);
  std::vector<int64_t> Iv(N, I);
  Modes m{};
  int rc = make_modes(ctx, N, Iv.data(), host_J, ldh, &m);
  if (rc) return rc;
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (K < 1 || L < 1 || L > 65535 || n_iter < 0)
    return set_error(ctx, FCS_EINVAL, "need K >= 1, 1 <= L <= 65535, n_iter >= 0");
  if (!fcsT || !h || !s || !init || !lambda || !U)
    return set_error(ctx, FCS_EINVAL, "NULL pointer argument");
  const int64_t Jt = m.Jt;
  const size_t sk = sizeof(float) * size_t(D) * size_t(Jt);
  const size_t vb = sizeof(float) * size_t(L) * size_t(I);
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  DeviceGuard g(ctx->device);
  rc = ensure_algo(ctx, 2 * up(sk) + 2 * up(vb) + up(sizeof(float) * size_t(L)));
  if (rc) return rc;
  char *base = static_cast<char *>(ctx->algo);
  float *S = reinterpret_cast<float *>(base);
  float *R1 = reinterpret_cast<float *>(base + up(sk));
  float *V = reinterpret_cast<float *>(base + 2 * up(sk));
  float *W = reinterpret_cast<float *>(base + 2 * up(sk) + up(vb));
  float *lamL = reinterpret_cast<float *>(base + 2 * up(sk) + 2 * up(vb));
  fcs_forget(ctx, S);
  rc = check_cuda(ctx, cudaMemcpyAsync(S, fcsT, sk, cudaMemcpyDeviceToDevice, ctx->stream),
                  "cudaMemcpyAsync(sketch copy)");
  if (rc) return rc;
  CacheScope cache(ctx);
  cache.keys.push_back(S);
  const int nt = int(std::min<int64_t>(256, (I + 31) / 32 * 32));
  std::vector<const float *> vv(N);
  std::vector<const float *> uu(N);
  std::vector<int64_t> ld1(N, 1);
  for (int k = 0; k < K; ++k) {
    rc = check_cuda(ctx, cudaMemcpyAsync(V, init + size_t(k) * L * I, vb,
                                         cudaMemcpyDeviceToDevice, ctx->stream),
                    "cudaMemcpyAsync(init)");
    if (rc) return rc;
    normalize_rows_kernel<<<L, nt, 0, ctx->stream>>>(V, I);
    rc = check_cuda(ctx, cudaGetLastError(), "normalize_rows_kernel");
    if (rc) return rc;
    for (int it = 0; it < n_iter; ++it) {
      vv[0] = nullptr;
      for (int n = 1; n < N; ++n) vv[n] = V;
      rc = fcs_contract(ctx, FCS_CONTRACT_FREE, 0, N, Iv.data(), host_J, D, S, L, vv.data(), h,
                        s, ldh, W, nullptr);
      if (rc) return rc;
      normalize_rows_kernel<<<L, nt, 0, ctx->stream>>>(W, I);
      rc = check_cuda(ctx, cudaGetLastError(), "normalize_rows_kernel");
      if (rc) return rc;
      std::swap(V, W);
    }
    for (int n = 0; n < N; ++n) vv[n] = V;
    rc = fcs_contract(ctx, FCS_CONTRACT_ALL, 0, N, Iv.data(), host_J, D, S, L, vv.data(), h, s,
                      ldh, lamL, nullptr);
    if (rc) return rc;
    float *uk = U + size_t(k) * I;
    pick_best_kernel<<<1, nt, 0, ctx->stream>>>(lamL, L, V, I, uk, lambda + k);
    rc = check_cuda(ctx, cudaGetLastError(), "pick_best_kernel");
    if (rc) return rc;
    if (k + 1 == K) break;
    // deflation: S <- S - lambda_k FCS(u o .. o u)
    for (int n = 0; n < N; ++n) uu[n] = uk;
    rc = fcs_sketch_cp(ctx, N, Iv.data(), host_J, 1, D, uu.data(), ld1.data(), lambda + k, h, s,
                       ldh, R1);
    if (rc) return rc;
    fcs_forget(ctx, S);
    const int64_t n = int64_t(D) * Jt;
    subtract_kernel<<<unsigned(std::min<int64_t>((n + 255) / 256, 1024)), 256, 0, ctx->stream>>>(
        S, R1, n);
    rc = check_cuda(ctx, cudaGetLastError(), "subtract_kernel");
    if (rc) return rc;
  }
  return FCS_OK;
}

extern "C" int fcs_als(fcs_ctx *ctx, int N, const int64_t *host_I, const int32_t *host_J, int D,
                       const float *fcsT, const int32_t *h, const int8_t *s, int64_t ldh, int R,
                       int n_iter, float *const *host_F, float *lambda) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  if (N < 2 || N > kMaxN) return set_error(ctx, FCS_EINVAL, "N=%d outside [2,%d]", N, kMaxN);
  Modes m{};
  int rc = make_modes(ctx, N, host_I, host_J, ldh, &m);
  if (rc) return rc;
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (R < 1 || R > kMaxRank)
    return set_error(ctx, FCS_EINVAL, "R=%d outside [1,%d]", R, kMaxRank);
  if (n_iter < 0) return set_error(ctx, FCS_EINVAL, "n_iter must be >= 0");
  if (!fcsT || !h || !s || !host_F || !lambda)
    return set_error(ctx, FCS_EINVAL, "NULL pointer argument");
  int64_t imax = 0;
  for (int n = 0; n < N; ++n) {
    if (!host_F[n]) return set_error(ctx, FCS_EINVAL, "factor %d is NULL", n);
    imax = std::max<int64_t>(imax, host_I[n]);
  }
  DeviceGuard g(ctx->device);
  rc = ensure_algo(ctx, sizeof(float) * size_t(R) * size_t(imax));
  if (rc) return rc;
  float *Mt = static_cast<float *>(ctx->algo);
  CacheScope cache(ctx);
  if (!cache.prev) cache.keys.push_back(fcsT);
  std::vector<const float *> vv(N);
  AlsArgs a{};
  a.N = N;
  a.R = R;
  for (int n = 0; n < N; ++n) {
    a.I[n] = host_I[n];
    a.F[n] = host_F[n];
  }
  a.Mt = Mt;
  a.lambda = lambda;
  for (int it = 0; it < n_iter; ++it) {
    for (int mm = 0; mm < N; ++mm) {
      for (int n = 0; n < N; ++n) vv[n] = n == mm ? nullptr : host_F[n];
      rc = fcs_contract(ctx, FCS_CONTRACT_FREE, mm, N, host_I, host_J, D, fcsT, R, vv.data(), h,
                        s, ldh, Mt, nullptr);
      if (rc) return rc;
      a.m = mm;
      als_update_kernel<<<1, 1024, 0, ctx->stream>>>(a);
      rc = check_cuda(ctx, cudaGetLastError(), "als_update_kernel");
      if (rc) return rc;
    }
  }
  return FCS_OK;
}
