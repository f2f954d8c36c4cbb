// fcs_cp.cu -- fcs_sketch_cp: FCS of a CP tensor by eq. (FCS_syn):
//   FCS(T) = sum_r lambda_r IFFT( prod_n FFT_P( CS_n(U_n(:, r)) ) ),
// with P the smallest power of two >= Jt (any P >= Jt gives the exact linear
// convolution, so out = the first Jt samples).
//
// Two kernels.  (1) A transpose writes the factor columns contiguously
// (lambda folded into mode 1) so every column load is coalesced.  (2) The
// fused sketch kernel: CTA (g, d) owns sketch d and a contiguous group of
// ranks.  For each rank and mode it scatters the signed factor column into a
// compact shared-memory buffer of max_n J_n reals (the Count Sketch of
// Def. 1; the zero padding up to P is never stored), runs the block real FFT
// of fcs_fft.cuh whose last pass leaves the half spectrum in registers, and
// multiplies it into the per-thread mode product; after the last mode the
// product is added into a shared-memory rank accumulator.  The rank sum thus
// stays in the frequency domain (linearity moves the paper's sum of inverse
// transforms inside one inverse transform).  Each CTA adds its partial
// spectrum into a global accumulator with float2 atomics; the last CTA to
// finish for sketch d (ticket counter) runs the one inverse real FFT and
// writes FCS_d.  The next column's factor values and hashes are prefetched
// into registers while the current column is transformed.
#include <cstdarg>
#include <mutex>

#include "fcs_fft.cuh"

namespace fcs {
namespace {

struct CpArgs {
  Modes m;
  int D;
  int64_t R;
  int64_t ranks_per_cta;
  const float *UT;       // [sum_n R*I_n]: mode n column r at ut_off[n] + r*I_n
  int64_t ut_off[kMaxN];
  const int32_t *h;
  const int8_t *s;
  float2 *G;             // [D][M+1] spectrum accumulator, zeroed per call
  unsigned *counter;     // [D] tickets, zero at launch, reset by the last CTA
  float *out;            // [D][Jt]
  int sb;                // scatter buffer length (floats): max J_n rounded up to 4
};

// All modes in one launch: mode n = blockIdx.z.
struct TransposeArgs {
  const float *U[kMaxN];
  int64_t I[kMaxN], ld[kMaxN], ut_off[kMaxN];
  int64_t R;
  const float *lambda;
  float *UT;
};

// UT[n][r][i] = U_n[i*ld + r] (times lambda_r for n = 0).
__global__ void transpose_all_kernel(TransposeArgs t) {
  __shared__ float tile[32][33];
  const int n = blockIdx.z;
  const int64_t I = t.I[n], R = t.R, ld = t.ld[n];
  const float *U = t.U[n];
  const float *lambda = n == 0 ? t.lambda : nullptr;
  float *UT = t.UT + t.ut_off[n];
  const int64_t i0 = blockIdx.x * 32ll, r0 = blockIdx.y * 32ll;
  if (i0 >= I) return;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = i0 + k, r = r0 + threadIdx.x;
    if (i < I && r < R) tile[k][threadIdx.x] = U[i * ld + r];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k, i = i0 + threadIdx.x;
    if (i < I && r < R) {
      const float lam = lambda ? __ldg(lambda + r) : 1.f;
      UT[r * I + i] = tile[threadIdx.x][k] * lam;
    }
  }
}

// UT[n][r][i] = U_n[i*ld + r] (times lambda_r for n = 0).
__global__ void transpose_factors_kernel(const float *__restrict__ U, int64_t I, int64_t R,
                                         int64_t ld, const float *__restrict__ lambda,
                                         float *__restrict__ UT) {
  __shared__ float tile[32][33];
  const int64_t i0 = blockIdx.x * 32ll, r0 = blockIdx.y * 32ll;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = i0 + k, r = r0 + threadIdx.x;
    if (i < I && r < R) tile[k][threadIdx.x] = U[i * ld + r];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k, i = i0 + threadIdx.x;
    if (i < I && r < R) {
      const float lam = lambda ? __ldg(lambda + r) : 1.f;
      UT[r * I + i] = tile[threadIdx.x][k] * lam;
    }
  }
}

// Shared-memory layout of cp_kernel; every region starts on a 16-byte
// boundary (the scatter buffer is cleared with float4 stores).
template <int LOG2M, int NT>
struct CpSmem {
  static constexpr size_t up16(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t kB = 0;
  static constexpr size_t kAcc = up16(kB + sizeof(float2) * padded_len(1 << LOG2M));
  static constexpr size_t kTw =
      up16(kAcc + sizeof(float2) * LastPass<LOG2M, NT>::NV * NT);
  static constexpr size_t kA = up16(kTw + sizeof(float2) * plan_twlen(LOG2M));
  static size_t bytes(int sb) { return kA + sizeof(float) * size_t(sb); }
};

template <int LOG2M, int NT, int CPT>
__global__ void __launch_bounds__(NT) cp_kernel(CpArgs a, const float2 *__restrict__ tw) {
  using LPs = LastPass<LOG2M, NT>;
  constexpr int M = 1 << LOG2M;
  constexpr int HALF = M / 2;
  constexpr int RL = LPs::RL, EPS = LPs::EPS, NV = LPs::NV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using Lay = CpSmem<LOG2M, NT>;
  float2 *B = reinterpret_cast<float2 *>(smem_raw + Lay::kB);      // padded_len(M)
  float2 *accS = reinterpret_cast<float2 *>(smem_raw + Lay::kAcc); // NV * NT
  float2 *tws = reinterpret_cast<float2 *>(smem_raw + Lay::kTw);   // plan_twlen
  float *A = reinterpret_cast<float *>(smem_raw + Lay::kA);        // a.sb floats
  __shared__ int is_last;
  const int tid = threadIdx.x;
  const int d = blockIdx.y;
  const int N = a.m.N;
  const int64_t r0 = blockIdx.x * a.ranks_per_cta;
  const int64_t r1 = min(a.R, r0 + a.ranks_per_cta);
  const int sb = a.sb;

  fill_twiddles<LOG2M, NT>(tws, tw);
  for (int e = tid; e < sb / 4; e += NT) reinterpret_cast<float4 *>(A)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int v = 0; v < NV; ++v) accS[v * NT + tid] = make_float2(0.f, 0.f);

  // prefetched column: signed factor values and hash bins
  float pv[CPT];
  int ph[CPT];
  auto fetch = [&](int64_t r, int n) {
    const int64_t In = a.m.I[n];
    const float *col = a.UT + a.ut_off[n] + r * In;
    const int32_t *hn = a.h + d * a.m.ldh + a.m.off[n];
    const int8_t *sn = a.s + d * a.m.ldh + a.m.off[n];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int64_t i = tid + int64_t(c) * NT;
      ph[c] = -1;
      pv[c] = 0.f;
      if (i < In) {
        const float v = __ldg(col + i);
        pv[c] = __ldg(sn + i) < 0 ? -v : v;
        ph[c] = __ldg(hn + i);
      }
    }
  };
  fetch(r0, 0);
  __syncthreads();

  float2 X[EPS][2][RL], p[EPS][2][RL];
  for (int64_t r = r0; r < r1; ++r) {
    for (int n = 0; n < N; ++n) {
#pragma unroll
      for (int c = 0; c < CPT; ++c)
        if (unsigned(ph[c]) < unsigned(sb)) atomicAdd(A + ph[c], pv[c]);
      if (a.m.I[n] > int64_t(CPT) * NT) {
        // entries beyond the prefetched chunk: load and scatter directly
        const int64_t In = a.m.I[n];
        const float *col = a.UT + a.ut_off[n] + r * In;
        const int32_t *hn = a.h + d * a.m.ldh + a.m.off[n];
        const int8_t *sn = a.s + d * a.m.ldh + a.m.off[n];
        for (int64_t i = int64_t(CPT) * NT + tid; i < In; i += NT) {
          const int hb = __ldg(hn + i);
          const float v = __ldg(col + i);
          if (unsigned(hb) < unsigned(sb)) atomicAdd(A + hb, __ldg(sn + i) < 0 ? -v : v);
        }
      }
      // prefetch the next column while this one is transformed
      if (n + 1 < N)
        fetch(r, n + 1);
      else if (r + 1 < r1)
        fetch(r + 1, 0);
      __syncthreads();
      fft_first_pass<LOG2M, NT>(A, sb, B);
      __syncthreads();
      for (int e = tid; e < sb / 4; e += NT)
        reinterpret_cast<float4 *>(A)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
      fft_middle_passes<LOG2M, NT, 1>(B, tws);
      fft_last_pass_unpack<LOG2M, NT>(B, tw, X);
#pragma unroll
      for (int e = 0; e < EPS; ++e)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int q = 0; q < RL; ++q) {
            if (n == 0) {
              p[e][b][q] = X[e][b][q];
            } else {
              const bool packed = (b == 0 && q == 0 && tid + e * NT == 0);
              p[e][b][q] = slot_mul(p[e][b][q], X[e][b][q], packed);
            }
          }
    }
#pragma unroll
    for (int e = 0; e < EPS; ++e)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int q = 0; q < RL; ++q) {
          float2 &acc = accS[((e * 2 + b) * RL + q) * NT + tid];
          acc = cadd(acc, p[e][b][q]);
        }
  }

  // publish the partial spectrum
  float2 *Gd = a.G + d * int64_t(M + 1);
#pragma unroll
  for (int e = 0; e < EPS; ++e) {
    if (LPs::SLOTS % NT != 0 && tid + e * NT >= LPs::SLOTS) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int q = 0; q < RL; ++q) {
        const float2 v = accS[((e * 2 + b) * RL + q) * NT + tid];
        const int k = last_pass_index<LOG2M, NT>(e, b, q);
        if (k == 0) {
          atomicAdd(&Gd[0].x, v.x);
          atomicAdd(&Gd[M].x, v.y);
        } else {
          atomicAdd(&Gd[k], v);
        }
      }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = (atomicAdd(&a.counter[d], 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  // last CTA for sketch d: one inverse real FFT of the summed spectrum
  for (int q = tid; q < HALF; q += NT) {
    float2 Av, Bv;
    if (q == 0) {
      Av = make_float2(__ldcg(&Gd[0].x), __ldcg(&Gd[M].x));
      Bv = __ldcg(&Gd[HALF]);
    } else {
      Av = __ldcg(&Gd[q]);
      Bv = __ldcg(&Gd[M - q]);
    }
    pack_pair_conj<LOG2M>(B, q, Av, Bv, tw);
  }
  __syncthreads();
  block_fft<LOG2M, NT>(B, tw);
  const float sc = 1.0f / float(M);
  float *od = a.out + d * a.m.Jt;
  float *Br = reinterpret_cast<float *>(B);
  for (int64_t j = tid; j < a.m.Jt; j += NT) {
    const float v = Br[real_off(int(j))];
    od[j] = (j & 1) ? -v * sc : v * sc;
  }
  if (tid == 0) a.counter[d] = 0u;
}

template <int LOG2M>
int launch_cp(fcs_ctx *ctx, CpArgs &a, int64_t groups, int64_t Imax) {
  constexpr int NT = fft_threads(LOG2M);
  const size_t smem = CpSmem<LOG2M, NT>::bytes(a.sb);
  const int cpt = int((Imax + NT - 1) / NT);
  auto go = [&](auto kern) -> int {
    if (smem > 48 * 1024) {
      cudaError_t e =
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(cp)");
    }
    kern<<<dim3(unsigned(groups), unsigned(a.D)), NT, smem, ctx->stream>>>(a, ctx->twiddle);
    return check_cuda(ctx, cudaGetLastError(), "cp_kernel");
  };
  if (cpt <= 1) return go(cp_kernel<LOG2M, NT, 1>);
  if (cpt <= 2) return go(cp_kernel<LOG2M, NT, 2>);
  return go(cp_kernel<LOG2M, NT, 4>);       // larger modes add a direct tail loop
}

}  // namespace
}  // namespace fcs

using namespace fcs;

extern "C" int fcs_sketch_cp(fcs_ctx *ctx, int N, const int64_t *host_I,
                             const int32_t *host_J, int64_t R, int D,
                             const float *const *host_U, const int64_t *host_ldU,
                             const float *lambda, const int32_t *h, const int8_t *s,
                             int64_t ldh, float *out) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  CpArgs a{};
  int rc = make_modes(ctx, N, host_I, host_J, ldh, &a.m);
  if (rc) return rc;
  if (D < 1 || D > kMaxD) return set_error(ctx, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (R < 1) return set_error(ctx, FCS_EINVAL, "R=%lld must be >= 1", (long long)R);
  if (!host_U || !host_ldU || !h || !s || !out)
    return set_error(ctx, FCS_EINVAL, "NULL pointer argument");
  for (int n = 0; n < N; ++n) {
    if (!host_U[n]) return set_error(ctx, FCS_EINVAL, "U[%d] is NULL", n);
    if (host_ldU[n] < R)
      return set_error(ctx, FCS_EINVAL, "ldU[%d]=%lld < R", n, (long long)host_ldU[n]);
  }
  const int log2p = ilog2_ceil(a.m.Jt) < kMinLog2P ? kMinLog2P : ilog2_ceil(a.m.Jt);
  if (log2p > kMaxLog2P)
    return set_error(ctx, FCS_EUNSUPPORTED, "Jt=%lld needs FFT length > %d",
                     (long long)a.m.Jt, 1 << kMaxLog2P);
  const int log2m = log2p - 1;
  const int M = 1 << log2m;
  a.D = D;
  a.R = R;
  a.h = h;
  a.s = s;
  a.out = out;
  // rank groups: about one CTA per SM over all sketches
  int64_t groups = (int64_t(ctx->sm_count) + D - 1) / D;
  if (groups < 1) groups = 1;
  if (groups > R) groups = R;
  a.ranks_per_cta = (R + groups - 1) / groups;
  groups = (R + a.ranks_per_cta - 1) / a.ranks_per_cta;

  int64_t Imax = 0, Jmax = 0, utlen = 0;
  for (int n = 0; n < N; ++n) {
    a.ut_off[n] = utlen;
    utlen += R * host_I[n];
    if (host_I[n] > Imax) Imax = host_I[n];
    if (host_J[n] > Jmax) Jmax = host_J[n];
  }
  a.sb = int((Jmax + 3) / 4 * 4);
  const size_t gbytes = (sizeof(float2) * size_t(D) * size_t(M + 1) + 255) & ~size_t(255);
  const size_t cbytes = 256;
  void *ws = nullptr;
  rc = ensure_workspace(ctx, gbytes + cbytes + sizeof(float) * size_t(utlen), &ws);
  if (rc) return rc;
  a.G = static_cast<float2 *>(ws);
  a.counter = reinterpret_cast<unsigned *>(static_cast<char *>(ws) + gbytes);
  float *UT = reinterpret_cast<float *>(static_cast<char *>(ws) + gbytes + cbytes);
  a.UT = UT;
  DeviceGuard g(ctx->device);
  rc = check_cuda(ctx, cudaMemsetAsync(ws, 0, gbytes + cbytes, ctx->stream),
                  "cudaMemsetAsync(cp workspace)");
  if (rc) return rc;
  {
    TransposeArgs t{};
    for (int n = 0; n < N; ++n) {
      t.U[n] = host_U[n];
      t.I[n] = host_I[n];
      t.ld[n] = host_ldU[n];
      t.ut_off[n] = a.ut_off[n];
    }
    t.R = R;
    t.lambda = lambda;
    t.UT = UT;
    dim3 grid(unsigned((Imax + 31) / 32), unsigned((R + 31) / 32), unsigned(N));
    if (grid.y > 65535 || grid.x > 0x7fffffffu)
      return set_error(ctx, FCS_EUNSUPPORTED, "factor matrices too large");
    transpose_all_kernel<<<grid, dim3(32, 8), 0, ctx->stream>>>(t);
    rc = check_cuda(ctx, cudaGetLastError(), "transpose_all_kernel");
    if (rc) return rc;
  }
  rc = FCS_EUNSUPPORTED;
  FCS_DISPATCH_LOG2M(log2m, rc = launch_cp<L>(ctx, a, groups, Imax));
  return rc;
}

// ---------------------------------------------------------------------------
// fcs_sketch_cp_noalloc: the CP-route sketch for callers that cannot allocate
// device memory.  It runs the same two kernels as fcs_sketch_cp, but its
// scratch (spectrum accumulator, tickets, transposed factor columns) and its
// twiddle table live in file-scope __device__ arrays of fixed size instead of
// a context workspace, so the call makes no cudaMalloc / cudaFree and needs
// no fcs_ctx.
namespace fcs {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;   // 4 MiB
constexpr int kNoAllocMaxDevices = 64;

// One copy of each array exists on every GPU that loads the library and is
// held until the process exits.  In host code these names are host-side
// stand-ins, not device addresses: kernels get the addresses that
// cudaGetSymbolAddress returns at set-up.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
__device__ __align__(256) float2 g_noalloc_twiddle[kTwN];

struct NoAllocDevice {
  bool ready;
  unsigned char *scratch;
  float2 *twiddle;
  int sm_count;
};
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// tw[k] = exp(-2 pi i k / kTwN) in FP64, rounded to FP32.
__global__ void noalloc_twiddle_kernel(float2 *tw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < kTwN) {
    double sn, cs;
    sincospi(2.0 * double(k) / double(kTwN), &sn, &cs);
    tw[k] = make_float2(float(cs), float(-sn));
  }
}

int noalloc_fail(char *err, size_t n, int code, const char *fmt, ...) {
  if (err && n) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, n, fmt, ap);
    va_end(ap);
  }
  return code;
}

// First call on a device (with that device current): look up the device
// addresses of the static arrays and fill the twiddle table (the stream is
// synchronised once so any later stream sees the table).
int noalloc_setup(int dev, cudaStream_t st, NoAllocDevice **out, char *err, size_t n) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocDevice &s = g_noalloc_dev[dev];
  if (!s.ready) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "cudaGetSymbolAddress(scratch): %s",
                          cudaGetErrorString(e));
    s.scratch = static_cast<unsigned char *>(p);
    e = cudaGetSymbolAddress(&p, g_noalloc_twiddle);
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "cudaGetSymbolAddress(twiddle): %s",
                          cudaGetErrorString(e));
    s.twiddle = static_cast<float2 *>(p);
    e = cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
    noalloc_twiddle_kernel<<<kTwN / 256, 256, 0, st>>>(s.twiddle);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "twiddle set-up: %s", cudaGetErrorString(e));
    s.ready = true;
  }
  *out = &s;
  return FCS_OK;
}

template <int LOG2M>
int noalloc_launch_cp(CpArgs &a, int64_t groups, int64_t Imax, const float2 *tw,
                      cudaStream_t st, char *err, size_t n) {
  constexpr int NT = fft_threads(LOG2M);
  const size_t smem = CpSmem<LOG2M, NT>::bytes(a.sb);
  const int cpt = int((Imax + NT - 1) / NT);
  auto go = [&](auto kern) -> int {
    if (smem > 48 * 1024) {
      cudaError_t e =
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess)
        return noalloc_fail(err, n, FCS_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    }
    kern<<<dim3(unsigned(groups), unsigned(a.D)), NT, smem, st>>>(a, tw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "cp_kernel: %s", cudaGetErrorString(e));
    return FCS_OK;
  };
  if (cpt <= 1) return go(cp_kernel<LOG2M, NT, 1>);
  if (cpt <= 2) return go(cp_kernel<LOG2M, NT, 2>);
  return go(cp_kernel<LOG2M, NT, 4>);
}

}  // namespace
}  // namespace fcs

extern "C" int fcs_sketch_cp_noalloc(void *stream, int N, const int64_t *host_I,
                                     const int32_t *host_J, int64_t R, int D,
                                     const float *const *host_U, const int64_t *host_ldU,
                                     const float *lambda, const int32_t *h, const int8_t *s,
                                     int64_t ldh, float *out, char *err, size_t err_len) {
  if (err && err_len) err[0] = '\0';
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CpArgs a{};
  if (make_modes(nullptr, N, host_I, host_J, ldh, &a.m) != FCS_OK)
    return noalloc_fail(err, err_len, FCS_EINVAL,
                        "invalid N, I_n, J_n or ldh (1 <= N <= %d, I_n >= 1, J_n >= 1)", kMaxN);
  if (D < 1 || D > kMaxD)
    return noalloc_fail(err, err_len, FCS_EINVAL, "D=%d outside [1,%d]", D, kMaxD);
  if (R < 1) return noalloc_fail(err, err_len, FCS_EINVAL, "R=%lld must be >= 1", (long long)R);
  if (!host_U || !host_ldU || !h || !s || !out)
    return noalloc_fail(err, err_len, FCS_EINVAL, "NULL pointer argument");
  for (int n = 0; n < N; ++n) {
    if (!host_U[n]) return noalloc_fail(err, err_len, FCS_EINVAL, "U[%d] is NULL", n);
    if (host_ldU[n] < R)
      return noalloc_fail(err, err_len, FCS_EINVAL, "ldU[%d]=%lld < R", n,
                          (long long)host_ldU[n]);
  }
  const int log2p = ilog2_ceil(a.m.Jt) < kMinLog2P ? kMinLog2P : ilog2_ceil(a.m.Jt);
  if (log2p > kMaxLog2P)
    return noalloc_fail(err, err_len, FCS_EUNSUPPORTED, "Jt=%lld needs FFT length > %d",
                        (long long)a.m.Jt, 1 << kMaxLog2P);
  const int log2m = log2p - 1;
  const int M = 1 << log2m;
  int64_t Imax = 0, Jmax = 0, utlen = 0;
  for (int n = 0; n < N; ++n) {
    a.ut_off[n] = utlen;
    utlen += R * host_I[n];
    if (host_I[n] > Imax) Imax = host_I[n];
    if (host_J[n] > Jmax) Jmax = host_J[n];
  }
  const size_t gbytes = (sizeof(float2) * size_t(D) * size_t(M + 1) + 255) & ~size_t(255);
  const size_t cbytes = 256;
  const size_t need = gbytes + cbytes + sizeof(float) * size_t(utlen);
  if (need > kNoAllocScratchBytes)
    return noalloc_fail(err, err_len, FCS_ENOMEM_BUDGET,
                        "problem needs %zu bytes of scratch; the static scratch array holds "
                        "%zu bytes (D*(P/2+1)*8 + R*sum(I_n)*4 must fit)",
                        need, kNoAllocScratchBytes);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return noalloc_fail(err, err_len, FCS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return noalloc_fail(err, err_len, FCS_EUNSUPPORTED, "device %d beyond %d", dev,
                        kNoAllocMaxDevices);
  NoAllocDevice *sd = nullptr;
  int rc = noalloc_setup(dev, st, &sd, err, err_len);
  if (rc) return rc;

  a.D = D;
  a.R = R;
  a.h = h;
  a.s = s;
  a.out = out;
  a.sb = int((Jmax + 3) / 4 * 4);
  int64_t groups = (int64_t(sd->sm_count) + D - 1) / D;
  if (groups < 1) groups = 1;
  if (groups > R) groups = R;
  a.ranks_per_cta = (R + groups - 1) / groups;
  groups = (R + a.ranks_per_cta - 1) / a.ranks_per_cta;
  a.G = reinterpret_cast<float2 *>(sd->scratch);
  a.counter = reinterpret_cast<unsigned *>(sd->scratch + gbytes);
  float *UT = reinterpret_cast<float *>(sd->scratch + gbytes + cbytes);
  a.UT = UT;
  // the accumulator and tickets must start at zero; the array keeps the
  // previous call's contents otherwise
  e = cudaMemsetAsync(sd->scratch, 0, gbytes + cbytes, st);
  if (e != cudaSuccess)
    return noalloc_fail(err, err_len, FCS_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  for (int n = 0; n < N; ++n) {
    dim3 grid(unsigned((host_I[n] + 31) / 32), unsigned((R + 31) / 32));
    if (grid.y > 65535) return noalloc_fail(err, err_len, FCS_EUNSUPPORTED, "rank too large");
    transpose_factors_kernel<<<grid, dim3(32, 8), 0, st>>>(
        host_U[n], host_I[n], R, host_ldU[n], n == 0 ? lambda : nullptr, UT + a.ut_off[n]);
    e = cudaGetLastError();
    if (e != cudaSuccess)
      return noalloc_fail(err, err_len, FCS_ECUDA, "transpose: %s", cudaGetErrorString(e));
  }
  rc = FCS_EUNSUPPORTED;
  FCS_DISPATCH_LOG2M(log2m, rc = noalloc_launch_cp<L>(a, groups, Imax, sd->twiddle, st, err,
                                                      err_len));
  return rc;
}
