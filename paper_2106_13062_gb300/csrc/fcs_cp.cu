// fcs_cp.cu -- fcs_sketch_cp: FCS of a CP tensor by eq. (FCS_syn):
//   FCS(T) = sum_r lambda_r IFFT( prod_n FFT_P( CS_n(U_n(:, r)) ) ),
// with P the smallest power of two >= Jt (any P >= Jt gives the exact linear
// convolution, so out = the first Jt samples).
//
// Two kernels.  (1) prep_kernel writes the factor columns contiguously
// (lambda folded into mode 1) so every column load is coalesced, clears
// the spectrum accumulator and, for fcs_sketch_cp_seeded, writes the hash
// tables of a seed (the same entries as fcs_make_hashes).  The sketch kernel
// is its programmatic dependent: placed while prep runs, it waits for the
// prep grid at its first instruction.  (2) The fused sketch kernel: CTA (g, d) owns
// sketch d and a contiguous group of ranks and runs cp_run (P <= 8192) or
// cp13_run (P = 16384) of fcs_cp_run.cuh: count sketch, block real FFT, mode
// product and rank sum in the frequency domain (linearity moves the paper's
// sum of inverse transforms inside one inverse transform), partial spectrum
// into a global accumulator, and the one inverse FFT by the CTA that
// completes sketch d.  Longer transforms go to the two-pass route of
// fcs_big.cu.
#include <algorithm>
#include <cstdarg>
#include <mutex>

#include "fcs_cp_run.cuh"
#include "fcs_hash.cuh"

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
  float2 *G;             // [D][M+2] spectrum accumulator (bins 0..M), zeroed per call
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

// cp_run / cp13_run's accessors over CpArgs (fcs_cp_run.cuh).
struct CpView {
  const CpArgs &a;
  int sb;
  // inputs written by the prep launch, which may still run when the sketch
  // kernel (its programmatic dependent) starts: ordinary cached loads (after
  // the grid wait), not the read-only path, whose data must not change
  // during the kernel
  template <class T>
  __device__ __forceinline__ T ld(const T *p) const {
    return __ldca(p);
  }
  __device__ __forceinline__ int modes() const { return a.m.N; }
  __device__ __forceinline__ int64_t dim(int n) const { return a.m.I[n]; }
  __device__ __forceinline__ const float *column(int n, int64_t r) const {
    return a.UT + a.ut_off[n] + r * a.m.I[n];
  }
  __device__ __forceinline__ const int32_t *hashes(int d, int n) const {
    return a.h + d * a.m.ldh + a.m.off[n];
  }
  __device__ __forceinline__ const int8_t *signs(int d, int n) const {
    return a.s + d * a.m.ldh + a.m.off[n];
  }
  __device__ __forceinline__ int64_t length() const { return a.m.Jt; }
  __device__ __forceinline__ float *sketch(int d) const { return a.out + d * a.m.Jt; }
  __device__ __forceinline__ float2 *spectrum() const { return a.G; }
  __device__ __forceinline__ unsigned *ticket(int d) const { return a.counter + d; }
};

// The sketch kernels of fcs_sketch_cp are launched as programmatic dependents
// of the prep launch, so their CTAs are placed while prep runs.  Every one of
// them waits for the prep grid to complete (and its writes to be visible:
// transposed factors, cleared accumulator and tickets, hash tables) before
// anything else; launched the ordinary way the wait returns at once.
__device__ __forceinline__ void wait_for_prep() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// CTA (g, d): ranks [g * ranks_per_cta, ...) of sketch d.
template <int LOG2M, int NT, int CPT>
__global__ void __launch_bounds__(NT) cp_kernel(CpArgs a, const float2 *__restrict__ tw) {
  wait_for_prep();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int is_last;
  const int64_t r0 = blockIdx.x * a.ranks_per_cta;
  const int64_t r1 = min(a.R, r0 + a.ranks_per_cta);
  const CpView view{a, a.sb};
  cp_run<LOG2M, NT, CPT>(view, blockIdx.y, r0, r1, gridDim.x, smem_raw, tw, &is_last);
}

// The same for P = 16384 on the warp-DIT engine.  RMAX = number of 32-entry
// blocks per scatter-buffer row (ra <= 32 RMAX).
template <int CPT, int RMAX>
__global__ void __launch_bounds__(wdit::kNT) cp13_kernel(CpArgs a, const float2 *__restrict__ tw) {
  wait_for_prep();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int is_last;
  const int64_t r0 = blockIdx.x * a.ranks_per_cta;
  const int64_t r1 = min(a.R, r0 + a.ranks_per_cta);
  const CpView view{a, a.sb};
  cp13_run<CPT, RMAX>(view, blockIdx.y, r0, r1, gridDim.x, smem_raw, tw, &is_last);
}

// The same for P = 8192 on the warp-DIT engine (256 threads, two CTAs per
// SM).  RMAX = number of 32-entry blocks per scatter-buffer row.
template <int CPT, int RMAX>
__global__ void __launch_bounds__(wdit::w12::kNT, 2) cp12_kernel(CpArgs a,
                                                                 const float2 *__restrict__ tw) {
  wait_for_prep();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int is_last;
  const int64_t r0 = blockIdx.x * a.ranks_per_cta;
  const int64_t r1 = min(a.R, r0 + a.ranks_per_cta);
  const CpView view{a, a.sb};
  cp12_run<CPT, RMAX>(view, blockIdx.y, r0, r1, gridDim.x, smem_raw, tw, &is_last);
}

// prep_kernel: in one launch, the factor transpose in 32 x 32 tiles,
// UT[n][r][i] = U_n[i*ld + r] (times lambda_r for n = 0), and the clearing
// of the spectrum accumulator and tickets.  256 threads per block.
struct PrepArgs {
  TransposeArgs t;
  int64_t tiles_x, tiles_y, ntile;     // transpose tiles per mode and in total
  float4 *zero;
  int64_t zero_n4;
  int zero_blocks;
  // hash tables from a seed (hash_blocks = 0: none): D x hash_per_d blocks
  HashArgs hs;
  int32_t *h;
  int8_t *s;
  int64_t hash_per_d, hash_blocks;
};

__global__ void __launch_bounds__(256) prep_kernel(PrepArgs a) {
  // the sketch kernel may be placed now; it waits for this grid to complete
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int64_t b = blockIdx.x;
  const int tid = threadIdx.x;
  if (b < a.ntile) {
    __shared__ float tile[32][33];
    const int64_t per = a.tiles_x * a.tiles_y;
    const int n = int(b / per);
    const int64_t rem = b % per;
    const int64_t bx = rem % a.tiles_x, by = rem / a.tiles_x;
    const int64_t I = a.t.I[n], R = a.t.R, ld = a.t.ld[n];
    const float *U = a.t.U[n];
    const float *lambda = n == 0 ? a.t.lambda : nullptr;
    float *UT = a.t.UT + a.t.ut_off[n];
    const int64_t i0 = bx * 32, rr0 = by * 32;
    if (i0 >= I) return;
    const int tx = tid & 31, ty = tid >> 5;
    for (int k = ty; k < 32; k += 8) {
      const int64_t i = i0 + k, r = rr0 + tx;
      if (i < I && r < R) tile[k][tx] = U[i * ld + r];
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
      const int64_t r = rr0 + k, i = i0 + tx;
      if (i < I && r < R) {
        const float lam = lambda ? __ldg(lambda + r) : 1.f;
        UT[r * I + i] = tile[tx][k] * lam;
      }
    }
    return;
  }
  const int64_t zb = b - a.ntile;
  if (zb < a.zero_blocks) {
    for (int64_t e = zb * 256 + tid; e < a.zero_n4; e += int64_t(a.zero_blocks) * 256)
      a.zero[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const int64_t hb = zb - a.zero_blocks;           // < hash_blocks
  const int d = int(hb / a.hash_per_d);
  const int64_t e = (hb - d * a.hash_per_d) * 256 + tid;
  if (e < a.hs.total) hash_entry(a.hs, d, e, a.h, a.s);
}

// Kernel for the given prefetch depth and scatter-buffer height.
template <int CPT>
const void *cp13_pick_rmax(int ra) {
  if (ra <= 128) return reinterpret_cast<const void *>(cp13_kernel<CPT, 4>);
  if (ra <= 256) return reinterpret_cast<const void *>(cp13_kernel<CPT, 8>);
  return reinterpret_cast<const void *>(cp13_kernel<CPT, 16>);
}
const void *cp13_pick(int64_t Imax, int sb) {
  const int ra = (sb + 31) >> 5;
  const int cpt = int((Imax + wdit::kNT - 1) / wdit::kNT);
  if (cpt <= 1) return cp13_pick_rmax<1>(ra);
  if (cpt <= 2) return cp13_pick_rmax<2>(ra);
  return cp13_pick_rmax<4>(ra);
}

// Launch a sketch kernel as a programmatic dependent of the prep launch
// before it on the context's stream.
cudaError_t launch_after_prep(fcs_ctx *ctx, const void *kern, dim3 grid, dim3 block, size_t smem,
                              void **args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, kern, args);
}

int launch_cp13(fcs_ctx *ctx, CpArgs &a, int64_t groups, int64_t Imax) {
  const size_t smem = Cp13Smem::bytes((a.sb + 31) >> 5);
  const void *kern = cp13_pick(Imax, a.sb);
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(cp13)");
  const float2 *twp = ctx->twiddle;
  void *args[] = {&a, &twp};
  e = launch_after_prep(ctx, kern, dim3(unsigned(groups), unsigned(a.D)), dim3(wdit::kNT), smem,
                        args);
  return check_cuda(ctx, e, "cp13_kernel");
}

template <int CPT>
const void *cp12_pick_rmax(int ra) {
  if (ra <= 128) return reinterpret_cast<const void *>(cp12_kernel<CPT, 4>);
  if (ra <= 256) return reinterpret_cast<const void *>(cp12_kernel<CPT, 8>);
  return reinterpret_cast<const void *>(cp12_kernel<CPT, 16>);
}

int launch_cp12(fcs_ctx *ctx, CpArgs &a, int64_t groups, int64_t Imax) {
  const int ra = (a.sb + 15) >> 4;
  const size_t smem = Cp12Smem::bytes(ra);
  const int cpt = int((Imax + wdit::w12::kNT - 1) / wdit::w12::kNT);
  const void *kern = cpt <= 1 ? cp12_pick_rmax<1>(ra) : cpt <= 2 ? cp12_pick_rmax<2>(ra)
                                                                 : cp12_pick_rmax<4>(ra);
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(cp12)");
  const float2 *twp = ctx->twiddle;
  void *args[] = {&a, &twp};
  e = launch_after_prep(ctx, kern, dim3(unsigned(groups), unsigned(a.D)), dim3(wdit::w12::kNT),
                        smem, args);
  return check_cuda(ctx, e, "cp12_kernel");
}

template <int LOG2M>
int launch_cp(fcs_ctx *ctx, CpArgs &a, int64_t groups, int64_t Imax) {
  if constexpr (LOG2M == wdit::kL) {
    return launch_cp13(ctx, a, groups, Imax);
  } else if constexpr (LOG2M == 12) {
    return launch_cp12(ctx, a, groups, Imax);
  } else {
    constexpr int NT = fft_threads(LOG2M);
    const size_t smem = CpSmem<LOG2M, NT>::bytes(a.sb);
    const int cpt = int((Imax + NT - 1) / NT);
    auto go = [&](auto kern) -> int {
      if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(cp)");
      }
      const float2 *twp = ctx->twiddle;
      void *args[] = {&a, &twp};
      return check_cuda(ctx,
                        launch_after_prep(ctx, reinterpret_cast<const void *>(kern),
                                          dim3(unsigned(groups), unsigned(a.D)), dim3(NT), smem,
                                          args),
                        "cp_kernel");
    };
    if (cpt <= 1) return go(cp_kernel<LOG2M, NT, 1>);
    if (cpt <= 2) return go(cp_kernel<LOG2M, NT, 2>);
    return go(cp_kernel<LOG2M, NT, 4>);       // larger modes add a direct tail loop
  }
}

}  // namespace
}  // namespace fcs

using namespace fcs;

namespace {

// Hash tables to generate from a seed into (h, s) (fcs_sketch_cp_seeded).
struct HashGen {
  uint64_t seed;
  int32_t *h;
  int8_t *s;
};

int sketch_cp_impl(fcs_ctx *ctx, int N, const int64_t *host_I, const int32_t *host_J,
                   int64_t R, int D, const float *const *host_U, const int64_t *host_ldU,
                   const float *lambda, const int32_t *h, const int8_t *s, int64_t ldh,
                   float *out, const HashGen *gen) {
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
    if (gen && host_I[n] > (int64_t(1) << 32))
      return set_error(ctx, FCS_EINVAL, "I[%d] too large for the hash family", n);
  }
  const int log2p = ilog2_ceil(a.m.Jt) < kMinLog2P ? kMinLog2P : ilog2_ceil(a.m.Jt);
  if (log2p > kMaxLog2PBig)
    return set_error(ctx, FCS_EUNSUPPORTED, "Jt=%lld needs FFT length > %d",
                     (long long)a.m.Jt, 1 << kMaxLog2PBig);
  if (log2p > kMaxLog2P) {
    if (gen) {                          // long route: tables by their own launch
      rc = fcs_make_hashes(ctx, gen->seed, N, host_I, host_J, D, gen->h, gen->s);
      if (rc) return rc;
    }
    DeviceGuard g(ctx->device);
    spec_cache_invalidate(ctx, out, sizeof(float) * size_t(D) * size_t(a.m.Jt));
    return big_sketch_cp(ctx, a.m, R, D, host_U, host_ldU, lambda, h, s, out, log2p);
  }
  const int log2m = log2p - 1;
  const int M = 1 << log2m;
  a.D = D;
  a.R = R;
  a.h = h;
  a.s = s;
  a.out = out;
  // rank groups: about one CTA per SM over all sketches (two for P = 8192,
  // whose engine fits two CTAs per SM)
  const int64_t slots = int64_t(ctx->sm_count) * (log2m == 12 ? 2 : 1);
  int64_t groups = (slots + D - 1) / D;
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
  const size_t gbytes = (sizeof(float2) * size_t(D) * size_t(M + 2) + 255) & ~size_t(255);
  const size_t cbytes = 256;
  void *ws = nullptr;
  rc = ensure_workspace(ctx, gbytes + cbytes + sizeof(float) * size_t(utlen), &ws);
  if (rc) return rc;
  a.G = static_cast<float2 *>(ws);
  a.counter = reinterpret_cast<unsigned *>(static_cast<char *>(ws) + gbytes);
  float *UT = reinterpret_cast<float *>(static_cast<char *>(ws) + gbytes + cbytes);
  a.UT = UT;
  DeviceGuard g(ctx->device);
  spec_cache_invalidate(ctx, out, sizeof(float) * size_t(D) * size_t(a.m.Jt));
  {
    // one launch: factor transpose (lambda folded into mode 1), clearing
    // of the accumulator and tickets, and the hash tables of a seed
    PrepArgs pa{};
    for (int n = 0; n < N; ++n) {
      pa.t.U[n] = host_U[n];
      pa.t.I[n] = host_I[n];
      pa.t.ld[n] = host_ldU[n];
      pa.t.ut_off[n] = a.ut_off[n];
    }
    pa.t.R = R;
    pa.t.lambda = lambda;
    pa.t.UT = UT;
    pa.tiles_x = (Imax + 31) / 32;
    pa.tiles_y = (R + 31) / 32;
    pa.ntile = pa.tiles_x * pa.tiles_y * N;
    pa.zero = static_cast<float4 *>(ws);
    pa.zero_n4 = int64_t(gbytes + cbytes) / 16;
    pa.zero_blocks = int(std::min<int64_t>(64, (pa.zero_n4 + 255) / 256));
    if (gen) {
      pa.hs = hash_args(gen->seed, N, D, host_I, host_J);
      pa.h = gen->h;
      pa.s = gen->s;
      pa.hash_per_d = (pa.hs.total + 255) / 256;
      pa.hash_blocks = int64_t(D) * pa.hash_per_d;
    }
    const int64_t blocks = pa.ntile + pa.zero_blocks + pa.hash_blocks;
    if (blocks > 0x7fffffffLL) return set_error(ctx, FCS_EUNSUPPORTED, "factor matrices too large");
    prep_kernel<<<unsigned(blocks), 256, 0, ctx->stream>>>(pa);
    rc = check_cuda(ctx, cudaGetLastError(), "prep_kernel");
    if (rc) return rc;
  }
  rc = FCS_EUNSUPPORTED;
  FCS_DISPATCH_LOG2M(log2m, rc = launch_cp<L>(ctx, a, groups, Imax));
  return rc;
}

}  // namespace

extern "C" int fcs_sketch_cp(fcs_ctx *ctx, int N, const int64_t *host_I,
                             const int32_t *host_J, int64_t R, int D,
                             const float *const *host_U, const int64_t *host_ldU,
                             const float *lambda, const int32_t *h, const int8_t *s,
                             int64_t ldh, float *out) {
  return sketch_cp_impl(ctx, N, host_I, host_J, R, D, host_U, host_ldU, lambda, h, s, ldh, out,
                        nullptr);
}

extern "C" int fcs_sketch_cp_seeded(fcs_ctx *ctx, uint64_t seed, int N, const int64_t *host_I,
                                    const int32_t *host_J, int64_t R, int D,
                                    const float *const *host_U, const int64_t *host_ldU,
                                    const float *lambda, int32_t *h, int8_t *s, float *out) {
  const HashGen g{seed, h, s};
  return sketch_cp_impl(ctx, N, host_I, host_J, R, D, host_U, host_ldU, lambda, h, s, 0, out,
                        h && s ? &g : nullptr);
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
  const size_t smem = LOG2M == wdit::kL ? Cp13Smem::bytes((a.sb + 31) >> 5)
                                        : CpSmem<LOG2M, NT>::bytes(a.sb);
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
  if constexpr (LOG2M == wdit::kL) {
    const void *kern = cp13_pick(Imax, a.sb);
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    void *args[] = {&a, &tw};
    e = cudaLaunchKernel(kern, dim3(unsigned(groups), unsigned(a.D)), dim3(NT), args, smem, st);
    if (e != cudaSuccess)
      return noalloc_fail(err, n, FCS_ECUDA, "cp13_kernel: %s", cudaGetErrorString(e));
    return FCS_OK;
  } else {
    if (cpt <= 1) return go(cp_kernel<LOG2M, NT, 1>);
    if (cpt <= 2) return go(cp_kernel<LOG2M, NT, 2>);
    return go(cp_kernel<LOG2M, NT, 4>);
  }
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
  {
    const int mrc = make_modes_msg(err, err_len, N, host_I, host_J, ldh, &a.m);
    if (mrc != FCS_OK) return mrc;
  }
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
  const size_t gbytes = (sizeof(float2) * size_t(D) * size_t(M + 2) + 255) & ~size_t(255);
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
  // the accumulator and tickets must start at zero (the array keeps the
  // previous call's contents); the same launch transposes the factors
  {
    PrepArgs pa{};
    for (int n = 0; n < N; ++n) {
      pa.t.U[n] = host_U[n];
      pa.t.I[n] = host_I[n];
      pa.t.ld[n] = host_ldU[n];
      pa.t.ut_off[n] = a.ut_off[n];
    }
    pa.t.R = R;
    pa.t.lambda = lambda;
    pa.t.UT = UT;
    pa.tiles_x = (Imax + 31) / 32;
    pa.tiles_y = (R + 31) / 32;
    pa.ntile = pa.tiles_x * pa.tiles_y * N;
    pa.zero = reinterpret_cast<float4 *>(sd->scratch);
    pa.zero_n4 = int64_t(gbytes + cbytes) / 16;
    pa.zero_blocks = int(std::min<int64_t>(64, (pa.zero_n4 + 255) / 256));
    prep_kernel<<<unsigned(pa.ntile + pa.zero_blocks), 256, 0, st>>>(pa);
    e = cudaGetLastError();
    if (e != cudaSuccess)
      return noalloc_fail(err, err_len, FCS_ECUDA, "prep: %s", cudaGetErrorString(e));
  }
  rc = FCS_EUNSUPPORTED;
  FCS_DISPATCH_LOG2M(log2m, rc = noalloc_launch_cp<L>(a, groups, Imax, sd->twiddle, st, err,
                                                      err_len));
  return rc;
}
