// fcs_ctx.cu -- context lifetime, errors, workspace and the twiddle table.
#include <cstdarg>
#include <cstring>

#include "fcs_internal.cuh"

namespace fcs {

int set_error(fcs_ctx *ctx, int code, const char *fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

int check_cuda(fcs_ctx *ctx, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return FCS_OK;
  return set_error(ctx, FCS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int grow_buffer(fcs_ctx *ctx, void **buf, size_t *have, size_t bytes, const char *what) {
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes <= *have) return FCS_OK;
  if (bytes > ctx->budget)
    return set_error(ctx, FCS_ENOMEM_BUDGET, "%s of %zu bytes exceeds the context budget of %zu",
                     what, bytes, ctx->budget);
  DeviceGuard g(ctx->device);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(ctx->stream, &cs);
  if (e != cudaSuccess) return check_cuda(ctx, e, "cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone)
    return set_error(ctx, FCS_EINVAL,
                     "%s would grow to %zu bytes while the stream is being captured: make the "
                     "same call once before capturing",
                     what, bytes);
  if (*buf) {
    // released after the work already queued on the stream has run
    e = cudaFreeAsync(*buf, ctx->stream);
    *buf = nullptr;
    *have = 0;
    if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFreeAsync");
  }
  e = cudaMallocAsync(buf, bytes, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return check_cuda(ctx, e, "cudaMallocAsync");
  }
  *have = bytes;
  return FCS_OK;
}

int ensure_workspace(fcs_ctx *ctx, size_t bytes, void **out) {
  int rc = grow_buffer(ctx, &ctx->ws, &ctx->ws_bytes, bytes, "workspace");
  if (rc) return rc;
  *out = ctx->ws;
  return FCS_OK;
}

int ensure_raw(fcs_ctx *ctx, size_t bytes) {
  void *p = ctx->raw;
  const int rc = grow_buffer(ctx, &p, &ctx->raw_bytes, bytes, "buffer");
  ctx->raw = static_cast<float *>(p);
  return rc;
}

namespace {
int msg_fail(char *err, size_t n, int code, const char *fmt, ...) {
  if (err && n) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, n, fmt, ap);
    va_end(ap);
  }
  return code;
}
}  // namespace

int make_modes_msg(char *err, size_t errn, int N, const int64_t *host_I,
                   const int32_t *host_J, int64_t ldh, Modes *m) {
  if (N < 1 || N > kMaxN) return msg_fail(err, errn, FCS_EINVAL, "N=%d outside [1,%d]", N, kMaxN);
  if (!host_I || !host_J) return msg_fail(err, errn, FCS_EINVAL, "host_I/host_J is NULL");
  m->N = N;
  int64_t tot = 0, jt = 1;
  for (int n = 0; n < N; ++n) {
    if (host_I[n] < 1 || host_I[n] > (int64_t(1) << 31) - 1)
      return msg_fail(err, errn, FCS_EINVAL, "I[%d]=%lld outside [1, 2^31)", n,
                      (long long)host_I[n]);
    if (host_J[n] < 1)
      return msg_fail(err, errn, FCS_EINVAL, "J[%d]=%d must be >= 1", n, host_J[n]);
    m->I[n] = host_I[n];
    m->J[n] = host_J[n];
    m->off[n] = tot;
    tot += host_I[n];
    jt += int64_t(host_J[n]) - 1;
  }
  for (int n = N; n < kMaxN; ++n) {
    m->I[n] = 1;
    m->J[n] = 1;
    m->off[n] = tot;
  }
  if (ldh == 0) ldh = tot;
  if (ldh < tot)
    return msg_fail(err, errn, FCS_EINVAL, "ldh=%lld smaller than sum(I)=%lld",
                    (long long)ldh, (long long)tot);
  if (jt > (int64_t(1) << 30))
    return msg_fail(err, errn, FCS_EUNSUPPORTED, "sketch length %lld too large", (long long)jt);
  m->ldh = ldh;
  m->Jt = jt;
  return FCS_OK;
}

int make_modes(fcs_ctx *ctx, int N, const int64_t *host_I, const int32_t *host_J,
               int64_t ldh, Modes *m) {
  char buf[256];
  buf[0] = '\0';
  const int rc = make_modes_msg(buf, sizeof(buf), N, host_I, host_J, ldh, m);
  if (rc) return set_error(ctx, rc, "%s", buf);
  return FCS_OK;
}

// tw[k] = exp(-2 pi i k / kTwN), evaluated in FP64 and rounded to FP32.
__global__ void twiddle_kernel(float2 *tw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < kTwN) {
    double s, c;
    sincospi(2.0 * double(k) / double(kTwN), &s, &c);
    tw[k] = make_float2(float(c), float(-s));
  }
}

}  // namespace fcs

using namespace fcs;

extern "C" int fcs_version(void) { return 10000; }

extern "C" int fcs_create(fcs_ctx **out, int device, void *stream, size_t budget) {
  if (!out) return FCS_EINVAL;
  *out = nullptr;
  fcs_ctx *ctx = new (std::nothrow) fcs_ctx();
  if (!ctx) return FCS_ENOMEM_BUDGET;
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->budget = budget;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    delete ctx;
    return FCS_ECUDA;
  }
  DeviceGuard g(device);
  int rc = FCS_OK;
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  cudaError_t e = cudaMalloc(&ctx->twiddle, sizeof(float2) * kTwN);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return FCS_ECUDA;
  }
  twiddle_kernel<<<kTwN / 256, 256, 0, ctx->stream>>>(ctx->twiddle);
  rc = check_cuda(ctx, cudaGetLastError(), "twiddle_kernel");
  if (rc == FCS_OK) rc = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "twiddle sync");
  if (rc != FCS_OK) {
    cudaFree(ctx->twiddle);
    delete ctx;
    return rc;
  }
  *out = ctx;
  return FCS_OK;
}

extern "C" int fcs_destroy(fcs_ctx *ctx) {
  if (!ctx) return FCS_OK;
  DeviceGuard g(ctx->device);
  // the buffers are stream-ordered allocations: nothing may still use them
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    cudaDeviceSynchronize();
  }
  batch_state_destroy(ctx);
  spec_cache_destroy(ctx);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->raw) cudaFree(ctx->raw);
  if (ctx->algo) cudaFree(ctx->algo);
  if (ctx->switch_ev) cudaEventDestroy(ctx->switch_ev);
  if (ctx->stage) cudaFree(ctx->stage);
  if (ctx->twiddle) cudaFree(ctx->twiddle);
  delete ctx;
  return FCS_OK;
}

extern "C" int fcs_set_stream(fcs_ctx *ctx, void *stream) {
  if (!ctx) return FCS_EINVAL;
  cudaStream_t next = static_cast<cudaStream_t>(stream);
  if (next == ctx->stream) return FCS_OK;
  // work queued so far may still use the context's buffers: the new stream
  // waits for it (no host synchronisation).  Skipped while either stream is
  // being captured into a CUDA graph, where the capture itself orders the work.
  DeviceGuard g(ctx->device);
  cudaStreamCaptureStatus c0 = cudaStreamCaptureStatusNone, c1 = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &c0) != cudaSuccess ||
      cudaStreamIsCapturing(next, &c1) != cudaSuccess ||
      c0 != cudaStreamCaptureStatusNone || c1 != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    ctx->stream = next;
    return FCS_OK;
  }
  if (!ctx->switch_ev) {
    cudaError_t e = cudaEventCreateWithFlags(&ctx->switch_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return check_cuda(ctx, e, "cudaEventCreate");
  }
  cudaError_t e = cudaEventRecord(ctx->switch_ev, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(next, ctx->switch_ev, 0);
  if (e != cudaSuccess) return check_cuda(ctx, e, "fcs_set_stream");
  ctx->stream = next;
  return FCS_OK;
}

extern "C" const char *fcs_last_error(const fcs_ctx *ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

extern "C" size_t fcs_workspace_bytes(const fcs_ctx *ctx) { return ctx ? ctx->ws_bytes : 0; }
