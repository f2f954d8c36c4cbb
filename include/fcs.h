/*
 * fcs.h -- C ABI of libfcs: Fast Count Sketch (FCS) on one GB300 (sm_103a).
 *
 * Method: X. Cao and J. Liu, "Efficient Tensor Contraction via Fast Count
 * Sketch" (arXiv 2106.13062).  Section, definition and equation names below
 * are the paper's.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an int status (FCS_OK on success).  On failure
 *    nothing is launched (argument errors) or the CUDA error is recorded
 *    (FCS_ECUDA); fcs_last_error() returns a message for the context.  No C++
 *    exception crosses this boundary.
 *  - Pointers are DEVICE pointers owned by the caller unless the parameter
 *    name starts with `host_`.  Results are written asynchronously on the
 *    context's stream and are valid once that stream has been synchronised.
 *  - Indices are 0-based.  The paper's 1-based bin sum_n h_n(i_n) - N + 1 is
 *    the bin sum_n h_n(i_n) here, so bins run over [0, Jt), with
 *    Jt = sum_n J_n - N + 1 (Def. 4).
 *  - Hash tables: h is int32, s is int8 (values +1/-1), both laid out
 *    [D][ldh] with mode n of sketch d at h[d*ldh + sum_{m<n} I_m + i].
 *    ldh = 0 means ldh = sum_n I_n (dense packing, as fcs_make_hashes writes).
 *    A larger ldh lets a call use a contiguous run of modes of a wider table
 *    (e.g. modes 3..4 of an order-4 table for the Kronecker workload).
 *  - Limits: 1 <= N <= 8, 1 <= D <= 16, 1 <= J_n, I_n >= 1, every entry of
 *    h for mode n in [0, J_n).  A hash value outside that range never makes
 *    a kernel touch memory out of bounds: the dense route drops the entries
 *    that use it (for that sketch only); gathers return NaN when the bin they
 *    read leaves their buffer -- recovery when the summed bin leaves
 *    [0, Jt) or an index i_n leaves [0, I_n), the free-mode gather of a
 *    contraction when h_m(i) leaves [0, P) -- and are otherwise unspecified;
 *    the Count Sketches of a contraction's vectors drop invalid entries.
 *    FFT-based calls (CP route, contractions, outer combine) need
 *    Jt <= 2^20: the FFT length is P = smallest power of
 *    two >= Jt, 16 <= P <= 2^20, else FCS_EUNSUPPORTED.  P <= 16384 runs one
 *    transform per CTA in shared memory.  The CP route at P = 32768 runs one
 *    fused kernel (one 2^14-point transform per CTA in shared memory, a
 *    128 KiB running-product slice per CTA in the context workspace, fewer
 *    CTAs when the budget is small).  Other longer transforms use a two-pass
 *    FFT through the context workspace (at most min(budget, 512 MiB), work
 *    split into chunks that fit; a few MiB suffice).  fcs_sketch_cp_noalloc
 *    takes P <= 16384.  Batch plans run P <= 16384 in their per-FFT-size
 *    launch chain and longer problems with the launches above.
 *  - The library allocates only its own context workspace (device memory
 *    reused across calls, bounded by the context's budget), a 256 KiB
 *    twiddle table, the staging buffer of fcs_sketch_cp_host when that is
 *    used and, when enabled, the spectrum cache of fcs_contract.
 *    A context must be used from one host thread at a time.
 *  - Floating point is FP32 throughout; sums use atomics, so the last bits
 *    of a result may differ from run to run.  Hashes and bins are exact.
 */
#ifndef FCS_H
#define FCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FCS_OK 0
#define FCS_EINVAL 1          /* bad argument (shape, pointer, limit)        */
#define FCS_ENOMEM_BUDGET 2   /* workspace would exceed the context budget    */
#define FCS_ECUDA 3           /* a CUDA runtime call failed                   */
#define FCS_ETIMEOUT 4        /* a bounded device wait gave up                */
#define FCS_EUNSUPPORTED 5    /* valid but outside what this build supports  */

/* contraction kinds for fcs_contract */
#define FCS_CONTRACT_ALL 0    /* T(v_1, ..., v_N): one scalar per batch item  */
#define FCS_CONTRACT_FREE 1   /* T(v_1, .., I (mode m), .., v_N): a vector    */

typedef struct fcs_ctx fcs_ctx;

/* Library version as 10000*major + 100*minor + patch. */
int fcs_version(void);

/* Create a context on CUDA device `device`, issuing all work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  `mem_budget_bytes`
 * caps the workspace the context may hold; (size_t)-1 means no cap, 0 means
 * no workspace at all (calls that need one return FCS_ENOMEM_BUDGET).
 * The workspace and the other context buffers grow on demand, ordered on the
 * context's stream (stream-ordered allocation: the old buffer is released
 * once the work queued before has run), so growth neither waits on the host
 * nor synchronises the device.  A call that would grow a buffer while the
 * stream is being captured into a CUDA graph returns FCS_EINVAL: make the
 * same call once before capturing.
 * Allocates the twiddle table (exp(-2 pi i k / 32768), k < 32768, computed in
 * FP64 on the device and rounded to FP32).  *ctx is NULL on failure. */
int fcs_create(fcs_ctx **ctx, int device, void *stream, size_t mem_budget_bytes);

/* Release the context, its workspace and twiddle table (synchronises its
 * stream first).  NULL is accepted. */
int fcs_destroy(fcs_ctx *ctx);

/* Change the stream later calls are issued on.  The new stream is made to
 * wait (an event, no host synchronisation) for the work already queued on
 * the old one, since both use the context's buffers; while either stream is
 * being captured into a CUDA graph the switch is made without that wait. */
int fcs_set_stream(fcs_ctx *ctx, void *stream);

/* Message for the last failing call on this context ("" if none).  The
 * pointer stays valid until the next call on the context. */
const char *fcs_last_error(const fcs_ctx *ctx);

/* Bytes of device workspace the context holds now. */
size_t fcs_workspace_bytes(const fcs_ctx *ctx);

/*
 * fcs_make_hashes -- the N hash pairs {h_n, s_n} of Def. 4 for D independent
 * sketches (the paper asks for 2-wise independent pairs, Def. 1; it fixes no
 * family).  Family: Carter-Wegman multiply-mod-prime over p = 2^61 - 1,
 *     h_n(i) = ((a_h i + b_h) mod p) mod J_n,
 *     s_n(i) = 1 - 2 (((a_s i + b_s) mod p) & 1),
 * with a = 1 + x mod (p-1), b = x mod p drawn from SplitMix64 seeded with
 * `seed`, four draws (a_h, b_h, a_s, b_s) per (d, n) in the order d-major,
 * n-minor.  Deterministic in (seed, N, I, J, D) and bit-identical to the
 * CPU oracle.
 *   host_I[N], host_J[N]: mode sizes and hash lengths (host memory).
 *   h [D][sum I] int32, s [D][sum I] int8: outputs, densely packed.
 */
int fcs_make_hashes(fcs_ctx *ctx, uint64_t seed, int N, const int64_t *host_I,
                    const int32_t *host_J, int D, int32_t *h, int8_t *s);

/*
 * fcs_sketch_dense -- FCS of a general tensor by the signed scatter of
 * eq. (FCS_asyn):  out_d[sum_n h_n(i_n)] += prod_n s_n(i_n) T(i_1..i_N).
 *   When one mode is contiguous (moved last internally if it is not the
 *   last; the sketch does not depend on mode order), the per-CTA partial
 *   sums are exact int32 fixed-point sums (power-of-two step per CTA, wraps
 *   carried, outliers and NaN/Inf added in FP32); the result is within FP32
 *   rounding of the exact sketch.  Other layouts accumulate in FP32.
 *   host_I[N]: mode sizes; host_stride[N]: element strides of T (NULL = C
 *   order, last mode contiguous); T: FP32 tensor; out [D][Jt] FP32 (zeroed
 *   by the call, then accumulated).  nbatch tensors of the same shape may be
 *   sketched in one launch: tensor b starts at T + b*T_batch_stride and its
 *   sketch at out + b*out_batch_stride (elements; nbatch = 1 ignores both).
 */
int fcs_sketch_dense(fcs_ctx *ctx, int N, const int64_t *host_I,
                     const int64_t *host_stride, const int32_t *host_J, int D,
                     const float *T, const int32_t *h, const int8_t *s,
                     int64_t ldh, float *out, int64_t nbatch,
                     int64_t T_batch_stride, int64_t out_batch_stride);

/*
 * fcs_sketch_cp -- FCS of a CP tensor [[lambda; U_1..U_N]] by eq. (FCS_syn):
 * per mode the Count Sketch of every factor column (Def. 1), a zero-padded
 * real FFT of length P >= Jt, the mode-wise product, the lambda-weighted sum
 * over rank (kept in the frequency domain; by linearity this equals the
 * paper's sum of inverse transforms) and one inverse FFT per sketch.
 *   host_U[N]: device pointers; U_n is I_n x R FP32 row-major with leading
 *   dimension host_ldU[n] >= R.  lambda [R] FP32 or NULL (all ones).
 *   out [D][Jt] FP32.
 *   Workspace for P <= 16384: A + 256 + 4*R*sum_n(I_n) bytes, rounded up to
 *   a multiple of 256, with A = D*(P/2+2)*8 rounded up to a multiple of 256
 *   (spectrum accumulator, tickets, factor columns transposed with lambda
 *   folded in).  P = 32768: A + 256 + 128 KiB per CTA (fewer CTAs, down to
 *   one, when the budget is smaller).  Longer: the two-pass route, chunked to
 *   what the budget allows (a few MiB suffice).
 */
int fcs_sketch_cp(fcs_ctx *ctx, int N, const int64_t *host_I,
                  const int32_t *host_J, int64_t R, int D,
                  const float *const *host_U, const int64_t *host_ldU,
                  const float *lambda, const int32_t *h, const int8_t *s,
                  int64_t ldh, float *out);

/*
 * fcs_sketch_cp_seeded -- fcs_make_hashes followed by fcs_sketch_cp in one
 * call: the hash tables of `seed` (bit for bit as fcs_make_hashes writes
 * them) go to h [D][sum I] int32 and s [D][sum I] int8 (device, densely
 * packed; the caller keeps them for contractions and recovery), and the
 * sketch of [[lambda; U_1..U_N]] to out [D][Jt], as fcs_sketch_cp with
 * those tables.  For P <= 16384 the tables are written by the same launch
 * that transposes the factors, so the call issues two kernels instead of
 * three; longer transforms generate them with their own launch first.
 * Arguments, workspace and errors otherwise as fcs_sketch_cp (and I_n <= 2^32
 * as fcs_make_hashes).
 */
int fcs_sketch_cp_seeded(fcs_ctx *ctx, uint64_t seed, int N, const int64_t *host_I,
                         const int32_t *host_J, int64_t R, int D,
                         const float *const *host_U, const int64_t *host_ldU,
                         const float *lambda, int32_t *h, int8_t *s, float *out);

/*
 * fcs_sketch_cp_host -- fcs_sketch_cp from and to HOST memory, with the hash
 * tables generated from `seed` (as fcs_make_hashes would, bit for bit).
 *   host_U[N]: HOST pointers, U_n is I_n x R FP32 row-major with leading
 *   dimension host_ldU[n] >= R; host_lambda: HOST [R] or NULL (all ones);
 *   host_out: HOST [D][Jt] FP32.
 * The call queues on the context's stream: the host-to-device copies of the
 * factors and lambda (ranges that follow each other in host memory move in
 * one copy; pinned memory makes them asynchronous), the hash generation, the
 * sketch, and the device-to-host copy of the result, which is complete once
 * the stream has been synchronised (the hash generation runs in the factor
 * transpose launch, as in fcs_sketch_cp_seeded).  The inputs must stay
 * unchanged until then.  Device staging of 4*(sum_n I_n*R + R) + 5*D*sum_n I_n + 4*D*Jt bytes
 * (each part rounded up to 256) is held by the context (within its budget,
 * beside the workspace fcs_sketch_cp uses).
 */
int fcs_sketch_cp_host(fcs_ctx *ctx, int N, const int64_t *host_I, const int32_t *host_J,
                       int64_t R, int D, const float *const *host_U, const int64_t *host_ldU,
                       const float *host_lambda, uint64_t seed, float *host_out);

/*
 * fcs_sketch_cp_noalloc -- fcs_sketch_cp for callers that cannot allocate
 * device memory.  (The paper has no counterpart: this is a deployment
 * variant.)  Some callers may not call cudaMalloc: code running inside a
 * host framework that owns every device byte through its own pool, loops
 * where the implicit device synchronisation of cudaMalloc / cudaFree would
 * stall other work, and processes whose device memory is fixed at start-up.
 * This entry point needs no fcs_ctx and allocates nothing: its scratch is a
 * file-scope __device__ array of 4 MiB (plus a 256 KiB twiddle table) that
 * every GPU loading the library holds until the process exits.
 *   - Runs on the calling thread's current device, on `stream`; every
 *     pointer must be memory of that device.
 *   - The first call on a device looks up the arrays' device addresses and
 *     fills the twiddle table, synchronising `stream` once; make that first
 *     call before any stream capture.
 *   - The scratch a problem needs is A + 256 + 4*R*sum_n(I_n) bytes, with
 *     A = D*(P/2+2)*8 rounded up to a multiple of 256 (P = FFT length <=
 *     16384).  Problems that need more than 4 MiB are rejected with
 *     FCS_ENOMEM_BUDGET (nothing is launched); longer FFTs with
 *     FCS_EUNSUPPORTED.
 *   - All calls share the one array: calls that overlap on the GPU (other
 *     streams, other host threads) race and corrupt each other's results.
 *     Each call clears the parts that must start at zero.
 *   - Having no context, it cannot drop spectrum-cache entries
 *     (fcs_cache_spectra) of `out`: after re-sketching into a buffer that a
 *     context has cached, call fcs_forget(ctx, out) on that context.
 *   - err (may be NULL) receives a message of at most err_len bytes.
 * Arguments and output otherwise as fcs_sketch_cp.
 */
int fcs_sketch_cp_noalloc(void *stream, int N, const int64_t *host_I,
                          const int32_t *host_J, int64_t R, int D,
                          const float *const *host_U, const int64_t *host_ldU,
                          const float *lambda, const int32_t *h, const int8_t *s,
                          int64_t ldh, float *out, char *err, size_t err_len);

/*
 * Batched CP-route sketches.  (The paper sketches one tensor at a time; this
 * is the batching layer over eq. (FCS_syn).)  Many CP tensors of uneven
 * order, sizes, rank and sketch length run in a few launches: the work is
 * cut into items (problem, sketch d, group of `grain` ranks) and grouped by
 * FFT length; one batched launch transposes every problem's factor columns,
 * then one kernel per FFT length P <= 16384 runs its items (one CTA per
 * item, largest FFT first), the kernels chained by programmatic dependent
 * launch so that each starts while the previous one drains.  The item that
 * completes a sketch (a ticket counter) runs its inverse FFT.  Problems with
 * P > 16384 follow with the long-FFT launches of fcs_sketch_cp, from
 * plan-owned scratch.  Results equal fcs_sketch_cp on each problem up to
 * FP32 summation order.
 */
typedef struct fcs_cp_problem {
  int N;                    /* order, 1..8 */
  int D;                    /* independent sketches, 1..16 */
  int64_t R;                /* CP rank, >= 1 */
  int64_t I[8];             /* mode sizes (first N used) */
  int32_t J[8];             /* hash lengths (first N used) */
  const float *U[8];        /* device: U_n, I_n x R row-major */
  int64_t ldU[8];           /* leading dimensions, >= R */
  const float *lambda;      /* device [R] or NULL (all ones) */
  const int32_t *h;         /* device hash table [D][ldh] */
  const int8_t *s;          /* device sign table [D][ldh] */
  int64_t ldh;              /* 0 = sum I_n */
  float *out;               /* device [D][Jt] */
} fcs_cp_problem;

typedef struct fcs_batch_plan fcs_batch_plan;

/* Validate a batch, cut its items and upload descriptors into plan-owned
 * device memory (counted against the context budget).  grain = ranks per
 * item; 0 = the autotuned grain for this batch shape if fcs_batch_autotune
 * has seen it (this context or the FCS_AUTOTUNE_CACHE file), else a default
 * of about four items per SM.  The class shapes are the autotuned ones for
 * this batch shape when known, else the defaults.  The plan records the problems' device
 * pointers: later launches read whatever those buffers hold then. */
int fcs_batch_plan_create(fcs_ctx *ctx, int nprob, const fcs_cp_problem *host_probs,
                          int grain, fcs_batch_plan **plan);

/* Issue the batch on the context's stream: one memset, one batched factor
 * transpose, one kernel per FFT length (the chain above) and the long
 * problems' launches.  No allocation and no host synchronisation, so the
 * call may be captured into a CUDA graph. */
int fcs_batch_plan_launch(fcs_ctx *ctx, const fcs_batch_plan *plan);

/* Release a plan (synchronises its context's stream first). */
int fcs_batch_plan_destroy(fcs_batch_plan *plan);

/* One-shot: create a plan, launch it, wait for it and release it. */
int fcs_batch_sketch_cp(fcs_ctx *ctx, int nprob, const fcs_cp_problem *host_probs,
                        int grain);

/* Shape of one FFT-length class of a batch plan.  engine: 0 = the slot FFT
 * (Stockham passes in shared memory, P <= 8192), 1 = the warp-DIT engine
 * (512-point sub-FFTs per warp, then a column step per thread; P = 8192, where
 * it is the default, and P = 16384, the only engine there).  thread_mult (slot FFT only): 1 = one
 * radix-16 butterfly per thread (P/32 threads, at least 32), 2 = twice as
 * many threads.  items_per_cta: 1, 2 or 4 work items run one after another by
 * each CTA.  threads: the block size that results (output of
 * fcs_batch_plan_config, ignored on input). */
typedef struct fcs_batch_class_cfg {
  int fft_len;              /* P, a power of two in [16, 16384] */
  int engine;
  int thread_mult;
  int items_per_cta;
  int threads;
} fcs_batch_class_cfg;

/* fcs_batch_plan_create with explicit class shapes (classes not listed take
 * the warp-DIT engine at P = 8192 and 16384, the slot FFT below, with
 * thread_mult = 1 and items_per_cta = 1) and grain (0 = the default grain). */
int fcs_batch_plan_create_cfg(fcs_ctx *ctx, int nprob, const fcs_cp_problem *host_probs,
                              int grain, int ncfg, const fcs_batch_class_cfg *host_cfg,
                              fcs_batch_plan **plan);

/* The grain and class shapes a plan was built with: *host_ncfg classes (the
 * first max_cfg of them copied to host_cfg, largest FFT first). */
int fcs_batch_plan_config(const fcs_batch_plan *plan, int *host_grain, int max_cfg,
                          fcs_batch_class_cfg *host_cfg, int *host_ncfg);

/* Autotuner: times the whole batch on the device.  First the grain (ranks
 * per item: 1, 2, 4, ... up to 64 and 2R) with every class at its default
 * shape; then, class by class from the largest FFT, every engine (for
 * P = 8192), thread_mult and items_per_cta with the other classes at their
 * best so far, a shape replacing the current one only when at least 3 %
 * faster.  The winner is
 * kept for this batch shape (sorted (FFT length, N, D, R, max I_n) of every
 * problem) and used by later plans of the same shape created with grain 0;
 * the grain goes to *host_best_grain; when the environment variable
 * FCS_AUTOTUNE_CACHE names a file, the table is persisted there. */
int fcs_batch_autotune(fcs_ctx *ctx, int nprob, const fcs_cp_problem *host_probs,
                       int *host_best_grain);

/*
 * Request server with continuous batching.  (No counterpart in the paper:
 * this is the serving layer over fcs_batch_* and fcs_contract.)
 * Clients on any host thread submit requests; one scheduler thread owns the
 * GPU.  It admits queued requests in FIFO order while in-flight slots, device
 * arena memory and pinned staging memory allow, and issues each admitted
 * group as one round on one of `streams` CUDA streams: host->device copies,
 * hash generation, one batched launch for all CP requests of the round,
 * contractions against resident sketches, device->host copies.  Several
 * rounds run at once, so requests that arrive while others are on the GPU
 * are admitted as soon as slots and memory free up and overlap with them.
 * Host buffers named in a request must stay valid until it completes.
 */
#define FCS_REQ_CP 0          /* sketch a CP tensor given by host factors     */
#define FCS_REQ_CONTRACT 1    /* contract vectors with a resident sketch      */

typedef struct fcs_server fcs_server;

typedef struct fcs_server_config {
  int device;               /* CUDA device */
  int streams;              /* rounds in flight at once, 1..8 */
  int max_inflight;         /* admitted, not yet completed requests */
  int max_batch;            /* CP requests per round */
  size_t arena_bytes;       /* device arena: request data, plans, resident sketches */
  size_t staging_bytes;     /* pinned host staging for copies and descriptors */
  size_t workspace_bytes;   /* per-stream context workspace budget */
} fcs_server_config;

typedef struct fcs_request {
  int kind;                 /* FCS_REQ_CP or FCS_REQ_CONTRACT */
  int N;                    /* order */
  int64_t I[8];             /* mode sizes */
  int32_t J[8];             /* hash lengths */
  /* FCS_REQ_CP */
  int D;                    /* sketches */
  int64_t R;                /* rank */
  uint64_t seed;            /* hash seed (fcs_make_hashes) */
  const float *host_U[8];   /* I_n x R row-major (leading dimension R) */
  const float *host_lambda; /* [R] or NULL */
  float *host_out;          /* [D][Jt] or NULL (then keep_resident must be 1) */
  int keep_resident;        /* keep sketch and hash tables on the device */
  /* FCS_REQ_CONTRACT */
  int64_t sketch_id;        /* a resident sketch (same N, I, J) */
  int contract_kind;        /* FCS_CONTRACT_ALL / FCS_CONTRACT_FREE */
  int free_mode;
  int64_t B;                /* vectors per mode */
  const float *host_vecs[8];/* [B][I_n] (free mode's may be NULL) */
  float *host_result;       /* [B] or [B][I_free] (median over D) */
} fcs_request;

typedef struct fcs_result {
  int64_t ticket;
  int state;                /* 0 queued, 1 running, 2 done, 3 failed, 4 cancelled */
  int status;               /* FCS_* of the request once finished */
  int64_t sketch_id;        /* CP with keep_resident: id for contractions */
  double latency_s;         /* submit -> completion, -1 while unfinished */
} fcs_result;

typedef struct fcs_stats {
  int64_t submitted, completed, failed, cancelled, rounds, sketches;
  int64_t max_inflight_seen;
  size_t arena_used;
  double p50_latency_s, p99_latency_s, mean_latency_s;
  double busy_s;            /* first submit -> last completion */
  int64_t batch_launches;   /* kernels of the rounds' batched CP launches
                               (a transpose and one per FFT size, per round) */
} fcs_stats;

/* Start a server (allocates the arena, staging and streams once). */
int fcs_server_create(const fcs_server_config *cfg, fcs_server **server);
/* Stop admitting, finish in-flight rounds, cancel queued requests, free. */
int fcs_server_destroy(fcs_server *server);
/* Queue a request; never blocks on the GPU.  FCS_ENOMEM_BUDGET when it could
 * never fit the arena or staging; FCS_EINVAL for bad fields or an unknown or
 * released sketch_id. */
int fcs_server_submit(fcs_server *server, const fcs_request *req, int64_t *ticket);
/* Non-blocking state of a request. */
int fcs_server_poll(fcs_server *server, int64_t ticket, fcs_result *res);
/* Wait at most timeout_s seconds; FCS_ETIMEOUT if still unfinished. */
int fcs_server_wait(fcs_server *server, int64_t ticket, double timeout_s, fcs_result *res);
/* Cancel a request that has not been admitted yet (else FCS_EINVAL). */
int fcs_server_cancel(fcs_server *server, int64_t ticket);
/* Drop a resident sketch once no queued or running request uses it. */
int fcs_server_release(fcs_server *server, int64_t sketch_id);
/* Counters and latency percentiles of completed requests. */
int fcs_server_stats(fcs_server *server, fcs_stats *out);
int fcs_server_reset_stats(fcs_server *server);

/*
 * fcs_contract -- sketched contractions of Sec. 4.1, one per batch item b:
 *  kind FCS_CONTRACT_ALL, eq. (T_uvw):
 *      raw[b][d] = < FCS_d(T), FCS_d(v_1 o ... o v_N) >, evaluated as
 *      (1/P) Re sum_k conj(F(FCS_d T))[k] prod_n F(CS_n v_n)[k] (Parseval);
 *      out_median[b] = median_d raw[b][d].
 *  kind FCS_CONTRACT_FREE with free mode m, eq. (T_Ivw) (m = 0) and the ALS
 *  columns T_(m)(...) (any m):
 *      z_d = IFFT(F(FCS_d T) prod_{n != m} conj F(CS_n v_n)),
 *      raw[b][d][i] = s_m(i) z_d[h_m(i)],  out_median[b][i] = median_d.
 *  fcsT [D][Jt]: the tensor's sketches (e.g. from fcs_sketch_dense).
 *  host_vecs[N]: device pointers, vector n is [B][I_n] FP32 (row b
 *  contiguous); for FREE the pointer of mode m is ignored and may be NULL.
 *  out_median: [B] (ALL) or [B][I_m] (FREE).  out_raw: NULL or [B][D] (ALL)
 *  / [B][D][I_m] (FREE).  Median over even D is the mean of the two middle
 *  values.  Workspace: D*(P/2+1)*8 bytes for the sketch spectra (none on a
 *  spectrum-cache hit) plus, when out_raw is NULL, 4*B*D*W bytes of raw
 *  estimates (W = 1 for ALL, I_m for FREE), each part rounded up to a
 *  multiple of 256.  For P > 16384 the raw buffer is a separate
 *  context-owned allocation counted against the same budget.
 */
int fcs_contract(fcs_ctx *ctx, int kind, int free_mode, int N,
                 const int64_t *host_I, const int32_t *host_J, int D,
                 const float *fcsT, int64_t B, const float *const *host_vecs,
                 const int32_t *h, const int8_t *s, int64_t ldh,
                 float *out_median, float *out_raw);

/*
 * fcs_contract_both -- both contractions of Sec. 4.1 for one set of vectors,
 * from one set of transforms: with p_d = F(FCS_d T) prod_{n != m}
 * conj F(CS_n v_n), the FREE result is IFFT(p_d) gathered as in
 * fcs_contract, and the ALL result is (1/P) Re sum_k conj(p_d[k])
 * F(CS_m v_m)[k], equal to eq. (T_uvw) because conj(p_d) F(CS_m v_m) =
 * conj(F(FCS_d T)) prod_n F(CS_n v_n).  N + 1 transforms per (item, sketch)
 * instead of 2N (the RTPM step: T(I,u,u) for the power iteration and
 * T(u,u,u) for the eigenvalue).
 *  host_vecs[N]: all N vectors, [B][I_n] each (the one of mode m too).
 *  out_all [B], out_free [B][I_m]: medians over the D sketches.
 *  out_all_raw: NULL or [B][D]; out_free_raw: NULL or [B][D][I_m].
 *  Other arguments and the workspace as for fcs_contract.  For FFT lengths
 *  above 16384 the two contractions run one after the other.
 */
int fcs_contract_both(fcs_ctx *ctx, int free_mode, int N, const int64_t *host_I,
                      const int32_t *host_J, int D, const float *fcsT, int64_t B,
                      const float *const *host_vecs, const int32_t *h,
                      const int8_t *s, int64_t ldh, float *out_all, float *out_free,
                      float *out_all_raw, float *out_free_raw);

/*
 * fcs_cache_spectra -- enable (1) or disable (0, the default; drops every
 * entry) the context's cache of sketch spectra for fcs_contract.  When on,
 * the D half spectra of fcsT that a contraction computes are kept in device
 * memory outside the workspace (at most 16 entries and min(budget/2, 512 MiB),
 * least recently used evicted) and reused by later contractions with the
 * same fcsT pointer, Jt, D and FFT length, which then skip the transform of
 * the sketch (e.g. the many contractions of one RTPM or ALS loop).  The key
 * is the pointer: the sketch calls made through this context drop the
 * entries of the buffers they write; after changing a cached sketch any
 * other way (another context, fcs_sketch_cp_noalloc, a copy), or before
 * freeing it, call fcs_forget.
 */
int fcs_cache_spectra(fcs_ctx *ctx, int enable);

/* fcs_forget -- invalidate the cached spectra of the sketch at ptr (recomputed
 * on next use; no-op if none).  Does not wait for the device. */
int fcs_forget(fcs_ctx *ctx, const void *ptr);

/*
 * fcs_fold -- Tensor Sketch (Def. 2) from Fast Count Sketch: with every
 * J_n = J the TS bin (sum_n h_n) mod J is the FCS bin reduced mod J, so
 *     out[r][j] = sum_{k = j mod J} in[r][k]
 * turns FCS sketches into the TS sketches with the same hash functions (the
 * comparison of Prop. 1).  in [nrows][Jt], out [nrows][J], rows contiguous;
 * 1 <= nrows <= 65535.
 */
int fcs_fold(fcs_ctx *ctx, int64_t nrows, int64_t Jt, const float *in, int64_t J, float *out);

/*
 * fcs_sketch_inner -- the compressed tensor regression layer (TRL
 * subsection, eq. net_compress): with the activation sketches sa
 * [B][D][Jt] (FCS_d of each input X_b) and weight sketches sw [C][D][Jt]
 * (FCS_d of each class's weight tensor W_c), all with the same hashes,
 *     raw[b][c][d] = < sa[b][d], sw[c][d] >,
 *     out_median[b][c] = median_d raw[b][c][d] + bias[c].
 * bias NULL or [C]; out_raw NULL or [B][C][D].  B <= 4194240.
 */
int fcs_sketch_inner(fcs_ctx *ctx, int D, int64_t Jt, int64_t B, const float *sa, int64_t C,
                     const float *sw, const float *bias, float *out_median, float *out_raw);

/*
 * fcs_rtpm -- sketched robust tensor power method (RTPM subsection) for a
 * symmetric order-N tensor of dimension I, from its sketches fcsT [D][Jt]
 * (hash tables h, s, ldh; every J_n from host_J[0..N)): for each of K
 * components, L starting vectors init[k][l][:] (normalised by the call),
 * n_iter power iterations u <- T(I,u,..,u) / ||T(I,u,..,u)|| (eq. T_Ivw,
 * free mode 0), eigenvalues T(u,..,u) (eq. T_uvw), both with the median
 * over the D sketches; the start with the largest eigenvalue gives
 * lambda[k] and U[k][:]; then the sketch is deflated,
 * FCS(T) <- FCS(T) - lambda_k FCS(u o .. o u) (linearity, eq. FCS_syn with
 * R = 1).  fcsT is not modified (the deflation runs on a copy in the
 * context's scratch).  init [K][L][I], lambda [K], U [K][I]: device.
 * 2 <= N <= 8, 1 <= L <= 65535.
 */
int fcs_rtpm(fcs_ctx *ctx, int N, int64_t I, const int32_t *host_J, int D, const float *fcsT,
             const int32_t *h, const int8_t *s, int64_t ldh, int K, int L, int n_iter,
             const float *init, float *lambda, float *U);

/*
 * fcs_als -- sketched CP-ALS (ALS subsection) of rank R <= 32 for an
 * order-N tensor from its sketches fcsT [D][Jt]: n_iter sweeps; for each
 * mode m the columns [T(.., I (mode m), ..)]_r with the other factors' r-th
 * columns (eq. T_Ivw, median over D), then F_m^T <- G^{-1} M^T with
 * G = *_{n != m} F_n F_n^T (Cholesky) and column normalisation.
 * host_F[n]: device [R][I_n], the transposed factor matrices (row r = column
 * r of U_n): starting values in, unit-norm factors out; lambda [R] out.
 */
int fcs_als(fcs_ctx *ctx, int N, const int64_t *host_I, const int32_t *host_J, int D,
            const float *fcsT, const int32_t *h, const int8_t *s, int64_t ldh, int R,
            int n_iter, float *const *host_F, float *lambda);

/*
 * fcs_recover -- entry estimates from sketches, the decompressing rule of the
 * Kronecker / tensor-contraction compression subsections (its mod(., Jt) never
 * wraps and is dropped):
 *     raw[d][q] = prod_n s_n(i_n) sketch_d[sum_n h_n(i_n)],  out[q] = median_d.
 *   sketch [D][Jt]; idx [M][N] int32 multi-indices, 0 <= i_n < I_n (checked
 *   on the device before any load: an index outside that range gives NaN,
 *   in out and in every raw value of that sample).  out [M]; out_raw NULL or [D][M].  nbatch problems sharing the
 *   hash tables: problem b uses sketch + b*sketch_batch_stride, idx +
 *   b*idx_batch_stride, out + b*out_batch_stride (elements; out_raw must be
 *   NULL when nbatch > 1).
 */
int fcs_recover(fcs_ctx *ctx, int N, const int64_t *host_I,
                const int32_t *host_J, int D, const float *sketch,
                const int32_t *h, const int8_t *s, int64_t ldh, int64_t M,
                const int32_t *idx, float *out, float *out_raw, int64_t nbatch,
                int64_t sketch_batch_stride, int64_t idx_batch_stride,
                int64_t out_batch_stride);

/*
 * fcs_sketch_outer -- sketch of an outer product (Kronecker product
 * compression): FCS(A o B) = IFFT(FFT(FCS A) * FFT(FCS B)), zero-padded to a
 * power of two P >= La + Lb - 1, i.e. the full linear convolution of the two
 * sketches.  fa [nbatch][D][La], fb [nbatch][D][Lb] -> out
 * [nbatch][D][La+Lb-1], all contiguous FP32.
 */
int fcs_sketch_outer(fcs_ctx *ctx, int64_t nbatch, int D, int64_t La,
                     int64_t Lb, const float *fa, const float *fb, float *out);

/*
 * fcs_sketch_outer_sum -- sketch of a contraction over one mode from the
 * sketches of its slices (tensor contraction compression): for A with
 * slices A_l = A(:,:,l) and B with slices B_l = B(l,:,:),
 *     FCS_d(A (x)_{3,1} B) = sum_l FCS_d(A_l) (*) FCS_d(B_l),
 * the full linear convolutions summed in the frequency domain (one inverse
 * per item and sketch).  fa [nbatch][L][D][La] (slice sketches with the
 * hash tables of the first two modes), fb [nbatch][L][D][Lb] (the last
 * two), out [nbatch][D][La+Lb-1].  L = 1 is fcs_sketch_outer.
 */
int fcs_sketch_outer_sum(fcs_ctx *ctx, int64_t nbatch, int64_t L, int D, int64_t La, int64_t Lb,
                         const float *fa, const float *fb, float *out);

/*
 * fcs_outer_autotune -- choose the block shape of fcs_sketch_outer /
 * fcs_sketch_outer_sum for one problem shape (nbatch, L, D, La, Lb; L = 1 for
 * fcs_sketch_outer).  Each (item, sketch) runs on one CTA whose real FFTs use
 * M/16 threads (M = P/2, at least a warp) or twice that; the call runs both
 * on the given buffers (writing `out` several times, synchronising the
 * context's stream) and keeps the twice-as-many-threads shape for this
 * device and shape only when it is at least 3 % faster.  Later calls of the
 * same shape, in any context on this device, use the choice.  Shapes with
 * P > 16384 (the two-pass route) have one shape.  *host_threads (may be
 * NULL) receives the chosen block size (0 for P > 16384).  When the call
 * returns, `out` holds the result of the shape run last (the
 * twice-as-many-threads one where there are two); it is complete once the
 * context's stream has been synchronised.
 */
int fcs_outer_autotune(fcs_ctx *ctx, int64_t nbatch, int64_t L, int D, int64_t La, int64_t Lb,
                       const float *fa, const float *fb, float *out, int *host_threads);

#ifdef __cplusplus
}
#endif

#endif /* FCS_H */
