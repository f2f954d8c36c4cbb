// fcs_batch_internal.cuh -- batch building blocks shared by the batch API
// (fcs_batch.cu) and the request server (fcs_server.cu).  Not part of the ABI.
#pragma once

#include <vector>

#include "fcs_internal.cuh"

namespace fcs {

// Tunable shape of one FFT-size class (log2 M = L): the engine (for P = 8192
// the slot FFT or the warp-DIT engine; P = 16384 always runs warp-DIT, the
// other sizes the slot FFT), the slot FFT's thread multiplier ntm (1 or 2:
// M/16 or M/8 threads, at least a warp) and items run one after another per
// CTA (ipc: 1, 2 or 4).
struct ClassCfg {
  int L, ntm, ipc;
  int eng = 0;               // P = 8192: 0 = slot FFT, 1 = warp-DIT engine
};

// One launch of a batch: the items [first, first + count) of one FFT size.
struct BatchClass {
  const void *fn;            // kernel
  int nt;                    // threads per CTA
  size_t smem;               // dynamic shared memory per CTA
  int first, count;
  int L, ntm, ipc, eng;      // the configuration it was built with
};

// Layout of one batch in device memory (see batch_build).
struct BatchBuild {
  size_t total = 0;          // device bytes
  size_t desc_bytes = 0;     // descriptor image (host copy -> device base)
  size_t items_off = 0, tasks_off = 0;
  size_t clear_off = 0, clear_bytes = 0;
  int nitems = 0, ntasks = 0;
  int64_t tiles = 0;
  std::vector<BatchClass> classes;
};

// Lay the batch out at device address `base` (NULL: sizes only, in *out).
// cfg (may be NULL) gives the shape of each FFT-size class it names; other
// classes take ntm = 1, ipc = 1.
int batch_build(fcs_ctx *ctx, int nprob, const fcs_cp_problem *q, int grain, char *base,
                std::vector<char> *host_desc, BatchBuild *out,
                const std::vector<ClassCfg> *cfg = nullptr);
// Clear accumulators, transpose factors, run the class kernels on
// ctx->stream; the descriptor image must already be at `base`.
int batch_issue(fcs_ctx *ctx, char *base, const BatchBuild &b);
// About four work items per SM.
int batch_default_grain(fcs_ctx *ctx, int nprob, const fcs_cp_problem *q);

}  // namespace fcs
