// fcs_batch.cu -- fcs_batch_sketch_cp / fcs_batch_autotune: many CP-route
// sketches (eq. FCS_syn) of uneven order, sizes, rank and sketch length in a
// few launches.
//
// Host side (fcs_batch_plan_create): the work is cut into items (problem p,
// sketch d, group of `grain` ranks), grouped by FFT size (largest first;
// within a size, the longest items first), and uploaded once with the
// problem descriptors into plan-owned device memory.  A launch
// (fcs_batch_plan_launch) issues only device work -- clear the accumulators,
// transpose every problem's factor columns in one batched launch, run one
// kernel per FFT size -- so it can be captured into a CUDA graph and
// replayed.  Device side: each size class runs with the block size and
// engine of the single-problem kernel for that size (cp_run / cp13_run of
// fcs_cp_run.cuh), one CTA per item: count sketch into a compact shared
// buffer, block real FFT, mode product in registers, rank sum in shared
// memory, the item's partial spectrum into the problem's accumulator, and
// the item that completes sketch (p, d) (ticket counter) runs that sketch's
// inverse FFT.  The class launches form a chain of programmatic dependent
// launches, so a class starts while the previous one drains.  No CTA ever
// waits on another CTA of its own grid.
//
// The grain (ranks per item) trades load balance against the number of
// partial-spectrum flushes.  fcs_batch_autotune times the whole batch for
// each candidate grain on the device and keeps the fastest per batch
// signature (in the context, and in the file named by FCS_AUTOTUNE_CACHE
// when that variable is set).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <array>
#include <cstring>
#include <map>
#include <set>
#include <vector>

#include "fcs_batch_kernels.cuh"

struct fcs_batch_state {
  // batch signature -> autotuned grain and class shapes
  std::map<uint64_t, std::pair<int, std::vector<fcs::ClassCfg>>> tuned;
  bool cache_loaded = false;
  std::set<fcs_batch_plan *> plans;   // live plans; detached when the context goes
};

struct fcs_batch_plan {
  int device = 0;
  void *dev = nullptr;             // descriptors, items, tasks, tickets, G, UT
  size_t bytes = 0;
  fcs::BatchBuild build{};
  fcs_ctx *owner = nullptr;
  std::vector<std::pair<const void *, size_t>> outs;   // output sketches written
  std::vector<fcs_cp_problem> longp;   // problems with P > 16384: their own launches
  void *long_ws = nullptr;             // their scratch, owned by the plan (graph-safe)
  size_t long_bytes = 0;
  int grain = 0;                       // ranks per item it was built with
};

namespace fcs {
namespace {

struct TransposeTask {
  const float *U;
  const float *lambda;
  float *UT;
  int64_t I, R, ld;
  int64_t tiles_i, tile0;   // tiles along I; first flat tile index
};

// One CTA per 32x32 tile of one factor matrix; the task is found by binary
// search over the tasks' first tile indices.
__global__ void batch_transpose_kernel(const TransposeTask *__restrict__ tasks, int ntasks) {
  __shared__ float tile[32][33];
  const int64_t t = blockIdx.x;
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (tasks[mid].tile0 <= t) lo = mid; else hi = mid - 1;
  }
  const TransposeTask T = tasks[lo];
  const int64_t local = t - T.tile0;
  const int64_t i0 = (local % T.tiles_i) * 32, r0 = (local / T.tiles_i) * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = i0 + k, r = r0 + threadIdx.x;
    if (i < T.I && r < T.R) tile[k][threadIdx.x] = T.U[i * T.ld + r];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k, i = i0 + threadIdx.x;
    if (i < T.I && r < T.R) {
      const float lam = T.lambda ? __ldg(T.lambda + r) : 1.f;
      T.UT[r * T.I + i] = tile[threadIdx.x][k] * lam;
    }
  }
}

// Engine of a class without a tuned or explicit shape: the warp-DIT engines
// where they exist (P = 8192 and 16384), the slot FFT below.
int default_engine(int L) { return (L == wdit::kL || L == 12) ? 1 : 0; }

// Class kernel for log2 M = L with engine eng, at thread multiplier ntm (slot
// FFT only; the warp-DIT engines have one thread count) running ipc items
// per CTA.
ClassKernel class_kernel(int L, int eng, int ntm, int ipc, int64_t Imax, int sb) {
  if (L == wdit::kL) return class_kernel_13(ipc, Imax, sb);
  if (L == 12) return class_kernel_12(eng, ntm, ipc, Imax, sb);
  if (L >= 10) return class_kernel_mid(L, ntm, ipc, Imax, sb);
  return class_kernel_small(L, ntm, ipc, Imax, sb);
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Per-problem facts derived on the host.
struct HostProb {
  Modes m;
  int L, sb;
  int64_t R, utlen, Imax;
  bool longp;                  // P > 16384: not for the batch kernels
};

int check_problem(fcs_ctx *ctx, int k, const fcs_cp_problem &q, HostProb *hp) {
  int rc = make_modes(ctx, q.N, q.I, q.J, q.ldh, &hp->m);
  if (rc) return set_error(ctx, rc, "problem %d: %s", k, ctx->err.c_str());
  if (q.D < 1 || q.D > kMaxD) return set_error(ctx, FCS_EINVAL, "problem %d: D=%d", k, q.D);
  if (q.R < 1) return set_error(ctx, FCS_EINVAL, "problem %d: R=%lld", k, (long long)q.R);
  if (!q.h || !q.s || !q.out) return set_error(ctx, FCS_EINVAL, "problem %d: NULL pointer", k);
  int64_t ut = 0, imax = 0, jmax = 0;
  for (int n = 0; n < q.N; ++n) {
    if (!q.U[n]) return set_error(ctx, FCS_EINVAL, "problem %d: U[%d] is NULL", k, n);
    if (q.ldU[n] < q.R) return set_error(ctx, FCS_EINVAL, "problem %d: ldU[%d] < R", k, n);
    ut += q.R * q.I[n];
    imax = std::max<int64_t>(imax, q.I[n]);
    jmax = std::max<int64_t>(jmax, q.J[n]);
  }
  int log2p = ilog2_ceil(hp->m.Jt);
  if (log2p < kMinLog2P) log2p = kMinLog2P;
  if (log2p > kMaxLog2PBig)
    return set_error(ctx, FCS_EUNSUPPORTED, "problem %d: Jt=%lld needs FFT length > %d", k,
                     (long long)hp->m.Jt, 1 << kMaxLog2PBig);
  hp->longp = log2p > kMaxLog2P;
  hp->L = log2p - 1;
  hp->sb = int((jmax + 3) / 4 * 4);
  hp->R = q.R;
  hp->utlen = ut;
  hp->Imax = imax;
  return FCS_OK;
}

uint64_t batch_signature(int nprob, const std::vector<HostProb> &hp,
                         const fcs_cp_problem *q) {
  std::vector<std::array<int64_t, 5>> keys(nprob);
  for (int k = 0; k < nprob; ++k)
    keys[k] = {hp[k].L, q[k].N, q[k].D, hp[k].R, hp[k].Imax};
  std::sort(keys.begin(), keys.end());
  uint64_t x = 1469598103934665603ull;   // FNV-1a
  auto mixin = [&](uint64_t v) {
    for (int b = 0; b < 8; ++b) {
      x ^= (v >> (8 * b)) & 0xff;
      x *= 1099511628211ull;
    }
  };
  mixin(uint64_t(nprob));
  for (auto &k : keys)
    for (int64_t v : k) mixin(uint64_t(v));
  return x;
}

// Cache file: one line per batch signature, "sig grain L:ntm:ipc:eng ..."
// (a missing engine field reads as 0).
void load_cache(fcs_batch_state &st) {
  if (st.cache_loaded) return;
  st.cache_loaded = true;
  const char *path = getenv("FCS_AUTOTUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "r");
  if (!f) return;
  char line[4096];
  while (fgets(line, sizeof(line), f)) {
    unsigned long long sig;
    int g, used = 0;
    if (sscanf(line, "%llx %d%n", &sig, &g, &used) != 2) continue;
    std::vector<ClassCfg> cfg;
    const char *p = line + used;
    while (true) {
      ClassCfg c;
      int n = 0, n4 = 0;
      if (sscanf(p, " %d:%d:%d%n", &c.L, &c.ntm, &c.ipc, &n) != 3) break;
      if (sscanf(p + n, ":%d%n", &c.eng, &n4) == 1) n += n4;
      cfg.push_back(c);
      p += n;
    }
    st.tuned[sig] = {g, cfg};
  }
  fclose(f);
}

void save_cache(const fcs_batch_state &st) {
  const char *path = getenv("FCS_AUTOTUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "w");
  if (!f) return;
  for (auto &kv : st.tuned) {
    fprintf(f, "%016llx %d", (unsigned long long)kv.first, kv.second.first);
    for (const ClassCfg &c : kv.second.second)
      fprintf(f, " %d:%d:%d:%d", c.L, c.ntm, c.ipc, c.eng);
    fprintf(f, "\n");
  }
  fclose(f);
}

int default_grain(const fcs_ctx *ctx, int nprob, const fcs_cp_problem *q) {
  int64_t work = 0;
  int64_t rmax = 1;
  for (int k = 0; k < nprob; ++k) {
    work += int64_t(q[k].D) * q[k].R;
    rmax = std::max<int64_t>(rmax, q[k].R);
  }
  // about four items per SM, power-of-two grain
  int64_t g = work / (4 * int64_t(std::max(1, ctx->sm_count)));
  int grain = 1;
  while (grain * 2 <= g && grain < 64) grain *= 2;
  return int(std::min<int64_t>(grain, rmax));
}

}  // namespace

// Lay a batch out at device address `base` (NULL: sizes only).  The device
// image starts with the descriptors (probs | items | tasks), `desc_bytes`
// long, whose host copy goes to *host_desc; then the cleared region
// (tickets | spectrum accumulators) and the transposed factors.  Items are
// grouped into FFT-size classes, largest first, each class's longest items
// (ranks x modes) first.
int batch_build(fcs_ctx *ctx, int nprob, const fcs_cp_problem *q, int grain, char *base,
                std::vector<char> *host_desc, BatchBuild *out,
                const std::vector<ClassCfg> *cfg) {
  std::vector<HostProb> hp(nprob);
  for (int k = 0; k < nprob; ++k) {
    int rc = check_problem(ctx, k, q[k], &hp[k]);
    if (rc) return rc;
    if (hp[k].longp)
      return set_error(ctx, FCS_EUNSUPPORTED,
                       "problem %d: FFT length > %d is not run by the batch kernels", k,
                       1 << kMaxLog2P);
  }
  std::vector<int4> items;
  std::vector<BatchProb> probs(nprob);
  int ntask = 0;
  size_t g_bytes = 0, t_count = 0, ut_len = 0;
  for (int k = 0; k < nprob; ++k) {
    const int64_t rpi = std::min<int64_t>(std::max(grain, 1), hp[k].R);
    const int groups = int((hp[k].R + rpi - 1) / rpi);
    memset(&probs[k], 0, sizeof(BatchProb));
    probs[k].rpi = rpi;
    probs[k].groups = groups;
    for (int d = 0; d < q[k].D; ++d)
      for (int g = 0; g < groups; ++g) items.push_back(make_int4(k, d, g, 0));
    g_bytes += up256(sizeof(float2) * size_t(q[k].D) * size_t((1 << hp[k].L) + 2));
    t_count += size_t(q[k].D);
    ut_len += size_t(hp[k].utlen);
    ntask += q[k].N;
  }
  // largest FFT first, then the longest items (ranks x modes)
  std::stable_sort(items.begin(), items.end(), [&](const int4 &x, const int4 &y) {
    const int lx = hp[x.x].L, ly = hp[y.x].L;
    if (lx != ly) return lx > ly;
    return probs[x.x].rpi * q[x.x].N > probs[y.x].rpi * q[y.x].N;
  });
  const size_t b_probs = up256(sizeof(BatchProb) * nprob);
  const size_t b_items = up256(sizeof(int4) * items.size());
  const size_t b_tasks = up256(sizeof(TransposeTask) * ntask);
  const size_t b_tick = up256(sizeof(unsigned) * t_count);
  const size_t b_ut = up256(sizeof(float) * ut_len);
  BatchBuild bb{};
  bb.total = b_probs + b_items + b_tasks + b_tick + g_bytes + b_ut;
  bb.desc_bytes = b_probs + b_items + b_tasks;
  bb.items_off = b_probs;
  bb.tasks_off = b_probs + b_items;
  bb.clear_off = b_probs + b_items + b_tasks;
  bb.clear_bytes = b_tick + g_bytes;
  bb.nitems = int(items.size());
  bb.ntasks = ntask;
  if (!base) {
    *out = bb;
    return FCS_OK;
  }
  unsigned *d_tickets = reinterpret_cast<unsigned *>(base + bb.clear_off);
  char *g_base = base + bb.clear_off + b_tick;
  float *ut_base = reinterpret_cast<float *>(g_base + g_bytes);
  std::vector<TransposeTask> tasks;
  size_t goff = 0, toff = 0, uoff = 0;
  int64_t tiles = 0;
  for (int k = 0; k < nprob; ++k) {
    BatchProb &P = probs[k];
    P.N = q[k].N;
    P.D = q[k].D;
    P.L = hp[k].L;
    P.sb = hp[k].sb;
    P.R = hp[k].R;
    for (int n = 0; n < kMaxN; ++n) {
      P.I[n] = hp[k].m.I[n];
      P.off[n] = hp[k].m.off[n];
    }
    P.ldh = hp[k].m.ldh;
    P.Jt = hp[k].m.Jt;
    P.h = q[k].h;
    P.s = q[k].s;
    P.out = q[k].out;
    P.G = reinterpret_cast<float2 *>(g_base + goff);
    goff += up256(sizeof(float2) * size_t(P.D) * size_t((1 << P.L) + 2));
    P.tickets = d_tickets + toff;
    toff += size_t(P.D);
    P.UT = ut_base + uoff;
    int64_t local = 0;
    for (int n = 0; n < P.N; ++n) {
      P.ut_off[n] = local;
      TransposeTask T;
      T.U = q[k].U[n];
      T.lambda = n == 0 ? q[k].lambda : nullptr;
      T.UT = ut_base + uoff + local;
      T.I = q[k].I[n];
      T.R = P.R;
      T.ld = q[k].ldU[n];
      T.tiles_i = (T.I + 31) / 32;
      T.tile0 = tiles;
      tiles += T.tiles_i * ((T.R + 31) / 32);
      tasks.push_back(T);
      local += P.R * q[k].I[n];
    }
    uoff += size_t(local);
  }
  // one launch per FFT-size class: prefetch depth and scatter buffer sized
  // for the class's largest problem
  for (size_t i = 0; i < items.size();) {
    const int L = hp[items[i].x].L;
    size_t j = i;
    int64_t Imax = 0;
    int sb = 4;
    for (; j < items.size() && hp[items[j].x].L == L; ++j) {
      Imax = std::max(Imax, hp[items[j].x].Imax);
      sb = std::max(sb, hp[items[j].x].sb);
    }
    ClassCfg c{L, 1, 1, default_engine(L)};
    if (cfg)
      for (const ClassCfg &x : *cfg)
        if (x.L == L) c = x;
    c.eng = L == wdit::kL ? 1 : (L == 12 && c.eng == 1 ? 1 : 0);
    if (c.eng == 1 || (c.ntm != 1 && c.ntm != 2)) c.ntm = 1;
    if (c.ipc != 1 && c.ipc != 2 && c.ipc != 4) c.ipc = 1;
    const ClassKernel ck = class_kernel(L, c.eng, c.ntm, c.ipc, Imax, sb);
    if (!ck.fn) return set_error(ctx, FCS_EUNSUPPORTED, "no batch kernel for log2 M = %d", L);
    if (ck.smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(ck.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(ck.smem));
      if (e != cudaSuccess) return check_cuda(ctx, e, "cudaFuncSetAttribute(batch class)");
    }
    bb.classes.push_back(
        BatchClass{ck.fn, ck.nt, ck.smem, int(i), int(j - i), L, c.ntm, c.ipc, c.eng});
    i = j;
  }
  if (tiles > 0x7fffffffLL) return set_error(ctx, FCS_EUNSUPPORTED, "batch too large");
  host_desc->assign(bb.desc_bytes, 0);
  memcpy(host_desc->data(), probs.data(), sizeof(BatchProb) * nprob);
  memcpy(host_desc->data() + b_probs, items.data(), sizeof(int4) * items.size());
  memcpy(host_desc->data() + b_probs + b_items, tasks.data(),
         sizeof(TransposeTask) * tasks.size());
  bb.tiles = tiles;
  *out = bb;
  return FCS_OK;
}

// Device work of one batch on ctx->stream (descriptors already in place).
int batch_issue(fcs_ctx *ctx, char *base, const BatchBuild &b) {
  int rc = check_cuda(ctx, cudaMemsetAsync(base + b.clear_off, 0, b.clear_bytes, ctx->stream),
                      "cudaMemsetAsync(batch accumulators)");
  if (rc) return rc;
  batch_transpose_kernel<<<unsigned(b.tiles), dim3(32, 8), 0, ctx->stream>>>(
      reinterpret_cast<const TransposeTask *>(base + b.tasks_off), b.ntasks);
  rc = check_cuda(ctx, cudaGetLastError(), "batch_transpose_kernel");
  if (rc) return rc;
  // the classes as a chain of programmatic dependent launches: each may start
  // while its predecessor drains (their problems are disjoint), and each
  // completes after it
  const BatchProb *probs = reinterpret_cast<const BatchProb *>(base);
  const float2 *tw = ctx->twiddle;
  for (size_t c = 0; c < b.classes.size(); ++c) {
    const BatchClass &k = b.classes[c];
    const int4 *items = reinterpret_cast<const int4 *>(base + b.items_off) + k.first;
    int count = k.count, ipc = k.ipc;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned((k.count + k.ipc - 1) / k.ipc));
    cfg.blockDim = dim3(unsigned(k.nt));
    cfg.dynamicSmemBytes = k.smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = c > 0 ? 1 : 0;
    void *args[] = {&probs, &items, &tw, &count, &ipc};
    rc = check_cuda(ctx, cudaLaunchKernelExC(&cfg, k.fn, args), "batch_class_kernel");
    if (rc) return rc;
  }
  return FCS_OK;
}

int batch_default_grain(fcs_ctx *ctx, int nprob, const fcs_cp_problem *q) {
  return default_grain(ctx, nprob, q);
}

namespace {

// Build a plan: lay the batch out in plan-owned device memory and upload the
// descriptors.
int plan_create(fcs_ctx *ctx, int nprob_all, const fcs_cp_problem *q_all, int grain,
                fcs_batch_plan **out, const std::vector<ClassCfg> *cfg = nullptr) {
  *out = nullptr;
  // problems with P > 16384 run after the batch kernels, each with the
  // multi-kernel long-FFT route
  std::vector<fcs_cp_problem> shortp, longp;
  for (int k = 0; k < nprob_all; ++k) {
    HostProb hp{};
    int rc = check_problem(ctx, k, q_all[k], &hp);
    if (rc) return rc;
    (hp.longp ? longp : shortp).push_back(q_all[k]);
  }
  const int nprob = int(shortp.size());
  const fcs_cp_problem *q = shortp.data();
  BatchBuild bb{};
  std::vector<char> desc;
  int rc = nprob ? batch_build(ctx, nprob, q, grain, nullptr, &desc, &bb, cfg) : FCS_OK;
  if (rc) return rc;
  if (ctx->ws_bytes + ctx->plan_bytes + bb.total > ctx->budget)
    return set_error(ctx, FCS_ENOMEM_BUDGET,
                     "batch plan of %zu bytes exceeds the context budget of %zu", bb.total,
                     ctx->budget);
  fcs_batch_plan *plan = new (std::nothrow) fcs_batch_plan();
  if (!plan) return set_error(ctx, FCS_ENOMEM_BUDGET, "out of host memory");
  if (nprob) {
    cudaError_t e = cudaMalloc(&plan->dev, bb.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete plan;
      return check_cuda(ctx, e, "cudaMalloc(batch plan)");
    }
    rc = batch_build(ctx, nprob, q, grain, static_cast<char *>(plan->dev), &desc, &bb, cfg);
    if (rc == FCS_OK)
      rc = check_cuda(ctx,
                      cudaMemcpy(plan->dev, desc.data(), desc.size(), cudaMemcpyHostToDevice),
                      "cudaMemcpy(batch descriptors)");
    if (rc) {
      cudaFree(plan->dev);
      delete plan;
      return rc;
    }
  }
  plan->bytes = bb.total;
  plan->device = ctx->device;
  plan->owner = ctx;
  plan->longp = longp;
  if (!longp.empty()) {
    // one scratch buffer for the long problems, run one after another; a
    // modest cap keeps the plan small (the route works in chunks)
    size_t room = ctx->budget > ctx->ws_bytes + ctx->plan_bytes + bb.total
                      ? ctx->budget - (ctx->ws_bytes + ctx->plan_bytes + bb.total)
                      : 0;
    const size_t cap = std::min<size_t>(room, size_t(256) << 20);
    size_t need = 0;
    for (const fcs_cp_problem &p : longp) {
      Modes m{};
      make_modes(ctx, p.N, p.I, p.J, p.ldh, &m);
      const int log2p = ilog2_ceil(m.Jt);
      need = std::max(need, big_sketch_cp_bytes(m, p.R, p.D, log2p, cap, ctx->sm_count));
    }
    cudaError_t e = need > cap ? cudaErrorMemoryAllocation : cudaMalloc(&plan->long_ws, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (plan->dev) cudaFree(plan->dev);
      delete plan;
      return set_error(ctx, FCS_ENOMEM_BUDGET, "no room for the long problems' scratch (%zu B)",
                       need);
    }
    plan->long_bytes = need;
  }
  for (int k = 0; k < nprob_all; ++k) {
    int64_t jt = 1;
    for (int n = 0; n < q_all[k].N; ++n) jt += int64_t(q_all[k].J[n]) - 1;
    plan->outs.emplace_back(q_all[k].out, sizeof(float) * size_t(q_all[k].D) * size_t(jt));
  }
  plan->build = bb;
  plan->grain = grain;
  ctx->plan_bytes += bb.total + plan->long_bytes;
  ctx->batch->plans.insert(plan);
  *out = plan;
  return FCS_OK;
}

// Device work only: capturable into a CUDA graph.
int plan_launch(fcs_ctx *ctx, const fcs_batch_plan *plan) {
  if (ctx->spec_cache)
    for (const auto &o : plan->outs) spec_cache_invalidate(ctx, o.first, o.second);
  // The first long problem on the P = 2^15 warp-DIT route has its accumulator
  // cleared before the chain and its kernel launched as a programmatic
  // dependent of the chain's last class, so its CTAs take the SMs the chain
  // frees while it drains.  The other long problems share the scratch and
  // run one after another afterwards.
  bool split = false;
  auto long_call = [&](const fcs_cp_problem &p, int stage, bool *sp) -> int {
    Modes m{};
    int rc = make_modes(ctx, p.N, p.I, p.J, p.ldh, &m);
    if (rc) return rc;
    return big_sketch_cp(ctx, m, p.R, p.D, p.U, p.ldU, p.lambda, p.h, p.s, p.out,
                         ilog2_ceil(m.Jt), plan->long_ws, plan->long_bytes, stage, sp);
  };
  if (plan->dev && !plan->longp.empty()) {
    int rc = long_call(plan->longp[0], 1, &split);
    if (rc) return rc;
  }
  if (plan->dev) {
    int rc = batch_issue(ctx, static_cast<char *>(plan->dev), plan->build);
    if (rc) return rc;
  }
  for (size_t k = 0; k < plan->longp.size(); ++k) {
    int rc = long_call(plan->longp[k], k == 0 && split ? 2 : 0, nullptr);
    if (rc) return rc;
  }
  return FCS_OK;
}

void plan_free(fcs_batch_plan *plan) {
  if (!plan) return;
  if (plan->owner) {
    plan->owner->plan_bytes -= plan->bytes + plan->long_bytes;
    if (plan->owner->batch) plan->owner->batch->plans.erase(plan);
  }
  if (plan->dev) cudaFree(plan->dev);
  if (plan->long_ws) cudaFree(plan->long_ws);
  delete plan;
}

// The autotuned entry of this batch shape, or null.
const std::pair<int, std::vector<ClassCfg>> *tuned_entry(fcs_ctx *ctx, int nprob,
                                                         const fcs_cp_problem *q) {
  std::vector<HostProb> hp(nprob);
  for (int k = 0; k < nprob; ++k)
    if (check_problem(ctx, k, q[k], &hp[k]) != FCS_OK) return nullptr;
  auto it = ctx->batch->tuned.find(batch_signature(nprob, hp, q));
  return it != ctx->batch->tuned.end() ? &it->second : nullptr;
}

// Device time of `reps` launches of a plan after one warm-up (ms, summed).
int time_plan(fcs_ctx *ctx, fcs_batch_plan *plan, cudaEvent_t e0, cudaEvent_t e1, int reps,
              float *ms_out) {
  int rc = plan_launch(ctx, plan);
  float total = 0.f;
  for (int rep = 0; rep < reps && rc == FCS_OK; ++rep) {
    cudaEventRecord(e0, ctx->stream);
    rc = plan_launch(ctx, plan);
    cudaEventRecord(e1, ctx->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    total += ms;
  }
  cudaStreamSynchronize(ctx->stream);
  *ms_out = total;
  return rc;
}

}  // namespace
}  // namespace fcs

using namespace fcs;

namespace fcs {
void batch_state_destroy(fcs_ctx *ctx) {
  if (ctx && ctx->batch) {
    // plans outlive their context only as device memory: a later
    // fcs_batch_plan_destroy must not touch the context
    for (fcs_batch_plan *p : ctx->batch->plans) p->owner = nullptr;
    delete ctx->batch;
    ctx->batch = nullptr;
  }
}
}  // namespace fcs

static int ensure_batch_state(fcs_ctx *ctx) {
  if (!ctx->batch) {
    ctx->batch = new (std::nothrow) fcs_batch_state();
    if (!ctx->batch) return set_error(ctx, FCS_ENOMEM_BUDGET, "out of host memory");
  }
  load_cache(*ctx->batch);
  return FCS_OK;
}

extern "C" int fcs_batch_plan_create(fcs_ctx *ctx, int nprob, const fcs_cp_problem *host_probs,
                                     int grain, fcs_batch_plan **plan) {
  if (!ctx || !plan) return FCS_EINVAL;
  *plan = nullptr;
  ctx->err.clear();
  if (nprob < 1 || !host_probs) return set_error(ctx, FCS_EINVAL, "empty batch");
  int rc = ensure_batch_state(ctx);
  if (rc) return rc;
  DeviceGuard g(ctx->device);
  // the autotuned shape of this batch (grain and class shapes), if any
  const auto *t = tuned_entry(ctx, nprob, host_probs);
  if (grain < 1) grain = t ? t->first : default_grain(ctx, nprob, host_probs);
  return plan_create(ctx, nprob, host_probs, grain, plan, t ? &t->second : nullptr);
}

extern "C" int fcs_batch_plan_create_cfg(fcs_ctx *ctx, int nprob,
                                         const fcs_cp_problem *host_probs, int grain, int ncfg,
                                         const fcs_batch_class_cfg *host_cfg,
                                         fcs_batch_plan **plan) {
  if (!ctx || !plan) return FCS_EINVAL;
  *plan = nullptr;
  ctx->err.clear();
  if (nprob < 1 || !host_probs) return set_error(ctx, FCS_EINVAL, "empty batch");
  if (ncfg < 0 || (ncfg > 0 && !host_cfg)) return set_error(ctx, FCS_EINVAL, "bad class list");
  std::vector<ClassCfg> cfg;
  for (int c = 0; c < ncfg; ++c) {
    const fcs_batch_class_cfg &x = host_cfg[c];
    const int L = ilog2_ceil(x.fft_len) - 1;
    if (x.fft_len < 16 || x.fft_len > (1 << kMaxLog2P) || (x.fft_len & (x.fft_len - 1)))
      return set_error(ctx, FCS_EINVAL, "class %d: fft_len %d is not a power of two in [16, %d]",
                       c, x.fft_len, 1 << kMaxLog2P);
    const int eng_ok = L == wdit::kL ? x.engine == 1 : L == 12 ? (x.engine == 0 || x.engine == 1)
                                                               : x.engine == 0;
    if (!eng_ok)
      return set_error(ctx, FCS_EINVAL, "class %d: engine %d not available for P = %d", c,
                       x.engine, x.fft_len);
    if (x.thread_mult != 1 && !(x.thread_mult == 2 && x.engine == 0))
      return set_error(ctx, FCS_EINVAL, "class %d: thread_mult %d not available", c,
                       x.thread_mult);
    if (x.items_per_cta != 1 && x.items_per_cta != 2 && x.items_per_cta != 4)
      return set_error(ctx, FCS_EINVAL, "class %d: items_per_cta %d not in {1,2,4}", c,
                       x.items_per_cta);
    cfg.push_back(ClassCfg{L, x.thread_mult, x.items_per_cta, x.engine});
  }
  int rc = ensure_batch_state(ctx);
  if (rc) return rc;
  DeviceGuard g(ctx->device);
  if (grain < 1) grain = default_grain(ctx, nprob, host_probs);
  return plan_create(ctx, nprob, host_probs, grain, plan, &cfg);
}

extern "C" int fcs_batch_plan_config(const fcs_batch_plan *plan, int *host_grain, int max_cfg,
                                     fcs_batch_class_cfg *host_cfg, int *host_ncfg) {
  if (!plan || !host_ncfg || (max_cfg > 0 && !host_cfg)) return FCS_EINVAL;
  const auto &cls = plan->build.classes;
  *host_ncfg = int(cls.size());
  if (host_grain) *host_grain = plan->grain;
  for (int c = 0; c < int(cls.size()) && c < max_cfg; ++c)
    host_cfg[c] = fcs_batch_class_cfg{2 << cls[c].L, cls[c].eng, cls[c].ntm, cls[c].ipc, cls[c].nt};
  return FCS_OK;
}

extern "C" int fcs_batch_plan_launch(fcs_ctx *ctx, const fcs_batch_plan *plan) {
  if (!ctx || !plan) return FCS_EINVAL;
  ctx->err.clear();
  if (plan->owner != ctx) return set_error(ctx, FCS_EINVAL, "plan belongs to another context");
  DeviceGuard g(ctx->device);
  return plan_launch(ctx, plan);
}

extern "C" int fcs_batch_plan_destroy(fcs_batch_plan *plan) {
  if (!plan) return FCS_OK;
  DeviceGuard g(plan->device);
  if (plan->owner)
    cudaStreamSynchronize(plan->owner->stream);
  else
    cudaDeviceSynchronize();           // the context is gone: wait for any user of the plan
  plan_free(plan);
  return FCS_OK;
}

extern "C" int fcs_batch_sketch_cp(fcs_ctx *ctx, int nprob, const fcs_cp_problem *host_probs,
                                   int grain) {
  fcs_batch_plan *plan = nullptr;
  int rc = fcs_batch_plan_create(ctx, nprob, host_probs, grain, &plan);
  if (rc) return rc;
  DeviceGuard g(ctx->device);
  rc = plan_launch(ctx, plan);
  cudaStreamSynchronize(ctx->stream);   // the plan's memory is released below
  plan_free(plan);
  return rc;
}

extern "C" int fcs_batch_autotune(fcs_ctx *ctx, int nprob, const fcs_cp_problem *host_probs,
                                  int *host_best_grain) {
  if (!ctx) return FCS_EINVAL;
  ctx->err.clear();
  if (nprob < 1 || !host_probs) return set_error(ctx, FCS_EINVAL, "empty batch");
  int rc = ensure_batch_state(ctx);
  if (rc) return rc;
  DeviceGuard g(ctx->device);
  std::vector<HostProb> hp(nprob);
  int64_t rmax = 1;
  std::set<int> sizes;                       // FFT-size classes of the batch kernels
  for (int k = 0; k < nprob; ++k) {
    rc = check_problem(ctx, k, host_probs[k], &hp[k]);
    if (rc) return rc;
    rmax = std::max<int64_t>(rmax, hp[k].R);
    if (!hp[k].longp) sizes.insert(hp[k].L);
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return set_error(ctx, FCS_ECUDA, "cudaEventCreate");
  // the whole batch timed on the device for each candidate
  auto timed = [&](int grain, const std::vector<ClassCfg> &cfg, float *ms) -> int {
    fcs_batch_plan *plan = nullptr;
    int r = plan_create(ctx, nprob, host_probs, grain, &plan, &cfg);
    if (r) return r;
    r = time_plan(ctx, plan, e0, e1, 3, ms);
    plan_free(plan);
    return r;
  };
  // 1. ranks per item, every class at its default shape
  std::vector<ClassCfg> cfg;
  for (int L : sizes) cfg.push_back(ClassCfg{L, 1, 1, default_engine(L)});
  int best = 1;
  float best_ms = 1e30f;
  for (int grain = 1; grain <= 64 && grain < 2 * rmax && rc == FCS_OK; grain *= 2) {
    float ms = 0.f;
    rc = timed(grain, cfg, &ms);
    if (rc == FCS_OK && ms < best_ms) {
      best_ms = ms;
      best = grain;
    }
  }
  // 2. per class, threads per transform and items per CTA, the other
  //    classes held at their best so far (one sweep, largest FFT first); a
  //    shape replaces the current one only if it is at least 3 % faster
  for (auto c = cfg.rbegin(); c != cfg.rend() && rc == FCS_OK; ++c) {
    const ClassCfg keep = *c;
    ClassCfg bestc = keep;
    // shapes (engine, threads): slot FFT at 1 or 2 x the threads; for
    // P = 8192 also the warp-DIT engine; P = 16384 has only warp-DIT
    std::vector<std::pair<int, int>> shapes;
    if (c->L == wdit::kL) {
      shapes = {{1, 1}};
    } else {
      shapes = {{0, 1}, {0, 2}};
      if (c->L == 12) shapes.push_back({1, 1});
    }
    for (const auto &sh : shapes) {
      for (int ipc : {1, 2, 4}) {
        if (sh.first == keep.eng && sh.second == keep.ntm && ipc == keep.ipc) continue;
        c->eng = sh.first;
        c->ntm = sh.second;
        c->ipc = ipc;
        float ms = 0.f;
        rc = timed(best, cfg, &ms);
        if (rc) break;
        if (ms < 0.97f * best_ms) {              // a clear gain, not timing noise
          best_ms = ms;
          bestc = *c;
        }
      }
      if (rc) break;
    }
    *c = bestc;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  ctx->batch->tuned[batch_signature(nprob, hp, host_probs)] = {best, cfg};
  save_cache(*ctx->batch);
  if (host_best_grain) *host_best_grain = best;
  return FCS_OK;
}
