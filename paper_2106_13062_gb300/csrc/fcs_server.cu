// fcs_server.cu -- a request server with continuous batching over the sketch
// path (CP-route sketches, eq. FCS_syn; contractions against resident
// sketches, eqs. T_uvw / T_Ivw).  No counterpart in the paper: this is the
// serving layer.
//
// Clients submit requests from any host thread; a scheduler thread owns the
// GPU work.  Its loop:
//   1. completes rounds whose CUDA event has fired (copies results out of the
//      pinned staging area, frees device memory and slots, records latency);
//   2. when a stream is free, admits queued requests in FIFO order while
//      in-flight slots, device arena memory and pinned staging memory allow,
//      and issues them as one round on that stream: host->device copies,
//      hash generation, ONE batched launch chain for all admitted CP
//      requests (fcs_batch building blocks), the contractions, and
//      device->host copies, closed by an event;
//   3. otherwise sleeps on a condition variable (woken by submit) for at most
//      100 us.
// Several rounds run at once on different streams, so requests that arrive
// while others are on the GPU are admitted as soon as slots and memory free
// up and their work overlaps with the running rounds on the device.  Sketches
// can be kept resident (with their hash tables) for later contraction
// requests.  Every host wait is bounded; nothing on the device waits.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "fcs_batch_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0, Clock::time_point t) {
  return std::chrono::duration<double>(t - t0).count();
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// First-fit allocator over [0, cap) with coalescing; offsets 256-aligned.
class Arena {
 public:
  void init(size_t cap) {
    cap_ = cap;
    free_.clear();
    if (cap) free_[0] = cap;
  }
  size_t capacity() const { return cap_; }
  bool alloc(size_t bytes, size_t *off) {
    bytes = up256(std::max<size_t>(bytes, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = up256(std::max<size_t>(bytes, 1));
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  size_t cap_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;
};

struct Resident {
  int64_t id = 0;
  int N = 0, D = 0;
  int64_t I[8] = {};
  int32_t J[8] = {};
  int64_t Jt = 0;
  size_t off = 0, bytes = 0;   // device arena block: h | s | sketch
  int32_t *h = nullptr;
  int8_t *s = nullptr;
  float *sketch = nullptr;
  int refs = 0;
  bool released = false;
};

enum State { kQueued, kRunning, kDone, kFailed, kCancelled };

struct Req {
  int64_t ticket = 0;
  fcs_request r{};
  State state = kQueued;
  int status = FCS_OK;
  Clock::time_point t_submit, t_done;
  int64_t Jt = 0, width = 0;          // CP: sketch length; contraction: result width
  size_t dev_bytes = 0, pin_bytes = 0, keep_bytes = 0;
  size_t dev_off = 0, pin_off = 0;
  Resident *res = nullptr;            // contraction target / CP sketch kept
  int64_t sketch_id = 0;
  // device and pinned views for the round
  float *dU[8] = {}, *dlam = nullptr, *dout = nullptr, *dvec[8] = {}, *dres = nullptr;
  int32_t *dh = nullptr;
  int8_t *ds = nullptr;
  char *pin = nullptr;
};

struct Round {
  int stream = -1;
  cudaEvent_t done = nullptr;
  std::vector<Req *> reqs;
  size_t plan_off = 0, plan_bytes = 0;   // device arena block for the batch
  size_t pin_off = 0, pin_bytes = 0;     // pinned block for descriptors
  bool busy = false;
  int status = FCS_OK;
  int batch_launches = 0;                // kernels of the round's batched CP launch
};

int64_t jtilde_of(int N, const int32_t *J) {
  int64_t t = 1;
  for (int n = 0; n < N; ++n) t += int64_t(J[n]) - 1;
  return t;
}

}  // namespace

struct fcs_server {
  fcs_server_config cfg{};
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::vector<fcs_ctx *> ctxs;          // one context per stream
  std::vector<Round> rounds;            // one round slot per stream
  char *dbase = nullptr;
  char *pbase = nullptr;
  Arena darena, parena;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req *> queue;
  std::map<int64_t, std::unique_ptr<Req>> reqs;
  std::map<int64_t, std::unique_ptr<Resident>> residents;
  int64_t next_ticket = 1, next_sketch = 1;
  int inflight = 0, max_inflight_seen = 0;
  bool stop = false;
  std::thread worker;
  // statistics
  std::vector<double> lat;
  int64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, nrounds = 0, sketches = 0;
  int64_t batch_launches = 0;
  Clock::time_point t_first, t_last;
  bool any_submit = false;
};

namespace {

// Device and pinned bytes one request needs while it runs, and device bytes
// it keeps afterwards (resident sketch).
void request_sizes(Req *q) {
  const fcs_request &r = q->r;
  size_t dev = 0, pin = 0, keep = 0;
  if (r.kind == FCS_REQ_CP) {
    int64_t tot = 0;
    for (int n = 0; n < r.N; ++n) {
      dev += up256(sizeof(float) * size_t(r.I[n]) * size_t(r.R));
      pin += up256(sizeof(float) * size_t(r.I[n]) * size_t(r.R));
      tot += r.I[n];
    }
    dev += up256(sizeof(float) * size_t(r.R));
    pin += up256(sizeof(float) * size_t(r.R));
    q->Jt = jtilde_of(r.N, r.J);
    const size_t tabs = up256(size_t(r.D) * size_t(tot) * 4) + up256(size_t(r.D) * size_t(tot));
    const size_t sk = up256(sizeof(float) * size_t(r.D) * size_t(q->Jt));
    if (r.keep_resident)
      keep = tabs + sk;
    else
      dev += tabs + sk;
    pin += sk;
  } else {
    for (int n = 0; n < r.N; ++n) {
      dev += up256(sizeof(float) * size_t(r.B) * size_t(r.I[n]));
      pin += up256(sizeof(float) * size_t(r.B) * size_t(r.I[n]));
    }
    q->width = r.contract_kind == FCS_CONTRACT_ALL ? 1 : r.I[r.free_mode];
    dev += up256(sizeof(float) * size_t(r.B) * size_t(q->width));
    pin += up256(sizeof(float) * size_t(r.B) * size_t(q->width));
  }
  q->dev_bytes = dev;
  q->pin_bytes = pin;
  q->keep_bytes = keep;
}

void finish_request(fcs_server *S, Req *q, int status) {
  q->t_done = Clock::now();
  q->status = status;
  q->state = status == FCS_OK ? kDone : kFailed;
  if (status == FCS_OK) {
    S->completed++;
    S->lat.push_back(seconds_since(q->t_submit, q->t_done));
    if (q->r.kind == FCS_REQ_CP) S->sketches += q->r.D;
  } else {
    S->failed++;
  }
  S->t_last = q->t_done;
}

// Scheduler: complete a finished round (lock held).
void complete_round(fcs_server *S, Round &rd) {
  for (Req *q : rd.reqs) {
    int st = rd.status;
    if (st == FCS_OK) {
      const fcs_request &r = q->r;
      if (r.kind == FCS_REQ_CP) {
        if (r.host_out)
          memcpy(r.host_out, q->pin + (q->pin_bytes - up256(sizeof(float) * r.D * q->Jt)),
                 sizeof(float) * size_t(r.D) * size_t(q->Jt));
      } else {
        const size_t rb = sizeof(float) * size_t(r.B) * size_t(q->width);
        memcpy(r.host_result, q->pin + (q->pin_bytes - up256(rb)), rb);
      }
    }
    if (q->r.kind == FCS_REQ_CP && q->r.keep_resident) {
      if (st != FCS_OK || (q->res->released && q->res->refs == 0)) {
        S->darena.release(q->res->off, q->res->bytes);
        S->residents.erase(q->res->id);
        q->res = nullptr;
      }
    } else if (q->r.kind != FCS_REQ_CP && q->res) {
      Resident *rs = q->res;
      if (--rs->refs == 0 && rs->released) {
        S->darena.release(rs->off, rs->bytes);
        S->residents.erase(rs->id);
      }
    }
    S->darena.release(q->dev_off, q->dev_bytes);
    S->parena.release(q->pin_off, q->pin_bytes);
    S->inflight--;
    finish_request(S, q, st);
  }
  if (rd.plan_bytes) S->darena.release(rd.plan_off, rd.plan_bytes);
  if (rd.pin_bytes) S->parena.release(rd.pin_off, rd.pin_bytes);
  rd.reqs.clear();
  rd.plan_bytes = rd.pin_bytes = 0;
  rd.busy = false;
  rd.status = FCS_OK;
  S->cv_done.notify_all();
}

// Scheduler: admit the head of the queue while resources allow (lock held).
std::vector<Req *> admit(fcs_server *S) {
  std::vector<Req *> got;
  int ncp = 0;
  while (!S->queue.empty()) {
    Req *q = S->queue.front();
    if (q->state == kCancelled) {
      S->queue.pop_front();
      continue;
    }
    if (S->inflight >= S->cfg.max_inflight) break;
    if (q->r.kind == FCS_REQ_CP && ncp >= S->cfg.max_batch) break;
    // a CP request with P > 16384 (multi-kernel long-FFT route) gets a round
    // of its own, so it does not hold back the completion of short requests
    const bool longq = q->r.kind == FCS_REQ_CP && q->Jt > (int64_t(1) << fcs::kMaxLog2P);
    if (longq && !got.empty()) break;
    size_t doff = 0, poff = 0, koff = 0;
    if (!S->darena.alloc(q->dev_bytes, &doff)) break;
    if (!S->parena.alloc(q->pin_bytes, &poff)) {
      S->darena.release(doff, q->dev_bytes);
      break;
    }
    if (q->keep_bytes && !S->darena.alloc(q->keep_bytes, &koff)) {
      S->darena.release(doff, q->dev_bytes);
      S->parena.release(poff, q->pin_bytes);
      break;
    }
    S->queue.pop_front();
    q->dev_off = doff;
    q->pin_off = poff;
    q->pin = S->pbase + poff;
    if (q->keep_bytes) {
      auto rs = std::make_unique<Resident>();
      rs->id = q->sketch_id;
      rs->N = q->r.N;
      rs->D = q->r.D;
      for (int n = 0; n < q->r.N; ++n) {
        rs->I[n] = q->r.I[n];
        rs->J[n] = q->r.J[n];
      }
      rs->Jt = q->Jt;
      rs->off = koff;
      rs->bytes = q->keep_bytes;
      q->res = rs.get();
      S->residents[rs->id] = std::move(rs);
    }
    if (q->r.kind == FCS_REQ_CP) ncp++;
    q->state = kRunning;
    S->inflight++;
    S->max_inflight_seen = std::max(S->max_inflight_seen, S->inflight);
    got.push_back(q);
    if (longq) break;
  }
  return got;
}

// Scheduler: issue one round on stream `si` (lock NOT held for GPU work).
int issue_round(fcs_server *S, int si, std::vector<Req *> &reqs, Round &rd) {
  fcs_ctx *ctx = S->ctxs[si];
  cudaStream_t st = S->streams[si];
  std::vector<fcs_cp_problem> probs;
  std::vector<Req *> cps;
  for (Req *q : reqs) {
    const fcs_request &r = q->r;
    char *dv = S->dbase + q->dev_off;
    char *pn = q->pin;
    size_t dpos = 0, ppos = 0;
    if (r.kind == FCS_REQ_CP) {
      int64_t tot = 0;
      for (int n = 0; n < r.N; ++n) {
        const size_t b = sizeof(float) * size_t(r.I[n]) * size_t(r.R);
        memcpy(pn + ppos, r.host_U[n], b);
        q->dU[n] = reinterpret_cast<float *>(dv + dpos);
        if (cudaMemcpyAsync(q->dU[n], pn + ppos, b, cudaMemcpyHostToDevice, st) != cudaSuccess)
          return FCS_ECUDA;
        dpos += up256(b);
        ppos += up256(b);
        tot += r.I[n];
      }
      const size_t lb = sizeof(float) * size_t(r.R);
      q->dlam = reinterpret_cast<float *>(dv + dpos);
      if (r.host_lambda) {
        memcpy(pn + ppos, r.host_lambda, lb);
        if (cudaMemcpyAsync(q->dlam, pn + ppos, lb, cudaMemcpyHostToDevice, st) != cudaSuccess)
          return FCS_ECUDA;
      } else {
        q->dlam = nullptr;
      }
      dpos += up256(lb);
      ppos += up256(lb);
      char *tb = r.keep_resident ? S->dbase + q->res->off : dv + dpos;
      q->dh = reinterpret_cast<int32_t *>(tb);
      q->ds = reinterpret_cast<int8_t *>(tb + up256(size_t(r.D) * size_t(tot) * 4));
      q->dout = reinterpret_cast<float *>(tb + up256(size_t(r.D) * size_t(tot) * 4) +
                                          up256(size_t(r.D) * size_t(tot)));
      if (r.keep_resident) {
        q->res->h = q->dh;
        q->res->s = q->ds;
        q->res->sketch = q->dout;
      }
      int rc = fcs_make_hashes(ctx, r.seed, r.N, r.I, r.J, r.D, q->dh, q->ds);
      if (rc) return rc;
      fcs_cp_problem p{};
      p.N = r.N;
      p.D = r.D;
      p.R = r.R;
      for (int n = 0; n < r.N; ++n) {
        p.I[n] = r.I[n];
        p.J[n] = r.J[n];
        p.U[n] = q->dU[n];
        p.ldU[n] = r.R;
      }
      p.lambda = q->dlam;
      p.h = q->dh;
      p.s = q->ds;
      p.ldh = 0;
      p.out = q->dout;
      if (q->Jt > (int64_t(1) << fcs::kMaxLog2P)) {
        // too long for the batch kernels: its own (multi-kernel) launch
        rc = fcs_sketch_cp(ctx, p.N, p.I, p.J, p.R, p.D, p.U, p.ldU, p.lambda, p.h, p.s, p.ldh,
                           p.out);
        if (rc) return rc;
      } else {
        probs.push_back(p);
      }
      cps.push_back(q);
    } else {
      for (int n = 0; n < r.N; ++n) {
        q->dvec[n] = nullptr;
        if (r.contract_kind == FCS_CONTRACT_FREE && n == r.free_mode) continue;
        const size_t b = sizeof(float) * size_t(r.B) * size_t(r.I[n]);
        memcpy(pn + ppos, r.host_vecs[n], b);
        q->dvec[n] = reinterpret_cast<float *>(dv + dpos);
        if (cudaMemcpyAsync(q->dvec[n], pn + ppos, b, cudaMemcpyHostToDevice, st) != cudaSuccess)
          return FCS_ECUDA;
        dpos += up256(b);
        ppos += up256(b);
      }
      q->dres = reinterpret_cast<float *>(dv + dpos);
    }
  }
  // one batched launch for every CP request of the round
  if (!probs.empty()) {
    const int grain = fcs::batch_default_grain(ctx, int(probs.size()), probs.data());
    fcs::BatchBuild bb{};
    std::vector<char> desc;
    int rc = fcs::batch_build(ctx, int(probs.size()), probs.data(), grain, nullptr, &desc, &bb);
    if (rc) return rc;
    bool planned = false;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (S->darena.alloc(bb.total, &rd.plan_off)) {
        if (S->parena.alloc(bb.desc_bytes, &rd.pin_off)) {
          rd.plan_bytes = bb.total;
          rd.pin_bytes = bb.desc_bytes;
          planned = true;
        } else {
          S->darena.release(rd.plan_off, bb.total);
        }
      }
    }
    if (planned) {
      char *pb = S->dbase + rd.plan_off;
      rc = fcs::batch_build(ctx, int(probs.size()), probs.data(), grain, pb, &desc, &bb);
      if (rc) return rc;
      memcpy(S->pbase + rd.pin_off, desc.data(), desc.size());
      if (cudaMemcpyAsync(pb, S->pbase + rd.pin_off, desc.size(), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
        return FCS_ECUDA;
      rc = fcs::batch_issue(ctx, pb, bb);
      if (rc) return rc;
      rd.batch_launches = 1 + int(bb.classes.size());
    } else {
      // no room for a batch plan right now: one launch per request instead
      for (const fcs_cp_problem &p : probs) {
        rc = fcs_sketch_cp(ctx, p.N, p.I, p.J, p.R, p.D, p.U, p.ldU, p.lambda, p.h, p.s, p.ldh,
                           p.out);
        if (rc) return rc;
      }
    }
  }
  // contractions against resident sketches
  for (Req *q : reqs) {
    const fcs_request &r = q->r;
    if (r.kind == FCS_REQ_CP) continue;
    Resident *rs = q->res;
    int rc = fcs_contract(ctx, r.contract_kind, r.free_mode, rs->N, rs->I, rs->J, rs->D,
                          rs->sketch, r.B, q->dvec, rs->h, rs->s, 0, q->dres, nullptr);
    if (rc) return rc;
  }
  // results back to pinned staging
  for (Req *q : reqs) {
    const fcs_request &r = q->r;
    if (r.kind == FCS_REQ_CP) {
      if (!r.host_out) continue;
      const size_t b = sizeof(float) * size_t(r.D) * size_t(q->Jt);
      if (cudaMemcpyAsync(q->pin + (q->pin_bytes - up256(b)), q->dout, b, cudaMemcpyDeviceToHost,
                          st) != cudaSuccess)
        return FCS_ECUDA;
    } else {
      const size_t b = sizeof(float) * size_t(r.B) * size_t(q->width);
      if (cudaMemcpyAsync(q->pin + (q->pin_bytes - up256(b)), q->dres, b, cudaMemcpyDeviceToHost,
                          st) != cudaSuccess)
        return FCS_ECUDA;
    }
  }
  return FCS_OK;
}

void worker_loop(fcs_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool progress = false;
    // 1. completions
    for (Round &rd : S->rounds) {
      if (rd.busy) {
        cudaError_t e = cudaEventQuery(rd.done);
        if (e == cudaSuccess) {
          complete_round(S, rd);
          progress = true;
        } else if (e != cudaErrorNotReady) {
          cudaGetLastError();
          rd.status = FCS_ECUDA;
          complete_round(S, rd);
          progress = true;
        }
      }
    }
    const bool any_busy = std::any_of(S->rounds.begin(), S->rounds.end(),
                                      [](const Round &r) { return r.busy; });
    if (S->stop && !any_busy) break;
    // 2. a new round on a free stream
    if (!S->stop) {
      int si = -1;
      for (int k = 0; k < int(S->rounds.size()); ++k)
        if (!S->rounds[k].busy) {
          si = k;
          break;
        }
      if (si >= 0 && !S->queue.empty()) {
        std::vector<Req *> got = admit(S);
        if (!got.empty()) {
          Round &rd = S->rounds[si];
          rd.busy = true;
          rd.reqs = got;
          rd.status = FCS_OK;
          rd.batch_launches = 0;
          S->nrounds++;
          lk.unlock();
          int rc = issue_round(S, si, got, rd);
          cudaEventRecord(rd.done, S->streams[si]);
          lk.lock();
          S->batch_launches += rd.batch_launches;
          if (rc != FCS_OK) rd.status = rc;
          progress = true;
        }
      }
    }
    if (!progress) S->cv_work.wait_for(lk, std::chrono::microseconds(100));
  }
  // stopping: whatever is still queued is cancelled
  while (!S->queue.empty()) {
    Req *q = S->queue.front();
    S->queue.pop_front();
    if (q->state == kQueued) {
      q->state = kCancelled;
      q->status = FCS_ETIMEOUT;
      S->cancelled++;
    }
  }
  S->cv_done.notify_all();
}

int validate(const fcs_server *S, const fcs_request &r) {
  if (r.kind != FCS_REQ_CP && r.kind != FCS_REQ_CONTRACT) return FCS_EINVAL;
  if (r.N < 1 || r.N > 8) return FCS_EINVAL;
  for (int n = 0; n < r.N; ++n)
    if (r.I[n] < 1 || r.J[n] < 1) return FCS_EINVAL;
  if (r.kind == FCS_REQ_CP) {
    if (r.D < 1 || r.D > 16 || r.R < 1) return FCS_EINVAL;
    for (int n = 0; n < r.N; ++n)
      if (!r.host_U[n]) return FCS_EINVAL;
    if (!r.host_out && !r.keep_resident) return FCS_EINVAL;
    int l = 0;
    while ((int64_t(1) << l) < jtilde_of(r.N, r.J)) ++l;
    if (l > fcs::kMaxLog2PBig) return FCS_EUNSUPPORTED;
  } else {
    if (r.B < 1 || r.B > 65535 || !r.host_result) return FCS_EINVAL;
    if (r.contract_kind != FCS_CONTRACT_ALL && r.contract_kind != FCS_CONTRACT_FREE)
      return FCS_EINVAL;
    if (r.contract_kind == FCS_CONTRACT_FREE && (r.free_mode < 0 || r.free_mode >= r.N))
      return FCS_EINVAL;
    for (int n = 0; n < r.N; ++n)
      if (!r.host_vecs[n] && !(r.contract_kind == FCS_CONTRACT_FREE && n == r.free_mode))
        return FCS_EINVAL;
  }
  (void)S;
  return FCS_OK;
}

}  // namespace

using namespace fcs;

extern "C" int fcs_server_create(const fcs_server_config *cfg, fcs_server **out) {
  if (!cfg || !out) return FCS_EINVAL;
  *out = nullptr;
  if (cfg->streams < 1 || cfg->streams > 8 || cfg->max_inflight < 1 || cfg->max_batch < 1)
    return FCS_EINVAL;
  auto S = std::make_unique<fcs_server>();
  S->cfg = *cfg;
  S->device = cfg->device;
  DeviceGuard g(cfg->device);
  if (cfg->arena_bytes) {
    if (cudaMalloc(&S->dbase, cfg->arena_bytes) != cudaSuccess) {
      cudaGetLastError();
      return FCS_ENOMEM_BUDGET;
    }
  }
  if (cfg->staging_bytes) {
    if (cudaHostAlloc(reinterpret_cast<void **>(&S->pbase), cfg->staging_bytes,
                      cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      if (S->dbase) cudaFree(S->dbase);
      return FCS_ENOMEM_BUDGET;
    }
  }
  S->darena.init(cfg->arena_bytes);
  S->parena.init(cfg->staging_bytes);
  S->streams.resize(cfg->streams);
  S->ctxs.resize(cfg->streams, nullptr);
  S->rounds.resize(cfg->streams);
  for (int k = 0; k < cfg->streams; ++k) {
    cudaStreamCreateWithFlags(&S->streams[k], cudaStreamNonBlocking);
    int rc = fcs_create(&S->ctxs[k], cfg->device, S->streams[k], cfg->workspace_bytes);
    if (rc) {
      for (int j = 0; j <= k; ++j) {
        if (S->ctxs[j]) fcs_destroy(S->ctxs[j]);
        cudaStreamDestroy(S->streams[j]);
      }
      if (S->dbase) cudaFree(S->dbase);
      if (S->pbase) cudaFreeHost(S->pbase);
      return rc;
    }
    cudaEventCreateWithFlags(&S->rounds[k].done, cudaEventDisableTiming);
    S->rounds[k].stream = k;
  }
  fcs_server *raw = S.release();
  raw->worker = std::thread(worker_loop, raw);
  *out = raw;
  return FCS_OK;
}

extern "C" int fcs_server_destroy(fcs_server *S) {
  if (!S) return FCS_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  DeviceGuard g(S->device);
  for (size_t k = 0; k < S->streams.size(); ++k) {
    cudaStreamSynchronize(S->streams[k]);
    cudaEventDestroy(S->rounds[k].done);
    fcs_destroy(S->ctxs[k]);
    cudaStreamDestroy(S->streams[k]);
  }
  if (S->dbase) cudaFree(S->dbase);
  if (S->pbase) cudaFreeHost(S->pbase);
  delete S;
  return FCS_OK;
}

extern "C" int fcs_server_submit(fcs_server *S, const fcs_request *r, int64_t *ticket) {
  if (!S || !r || !ticket) return FCS_EINVAL;
  int rc = validate(S, *r);
  if (rc) return rc;
  auto q = std::make_unique<Req>();
  q->r = *r;
  request_sizes(q.get());
  if (q->dev_bytes + q->keep_bytes > S->darena.capacity() ||
      q->pin_bytes > S->parena.capacity())
    return FCS_ENOMEM_BUDGET;          // could never be admitted
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return FCS_EINVAL;
  if (r->kind == FCS_REQ_CONTRACT) {
    auto it = S->residents.find(r->sketch_id);
    if (it == S->residents.end() || it->second->released) return FCS_EINVAL;
    Resident *rs = it->second.get();
    if (rs->N != r->N) return FCS_EINVAL;
    for (int n = 0; n < r->N; ++n)
      if (rs->I[n] != r->I[n] || rs->J[n] != r->J[n]) return FCS_EINVAL;
    rs->refs++;
    q->res = rs;
  }
  q->ticket = S->next_ticket++;
  if (r->kind == FCS_REQ_CP && r->keep_resident) q->sketch_id = S->next_sketch++;
  q->t_submit = Clock::now();
  if (!S->any_submit) {
    S->t_first = q->t_submit;
    S->any_submit = true;
  }
  S->submitted++;
  *ticket = q->ticket;
  S->queue.push_back(q.get());
  S->reqs[q->ticket] = std::move(q);
  S->cv_work.notify_one();
  return FCS_OK;
}

static int fill_result(fcs_server *S, Req *q, fcs_result *res) {
  res->ticket = q->ticket;
  res->state = q->state == kDone ? 2 : q->state == kFailed ? 3 : q->state == kCancelled ? 4
               : q->state == kRunning ? 1 : 0;
  res->status = q->status;
  res->sketch_id = q->sketch_id;
  res->latency_s = (q->state == kDone || q->state == kFailed)
                       ? seconds_since(q->t_submit, q->t_done) : -1.0;
  (void)S;
  return FCS_OK;
}

extern "C" int fcs_server_poll(fcs_server *S, int64_t ticket, fcs_result *res) {
  if (!S || !res) return FCS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return FCS_EINVAL;
  return fill_result(S, it->second.get(), res);
}

extern "C" int fcs_server_wait(fcs_server *S, int64_t ticket, double timeout_s,
                               fcs_result *res) {
  if (!S || !res) return FCS_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return FCS_EINVAL;
  Req *q = it->second.get();
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s));
  while (q->state == kQueued || q->state == kRunning) {
    if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
        (q->state == kQueued || q->state == kRunning)) {
      fill_result(S, q, res);
      return FCS_ETIMEOUT;
    }
  }
  return fill_result(S, q, res);
}

extern "C" int fcs_server_cancel(fcs_server *S, int64_t ticket) {
  if (!S) return FCS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return FCS_EINVAL;
  Req *q = it->second.get();
  if (q->state != kQueued) return FCS_EINVAL;     // already admitted
  q->state = kCancelled;
  q->status = FCS_ETIMEOUT;
  if (q->res && q->r.kind == FCS_REQ_CONTRACT) {
    Resident *rs = q->res;
    if (--rs->refs == 0 && rs->released) {
      S->darena.release(rs->off, rs->bytes);
      S->residents.erase(rs->id);
    }
  }
  q->res = nullptr;
  S->cancelled++;
  S->cv_done.notify_all();
  return FCS_OK;
}

extern "C" int fcs_server_release(fcs_server *S, int64_t sketch_id) {
  if (!S) return FCS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->residents.find(sketch_id);
  if (it == S->residents.end() || it->second->released) return FCS_EINVAL;
  Resident *rs = it->second.get();
  rs->released = true;
  // still being produced or read: freed by the last round that uses it
  bool producing = false;
  for (auto &kv : S->reqs)
    if (kv.second->res == rs && kv.second->r.kind == FCS_REQ_CP &&
        (kv.second->state == kQueued || kv.second->state == kRunning))
      producing = true;
  if (rs->refs == 0 && !producing) {
    S->darena.release(rs->off, rs->bytes);
    S->residents.erase(it);
  }
  return FCS_OK;
}

extern "C" int fcs_server_stats(fcs_server *S, fcs_stats *out) {
  if (!S || !out) return FCS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->cancelled = S->cancelled;
  out->rounds = S->nrounds;
  out->batch_launches = S->batch_launches;
  out->sketches = S->sketches;
  out->max_inflight_seen = S->max_inflight_seen;
  out->arena_used = S->darena.used();
  if (!S->lat.empty()) {
    std::vector<double> v = S->lat;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
      const size_t k = std::min(v.size() - 1, size_t(p * double(v.size() - 1) + 0.5));
      return v[k];
    };
    out->p50_latency_s = pct(0.50);
    out->p99_latency_s = pct(0.99);
    double sum = 0.0;
    for (double x : v) sum += x;
    out->mean_latency_s = sum / double(v.size());
  }
  if (S->any_submit && S->completed) out->busy_s = seconds_since(S->t_first, S->t_last);
  return FCS_OK;
}

extern "C" int fcs_server_reset_stats(fcs_server *S) {
  if (!S) return FCS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  S->lat.clear();
  S->submitted = S->completed = S->failed = S->cancelled = S->nrounds = S->sketches = 0;
  S->batch_launches = 0;
  S->max_inflight_seen = S->inflight;
  S->any_submit = false;
  return FCS_OK;
}
