// Serving runtime: a persistent request loop with continuous admission and batching.
//
// Requests (one single-RHS solve each, with its own lattice, kappa, tolerance, seeded gauge field
// and source) enter a queue. The scheduler (run by whichever thread submits, waits or finishes a
// job) admits them into execution slots as slots and device memory free up; memory is charged
// against the budget given at creation. Every slot has its own CUDA stream and worker thread, so
// admitted work runs concurrently and its kernels overlap on the device. The oldest waiting
// request is admitted first (or, under the shortest-first policy, the one with the least estimated
// work unless the oldest has waited too long), together with up to max_batch - 1 other requests of the same operator
// (lattice, precision, boundary, iteration limit) when that operator's CG loop is the persistent
// kernel: the slot solves them with cg_solve_batch, one loop launch for all of them per pass, each
// result bitwise the one of its solve alone. A slot keeps the contexts it created (links, Krylov
// workspace, CUDA graphs) resident between requests, so a request whose operator matches an idle
// slot's resident context runs warm: no allocation, no graph rebuild, only wd_set_kappa and the
// new fields. Least recently used residents of idle slots are evicted when new ones do not fit.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/wd.h"

namespace wdk {
void set_last_error(const std::string& msg);
// true when cg_solve_batch shares loop launches for this operator (its CG loop is the persistent kernel)
bool batch_capable(const int dims[4], int precision);
}

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

long long volume_of(const int d[4]) { return (long long)d[0] * d[1] * d[2] * d[3]; }

// Device bytes a context of this precision needs for one solve (gauge copies, vectors, and the
// canonical source and solution buffers of the slot).
size_t request_bytes(const int d[4], int precision) {
  const size_t V = (size_t)volume_of(d);
  const size_t extra = (precision & WD_EVEN_ODD) ? V * 192 * 3 : 0;  // odd-site temporaries
  precision &= ~WD_EVEN_ODD;
  const size_t f64 = V * 192, f32 = V * 96, f16 = V * 52;
  switch (precision) {
    // FP64: + two more p, r buffers of the small-volume loop and the loop's pre-scaled time links
    case WD_PREC_F64: return extra + V * 576 + 11 * f64 + 3 * f64 + (V / 32 + 64) * 8 * 12;
    case WD_PREC_F32: return extra + V * 288 + 6 * f32 + 2 * f64 + V * 12;
    // mixed: + double-float solution, residual, source (3 x 192 B) and links (576 B) per site
    case WD_PREC_MIXED_F32: return extra + V * 576 + V * 192 + 5 * f32 + 3 * f64 + 2 * f64 + V * 12 + V * 1152;
    case WD_PREC_MIXED_F16: return extra + V * 576 + V * 192 + 4 * f16 + f32 + 3 * f64 + 2 * f64 + V * 12 + V * 1152;
  }
  return 0;
}

struct Job {
  long long id;
  wd_request req;
  Clock::time_point t_submit, t_start, t_done;
  wd_result res;
  bool done = false;
  size_t bytes = 0;
  int res_idx = -1;  // the slot resident reserved for it
};

// A context kept on the device between requests, with the slot's source/solution buffers.
struct Resident {
  int dims[4] = {0, 0, 0, 0};
  int bc[4] = {1, 1, 1, -1};  // boundary phases the context was created with
  int precision = 0;
  wd_ctx* ctx = nullptr;
  double* src = nullptr;
  double* x = nullptr;
  size_t bytes = 0;
  unsigned long long last_used = 0;
  bool taken = false;  // reserved for a job of the batch being admitted or running
};

struct Slot {
  int index = 0;
  cudaStream_t stream = nullptr;
  std::vector<Resident> cache;  // resident contexts of this slot (guarded by the server mutex
                                // while the slot is idle; owned by the slot thread while busy)
  std::vector<Job*> batch;      // the jobs it runs; empty = idle
  std::thread th;
};

// The boundary phases a request asks for (wd_request.boundary_set = 0 means (1, 1, 1, -1)).
void request_bc(const wd_request& q, int (&bc)[4]) {
  const int def[4] = {1, 1, 1, -1};
  for (int i = 0; i < 4; ++i) bc[i] = q.boundary_set ? q.boundary[i] : def[i];
}

// A resident context (or the placeholder reserved for one) serves a request only when the operator
// is the same: volume, precision and boundary phases (kappa is set per request).
bool same_operator(const Resident& r, const wd_request& q) {
  int bc[4];
  request_bc(q, bc);
  return r.precision == q.precision && memcmp(r.dims, q.dims, sizeof(r.dims)) == 0 &&
         memcmp(r.bc, bc, sizeof(bc)) == 0;
}

// Requests that may share a batch: same operator and iteration limit.
bool same_batch_key(const wd_request& a, const wd_request& b) {
  int ba[4], bb[4];
  request_bc(a, ba);
  request_bc(b, bb);
  return a.precision == b.precision && a.maxit == b.maxit && memcmp(a.dims, b.dims, sizeof(a.dims)) == 0 &&
         memcmp(ba, bb, sizeof(ba)) == 0;
}

}  // namespace

struct wd_server {
  std::mutex mu;
  std::condition_variable cv_work;  // slots wait for jobs
  std::condition_variable cv_done;  // clients wait for results
  std::deque<Job*> pending;
  std::map<long long, std::unique_ptr<Job>> jobs;
  std::vector<std::unique_ptr<Slot>> slots;
  size_t budget = 0, used = 0;
  long long next_id = 1;
  unsigned long long tick = 0;
  int max_batch = 8;
  int policy = 0;             // 0: oldest first; 1: least estimated work first, with aging
  double max_wait_ms = 1000;  // policy 1: a request waiting longer than this goes first
  bool stopping = false;
  int device = 0;
  wd_server_stats stats;
};

namespace {

void free_resident(Resident& r) {
  if (r.ctx) wd_destroy(r.ctx);
  if (r.src) cudaFree(r.src);
  if (r.x) cudaFree(r.x);
  r.ctx = nullptr;
  r.src = r.x = nullptr;
}

// Runs on the slot thread: the job's reserved resident, created now if it is a placeholder. Only
// this thread touches the slot's cache while the slot is busy.
wd_status prepare(Slot* s, const Job* j, Resident** out) {
  if (j->res_idx < 0 || j->res_idx >= (int)s->cache.size()) {
    wdk::set_last_error("internal: no reserved resident for the job");
    return WD_ECUDA;
  }
  Resident* e = &s->cache[j->res_idx];
  const wd_request& r = j->req;
  if (e->ctx) {
    *out = e;
    return wd_set_kappa(e->ctx, r.kappa);
  }
  wd_status st = wd_create(r.dims, r.kappa, r.boundary_set ? r.boundary : nullptr, r.precision, s->stream, &e->ctx);
  if (st != WD_OK) return st;
  const size_t V = (size_t)volume_of(r.dims);
  if (cudaMalloc(&e->src, V * 192) != cudaSuccess || cudaMalloc(&e->x, V * 192) != cudaSuccess) {
    cudaGetLastError();
    free_resident(*e);
    wdk::set_last_error("cudaMalloc of the slot's source/solution buffers failed");
    return WD_ENOMEM;
  }
  *out = e;
  return WD_OK;
}

// The slot's batch: every job's fields on its own context, then one cg_solve_batch for all of them
// (a batch of one is the plain solve), then the solutions out.
void run_batch(Slot* s, std::vector<Job*>& batch) {
  nvtxRangePushA("wd:serve_batch");
  struct PopRange {
    ~PopRange() { nvtxRangePop(); }
  } pop_;
  const int n = (int)batch.size();
  std::vector<Resident*> res(n, nullptr);
  std::vector<wd_status> st(n, WD_OK);
  for (int i = 0; i < n; ++i) {
    Job* j = batch[i];
    const wd_request& r = j->req;
    memset(&j->res, 0, sizeof(j->res));
    Resident* e = nullptr;
    wd_status t = prepare(s, j, &e);
    const size_t V = (size_t)volume_of(r.dims);
    if (t == WD_OK)
      t = wd_generate_gauge(e->ctx, r.eps, r.gauge_seed, (r.precision & ~WD_EVEN_ODD) == WD_PREC_F64 ? 0 : 1, nullptr);
    if (t == WD_OK) {
      if (r.src_host) {
        if (cudaMemcpyAsync(e->src, r.src_host, V * 192, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) t = WD_ECUDA;
      } else {
        t = wd_generate_source(e->ctx, r.source_seed, e->src);
      }
    }
    if (t == WD_OK && cudaMemsetAsync(e->x, 0, V * 192, s->stream) != cudaSuccess) t = WD_ECUDA;
    res[i] = e;
    st[i] = t;
  }
  std::vector<wd_ctx*> ctxs;
  std::vector<const void*> srcs;
  std::vector<void*> xs;
  std::vector<double> tols;
  std::vector<int> idx;
  for (int i = 0; i < n; ++i)
    if (st[i] == WD_OK) {
      ctxs.push_back(res[i]->ctx);
      srcs.push_back(res[i]->src);
      xs.push_back(res[i]->x);
      tols.push_back(batch[i]->req.tol);
      idx.push_back(i);
    }
  const int m = (int)ctxs.size();
  std::vector<int> iters(m, 0), sts(m, WD_OK);
  std::vector<double> rel(m, 0.0);
  if (m > 0) {
    const wd_status all = cg_solve_batch(ctxs.data(), m, srcs.data(), xs.data(), tols.data(), batch[idx[0]]->req.maxit,
                                         iters.data(), rel.data(), sts.data());
    if (all != WD_OK && all != WD_NOT_CONVERGED && all != WD_BREAKDOWN)
      for (int k = 0; k < m; ++k) sts[k] = (int)all;  // an argument or device failure of the whole batch
  }
  for (int k = 0; k < m; ++k) {
    const int i = idx[k];
    st[i] = (wd_status)sts[k];
    Job* j = batch[i];
    const wd_request& r = j->req;
    const size_t V = (size_t)volume_of(r.dims);
    if ((st[i] == WD_OK || st[i] == WD_NOT_CONVERGED) && r.x_host) {
      if (cudaMemcpyAsync(r.x_host, res[i]->x, V * 192, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
          cudaStreamSynchronize(s->stream) != cudaSuccess)
        st[i] = WD_ECUDA;
    }
    j->res.iterations = iters[k];
    j->res.true_rel_residual = rel[k];
  }
  for (int i = 0; i < n; ++i) {
    Job* j = batch[i];
    wd_stats ws;
    memset(&ws, 0, sizeof(ws));
    if (res[i] && res[i]->ctx) wd_get_stats(res[i]->ctx, &ws);
    j->res.status = st[i];
    j->res.reliable_updates = ws.reliable_updates;
    j->res.slot = s->index;
    j->res.batch = n;
  }
}

void schedule(wd_server* srv);

void slot_main(wd_server* srv, Slot* s) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  for (;;) {
    srv->cv_work.wait(lk, [&] { return srv->stopping || !s->batch.empty(); });
    if (s->batch.empty() && srv->stopping) break;
    std::vector<Job*> batch = s->batch;
    lk.unlock();
    const Clock::time_point t0 = Clock::now();
    for (Job* j : batch) j->t_start = t0;
    run_batch(s, batch);
    const Clock::time_point t1 = Clock::now();
    lk.lock();
    for (Job* j : batch) {
      j->t_done = t1;
      j->res.queue_ms = ms_between(j->t_submit, j->t_start);
      j->res.solve_ms = ms_between(j->t_start, j->t_done);
      j->res.latency_ms = ms_between(j->t_submit, j->t_done);
      j->done = true;
      if (j->res.status != WD_OK) srv->stats.failed += 1;
      srv->stats.completed += 1;
    }
    if (batch.size() > 1) {
      srv->stats.batches += 1;
      srv->stats.batched_requests += (long long)batch.size();
    }
    // a context whose creation failed holds nothing: drop it and its charge
    for (auto& e : s->cache) {
      e.taken = false;
      if (!e.ctx) srv->used -= e.bytes;
    }
    s->cache.erase(std::remove_if(s->cache.begin(), s->cache.end(), [](const Resident& e) { return e.ctx == nullptr; }),
                   s->cache.end());
    s->batch.clear();
    schedule(srv);  // admit waiting requests into the freed slot
    srv->cv_done.notify_all();
  }
  lk.unlock();
  for (auto& e : s->cache) free_resident(e);
  s->cache.clear();
}

// Estimated work of a request (policy 1): sites times a per-precision factor (plain FP64 solves
// take about 8x a mixed-precision solve on GB300, plain FP32 ones about 0.5x; even-odd about
// 0.6x), times 1.2 for the tighter of the two tolerances. Only the order matters.
double job_cost(const wd_request& r) {
  double f = 1.0;
  switch (r.precision & ~WD_EVEN_ODD) {
    case WD_PREC_F64: f = 8.0; break;
    case WD_PREC_F32: f = 0.5; break;
    default: f = 1.0;
  }
  if (r.precision & WD_EVEN_ODD) f *= 0.6;
  if (r.tol < 1e-9) f *= 1.2;
  return f * (double)volume_of(r.dims);
}

// The request admitted next: the oldest, or (policy 1) the least work unless the oldest has waited
// longer than max_wait_ms (then it goes first, so that large requests are not starved).
Job* next_job(wd_server* srv) {
  Job* oldest = srv->pending.front();
  if (srv->policy == 0 || srv->pending.size() < 2) return oldest;
  if (ms_between(oldest->t_submit, Clock::now()) > srv->max_wait_ms) return oldest;
  Job* best = oldest;
  double bc = job_cost(oldest->req);
  for (Job* j : srv->pending) {
    const double c = job_cost(j->req);
    if (c < bc) {
      best = j;
      bc = c;
    }
  }
  return best;
}

size_t slot_bytes(const Slot* s) {
  size_t b = 0;
  for (const auto& e : s->cache) b += e.bytes;
  return b;
}

// Assign pending jobs to idle slots (called with the mutex held).
// The job next_job picks goes first (the oldest, or under policy 1 the least work unless the oldest
// has waited too long), with up to max_batch - 1 other queued jobs of the same operator when
// its CG loop is the persistent kernel (a batch shares its loop launches); other jobs keep their
// order. The slot: an idle one with resident contexts of the operator (the most of them), else the
// idle slot holding the fewest resident bytes. Jobs without an idle resident get a placeholder
// charged against the budget, after the least recently used residents of idle slots are freed until
// they fit (the batch shrinks to what fits). Only idle slots' residents are freed (here, under the
// lock: an idle slot's thread does not touch its cache), so device memory never exceeds what is
// charged.
void schedule(wd_server* srv) {
  while (!srv->pending.empty()) {
    Job* j = next_job(srv);
    Slot* pick = nullptr;
    int pick_warm = 0;
    for (auto& sp : srv->slots) {
      if (!sp->batch.empty()) continue;
      int w = 0;
      for (auto& e : sp->cache)
        if (e.ctx && same_operator(e, j->req)) ++w;
      if (w > pick_warm) {
        pick = sp.get();
        pick_warm = w;
      }
    }
    if (!pick) {
      for (auto& sp : srv->slots) {
        if (!sp->batch.empty()) continue;
        if (!pick || slot_bytes(sp.get()) < slot_bytes(pick)) pick = sp.get();
      }
    }
    if (!pick) break;  // every slot busy
    // the batch: j and later jobs of its operator, up to max_batch
    std::vector<Job*> members{j};
    if (srv->max_batch > 1 && wdk::batch_capable(j->req.dims, j->req.precision)) {
      for (size_t i = 0; i < srv->pending.size() && (int)members.size() < srv->max_batch; ++i)
        if (srv->pending[i] != j && same_batch_key(srv->pending[i]->req, j->req)) members.push_back(srv->pending[i]);
    }
    // residents: warm ones of the slot first, then placeholders charged against the budget
    std::vector<int> slots_idx;
    for (size_t i = 0; i < pick->cache.size() && slots_idx.size() < members.size(); ++i) {
      Resident& e = pick->cache[i];
      if (e.ctx && !e.taken && same_operator(e, j->req)) {
        e.taken = true;
        slots_idx.push_back((int)i);
      }
    }
    size_t evictable = 0;
    for (auto& sp : srv->slots) {
      if (!sp->batch.empty()) continue;
      for (auto& e : sp->cache)
        if (!e.taken) evictable += e.bytes;
    }
    size_t fresh_n = members.size() - slots_idx.size();
    while (fresh_n > 0 && srv->used - evictable + fresh_n * j->bytes > srv->budget) --fresh_n;
    if (slots_idx.empty() && fresh_n == 0) {  // not even the oldest job fits yet: wait for memory
      for (int i : slots_idx) pick->cache[i].taken = false;
      break;
    }
    members.resize(slots_idx.size() + fresh_n);
    while (srv->used + fresh_n * j->bytes > srv->budget) {
      Slot* vs = nullptr;
      size_t vi = 0;
      for (auto& sp : srv->slots) {
        if (!sp->batch.empty()) continue;
        for (size_t i = 0; i < sp->cache.size(); ++i)
          if (!sp->cache[i].taken && (!vs || sp->cache[i].last_used < vs->cache[vi].last_used)) {
            vs = sp.get();
            vi = i;
          }
      }
      if (!vs) break;
      srv->used -= vs->cache[vi].bytes;
      free_resident(vs->cache[vi]);
      vs->cache.erase(vs->cache.begin() + vi);
      if (vs == pick)  // indices of the slot's reserved residents shift past the erased one
        for (int& k : slots_idx)
          if (k > (int)vi) --k;
      srv->stats.evictions += 1;
    }
    srv->stats.warm_hits += (long long)slots_idx.size();
    for (size_t f = 0; f < fresh_n; ++f) {
      Resident fresh;
      memcpy(fresh.dims, j->req.dims, sizeof(fresh.dims));
      request_bc(j->req, fresh.bc);
      fresh.precision = j->req.precision;
      fresh.bytes = j->bytes;
      fresh.taken = true;
      pick->cache.push_back(fresh);
      slots_idx.push_back((int)pick->cache.size() - 1);
      srv->used += j->bytes;
    }
    for (size_t k = 0; k < members.size(); ++k) {
      members[k]->res_idx = slots_idx[k];
      pick->cache[slots_idx[k]].last_used = ++srv->tick;
    }
    for (Job* m : members) srv->pending.erase(std::find(srv->pending.begin(), srv->pending.end(), m));
    pick->batch = members;
    srv->stats.admitted += (long long)members.size();
  }
  if ((double)srv->used > srv->stats.peak_bytes) srv->stats.peak_bytes = (double)srv->used;
  srv->cv_work.notify_all();
}

}  // namespace

extern "C" {

wd_status wd_server_create(double budget_bytes, int slots, wd_server** out) {
  if (!out) {
    wdk::set_last_error("out is null");
    return WD_EINVAL;
  }
  *out = nullptr;
  if (!(budget_bytes > 0) || slots < 1 || slots > 64) {
    wdk::set_last_error("budget must be positive and slots in [1, 64]");
    return WD_EINVAL;
  }
  wd_server* srv = new wd_server;
  memset(&srv->stats, 0, sizeof(srv->stats));
  srv->budget = (size_t)budget_bytes;
  if (cudaGetDevice(&srv->device) != cudaSuccess) {
    delete srv;
    wdk::set_last_error("no CUDA device");
    return WD_ECUDA;
  }
  for (int i = 0; i < slots; ++i) {
    auto s = std::make_unique<Slot>();
    s->index = i;
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      wdk::set_last_error("stream creation failed");
      for (auto& t : srv->slots) cudaStreamDestroy(t->stream);
      delete srv;
      return WD_ECUDA;
    }
    srv->slots.push_back(std::move(s));
  }
  for (auto& s : srv->slots) s->th = std::thread(slot_main, srv, s.get());
  *out = srv;
  return WD_OK;
}

wd_status wd_server_submit(wd_server* srv, const wd_request* r, long long* id) {
  if (!srv || !r || !id) {
    wdk::set_last_error("null argument");
    return WD_EINVAL;
  }
  for (int i = 0; i < 4; ++i)
    if (r->dims[i] < 2) {
      wdk::set_last_error("every lattice extent must be >= 2");
      return WD_EINVAL;
    }
  if (r->boundary_set)
    for (int i = 0; i < 4; ++i)
      if (r->boundary[i] != 1 && r->boundary[i] != -1) {
        wdk::set_last_error("boundary entries must be +1 or -1");
        return WD_EINVAL;
      }
  if (!(r->tol > 0) || r->maxit < 0) {
    wdk::set_last_error("bad tol or maxit");
    return WD_EINVAL;
  }
  const size_t bytes = request_bytes(r->dims, r->precision);
  if (bytes == 0) {
    wdk::set_last_error("precision must be one of WD_PREC_*");
    return WD_EINVAL;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  if (bytes > srv->budget) {
    wdk::set_last_error("request needs more device memory than the whole budget");
    return WD_ENOMEM;
  }
  auto j = std::make_unique<Job>();
  j->id = srv->next_id++;
  j->req = *r;
  j->bytes = bytes;
  j->t_submit = Clock::now();
  *id = j->id;
  srv->pending.push_back(j.get());
  srv->jobs[j->id] = std::move(j);
  srv->stats.submitted += 1;
  schedule(srv);
  return WD_OK;
}

wd_status wd_server_wait(wd_server* srv, long long id, wd_result* out) {
  if (!srv || !out) {
    wdk::set_last_error("null argument");
    return WD_EINVAL;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(id);
  if (it == srv->jobs.end()) {
    wdk::set_last_error("unknown request id");
    return WD_EINVAL;
  }
  Job* j = it->second.get();
  for (;;) {
    schedule(srv);
    if (j->done) break;
    srv->cv_done.wait_for(lk, std::chrono::milliseconds(50));
  }
  *out = j->res;
  srv->jobs.erase(it);
  return WD_OK;
}

wd_status wd_server_poll(wd_server* srv, long long id, wd_result* out, int* done) {
  if (!srv || !out || !done) {
    wdk::set_last_error("null argument");
    return WD_EINVAL;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  schedule(srv);
  auto it = srv->jobs.find(id);
  if (it == srv->jobs.end()) {
    wdk::set_last_error("unknown request id");
    return WD_EINVAL;
  }
  *done = it->second->done ? 1 : 0;
  if (*done) {
    *out = it->second->res;
    srv->jobs.erase(it);
  }
  return WD_OK;
}

wd_status wd_server_set_max_batch(wd_server* srv, int max_batch) {
  if (!srv || max_batch < 1 || max_batch > 16) {
    wdk::set_last_error("null server or max_batch outside [1, 16]");
    return WD_EINVAL;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->max_batch = max_batch;
  return WD_OK;
}

wd_status wd_server_set_policy(wd_server* srv, int policy, double max_wait_ms) {
  if (!srv || (policy != 0 && policy != 1) || !(max_wait_ms >= 0.0)) {
    wdk::set_last_error("null server, policy not 0 or 1, or negative max_wait_ms");
    return WD_EINVAL;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->policy = policy;
  srv->max_wait_ms = max_wait_ms;
  return WD_OK;
}

wd_status wd_server_get_stats(wd_server* srv, wd_server_stats* out) {
  if (!srv || !out) {
    wdk::set_last_error("null argument");
    return WD_EINVAL;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  *out = srv->stats;
  out->used_bytes = (double)srv->used;
  out->pending = (int)srv->pending.size();
  return WD_OK;
}

void wd_server_destroy(wd_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stopping = true;
    srv->pending.clear();
  }
  srv->cv_work.notify_all();
  for (auto& s : srv->slots)
    if (s->th.joinable()) s->th.join();
  for (auto& s : srv->slots)
    if (s->stream) cudaStreamDestroy(s->stream);
  delete srv;
}

}  // extern "C"
