// Serving runtime: a persistent request loop with continuous admission.
//
// Requests (one single-RHS solve each, with its own lattice, kappa, tolerance, seeded gauge field
// and source) enter a FIFO queue. The scheduler (run by whichever thread submits, waits or
// finishes a job) admits them into execution slots as slots and device memory free up; memory is
// charged against the budget given at creation. Every slot has its own CUDA stream and worker
// thread, so admitted solves run concurrently and their kernels overlap on the device. A slot
// keeps the contexts it created (links, Krylov workspace, CUDA graphs) resident between requests,
// so a request whose volume and precision match an idle slot's resident context runs warm: no
// allocation, no graph rebuild, only wd_set_kappa and the new fields. Least recently used
// residents are evicted when a new volume does not fit in the budget.
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
    case WD_PREC_F64: return extra + V * 576 + 9 * f64 + 2 * f64 + (V / 32 + 64) * 8 * 12;
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
};

struct Slot {
  int index = 0;
  cudaStream_t stream = nullptr;
  std::vector<Resident> cache;  // resident contexts of this slot (guarded by the server mutex
                                // while the slot is idle; owned by the slot thread while busy)
  Job* job = nullptr;
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

bool same_key(const Resident& r, const wd_request& q) { return r.ctx && same_operator(r, q); }

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

// Runs on the slot thread: find the job's resident context, or create it in the placeholder the
// scheduler reserved. Only this thread touches the slot's cache while it holds a job.
wd_status prepare(Slot* s, const wd_request& r, Resident** out) {
  for (auto& e : s->cache) {
    if (same_key(e, r)) {
      wd_status st = wd_set_kappa(e.ctx, r.kappa);
      *out = &e;
      return st;
    }
  }
  Resident* e = nullptr;
  for (auto& c : s->cache)
    if (!c.ctx && same_operator(c, r)) e = &c;
  if (!e) {
    wdk::set_last_error("internal: no reserved resident for the job");
    return WD_ECUDA;
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

void run_job(Slot* s, Job* j) {
  nvtxRangePushA("wd:serve_job");
  struct PopRange {
    ~PopRange() { nvtxRangePop(); }
  } pop_;
  const wd_request& r = j->req;
  wd_result& out = j->res;
  memset(&out, 0, sizeof(out));
  Resident* e = nullptr;
  wd_status st = prepare(s, r, &e);
  const size_t V = (size_t)volume_of(r.dims);
  if (st == WD_OK) st = wd_generate_gauge(e->ctx, r.eps, r.gauge_seed, (r.precision & ~WD_EVEN_ODD) == WD_PREC_F64 ? 0 : 1, nullptr);
  if (st == WD_OK) {
    if (r.src_host) {
      if (cudaMemcpyAsync(e->src, r.src_host, V * 192, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) st = WD_ECUDA;
    } else {
      st = wd_generate_source(e->ctx, r.source_seed, e->src);
    }
  }
  if (st == WD_OK && cudaMemsetAsync(e->x, 0, V * 192, s->stream) != cudaSuccess) st = WD_ECUDA;
  int iters = 0;
  double res = 0.0;
  if (st == WD_OK) st = cg_solve(e->ctx, e->src, e->x, r.tol, r.maxit, &iters, &res);
  if ((st == WD_OK || st == WD_NOT_CONVERGED) && r.x_host) {
    if (cudaMemcpyAsync(r.x_host, e->x, V * 192, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
      st = WD_ECUDA;
  }
  wd_stats ws;
  memset(&ws, 0, sizeof(ws));
  if (e && e->ctx) wd_get_stats(e->ctx, &ws);
  out.status = st;
  out.iterations = iters;
  out.reliable_updates = ws.reliable_updates;
  out.true_rel_residual = res;
  out.slot = s->index;
}

void schedule(wd_server* srv);

void slot_main(wd_server* srv, Slot* s) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  for (;;) {
    srv->cv_work.wait(lk, [&] { return srv->stopping || s->job != nullptr; });
    if (s->job == nullptr && srv->stopping) break;
    Job* j = s->job;
    lk.unlock();
    j->t_start = Clock::now();
    run_job(s, j);
    j->t_done = Clock::now();
    lk.lock();
    j->res.queue_ms = ms_between(j->t_submit, j->t_start);
    j->res.solve_ms = ms_between(j->t_start, j->t_done);
    j->res.latency_ms = ms_between(j->t_submit, j->t_done);
    j->done = true;
    if (j->res.status != WD_OK) srv->stats.failed += 1;
    // a context whose creation failed holds nothing: drop it and its charge
    for (auto& e : s->cache)
      if (!e.ctx) srv->used -= e.bytes;
    s->cache.erase(std::remove_if(s->cache.begin(), s->cache.end(), [](const Resident& e) { return e.ctx == nullptr; }),
                   s->cache.end());
    s->job = nullptr;
    srv->stats.completed += 1;
    schedule(srv);  // admit waiting requests into the freed slot
    srv->cv_done.notify_all();
  }
  lk.unlock();
  for (auto& e : s->cache) free_resident(e);
  s->cache.clear();
}

// Assign pending jobs to idle slots (called with the mutex held), in FIFO order.
// 1) An idle slot with a resident context of the request's volume and precision (warm).
// 2) Else the idle slot holding the fewest resident bytes gets a new context, after the least
//    recently used residents of idle slots are freed until the request fits in the budget. Only
//    idle slots' residents are freed (here, under the lock: an idle slot's thread does not touch
//    its cache), so device memory never exceeds what is charged.
void schedule(wd_server* srv) {
  while (!srv->pending.empty()) {
    Job* j = srv->pending.front();
    Slot* pick = nullptr;
    Resident* warm = nullptr;
    for (auto& sp : srv->slots) {
      if (sp->job) continue;
      for (auto& e : sp->cache)
        if (same_key(e, j->req)) {
          pick = sp.get();
          warm = &e;
          break;
        }
      if (pick) break;
    }
    if (pick) {
      srv->stats.warm_hits += 1;
      warm->last_used = ++srv->tick;
    } else {
      size_t idle_bytes = 0;
      for (auto& sp : srv->slots) {
        if (sp->job) continue;
        size_t b = 0;
        for (auto& e : sp->cache) b += e.bytes;
        idle_bytes += b;
        if (!pick) {
          pick = sp.get();
        } else {
          size_t pb = 0;
          for (auto& e : pick->cache) pb += e.bytes;
          if (b < pb) pick = sp.get();
        }
      }
      if (!pick || srv->used - idle_bytes + j->bytes > srv->budget) break;  // wait for a slot or memory
      while (srv->used + j->bytes > srv->budget) {
        Slot* vs = nullptr;
        size_t vi = 0;
        for (auto& sp : srv->slots) {
          if (sp->job) continue;
          for (size_t i = 0; i < sp->cache.size(); ++i)
            if (!vs || sp->cache[i].last_used < vs->cache[vi].last_used) {
              vs = sp.get();
              vi = i;
            }
        }
        if (!vs) break;
        srv->used -= vs->cache[vi].bytes;
        free_resident(vs->cache[vi]);
        vs->cache.erase(vs->cache.begin() + vi);
        srv->stats.evictions += 1;
      }
      Resident fresh;
      memcpy(fresh.dims, j->req.dims, sizeof(fresh.dims));
      request_bc(j->req, fresh.bc);
      fresh.precision = j->req.precision;
      fresh.bytes = j->bytes;
      fresh.last_used = ++srv->tick;
      pick->cache.push_back(fresh);
      srv->used += j->bytes;
    }
    srv->pending.pop_front();
    pick->job = j;
    srv->stats.admitted += 1;
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
