// C ABI of the Wilson-Dirac CG library: context management, gauge loading, operator application
// and the CG drivers (plain FP64/FP32 and mixed precision with reliable updates).
//
// The CG iteration runs as one CUDA graph per context: a prologue (r = eta - D x, p = D^dag r,
// convergence check), a device-side while node whose body is one CG iteration (the body's last
// kernel sets the loop condition, so the host never polls inside a solve), and an epilogue that
// recomputes the true residual. The host launches the graph, waits once, and relaunches only if
// the recomputed residual has not reached the tolerance (a restart from the true residual).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/wd.h"
#include "wd_internal.h"

using namespace wdk;

namespace {

thread_local std::string g_err;

wd_status fail(wd_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

#define WD_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(WD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));               \
  } while (0)

bool is_mixed(int p) { return p == WD_PREC_MIXED_F32 || p == WD_PREC_MIXED_F16; }

}  // namespace

namespace wdk {
// Message for wd_last_error(), set by the other translation units of the library.
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace wdk

struct wd_ctx {
  int dims[4];
  int bc[4];
  int V;
  int precision;
  double kappa;
  GeomH geom;
  cudaStream_t stream;
  cudaStream_t cap;  // internal stream used only to capture graphs
  cudaStream_t cap2;
  int device;
  int sms;

  // working (inner) precision of the Krylov vectors and its gauge copy
  int wprec;  // SP64 / SP32 / SP16
  FieldPtr x, r, p, q, s, eta;  // plain modes: all in wprec; mixed: r, p, q, s in wprec, x = x_lo (SP32)
  // FP64 operator and outer vectors (FP64 context and mixed modes)
  FieldPtr x64, r64, eta64;
  void* gauge64;
  void* gauge32;
  int c12;
  bool gauge_loaded;

  double* partials;
  size_t partials_len;
  CgScalars* sc;
  CgScalars* sc_host;  // pinned

  // options
  double delta;
  int use_graph;
  int block_dslash;
  int block_blas;
  int max_restarts;

  // graph
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool graph_ready;

  wd_stats stats;
  cudaEvent_t ev0, ev1;
  void* staging;  // host gauge uploads (kept for reuse)
};

namespace {

size_t spinor_bytes(int prec, int V) {
  switch (prec) {
    case SP64: return (size_t)V * 12 * 16;
    case SP32: return (size_t)V * 12 * 8;
    case SP16: return (size_t)V * 12 * 4;
  }
  return 0;
}

wd_status alloc_field(wd_ctx* c, FieldPtr* f, int prec) {
  f->prec = prec;
  f->norm = nullptr;
  f->p = nullptr;
  if (cudaMalloc(&f->p, spinor_bytes(prec, c->V)) != cudaSuccess) {
    cudaGetLastError();
    return fail(WD_ENOMEM, "cudaMalloc of a spinor field failed");
  }
  if (cudaMemsetAsync(f->p, 0, spinor_bytes(prec, c->V), c->stream) != cudaSuccess)
    return fail(WD_ECUDA, "cudaMemsetAsync failed");
  if (prec == SP16) {
    if (cudaMalloc(&f->norm, sizeof(float) * (size_t)c->V) != cudaSuccess) {
      cudaGetLastError();
      return fail(WD_ENOMEM, "cudaMalloc of a norm field failed");
    }
    if (cudaMemsetAsync(f->norm, 0, sizeof(float) * (size_t)c->V, c->stream) != cudaSuccess)
      return fail(WD_ECUDA, "cudaMemsetAsync failed");
  }
  return WD_OK;
}

void free_field(FieldPtr* f) {
  if (f->p) cudaFree(f->p);
  if (f->norm) cudaFree(f->norm);
  f->p = nullptr;
  f->norm = nullptr;
}

Red red_to(wd_ctx* c, int slot, double* result) {
  Red r;
  r.partials = c->partials;
  r.ticket = &c->sc->ticket[slot];
  r.result = result;
  return r;
}

Red no_red() {
  Red r;
  r.partials = nullptr;
  r.ticket = nullptr;
  r.result = nullptr;
  return r;
}

int dslash_block(const wd_ctx* c, int prec) {
  if (c->block_dslash > 0) return c->block_dslash;
  return prec == SP64 ? 128 : 256;
}

GaugePtr gauge_for(const wd_ctx* c, int prec) {
  GaugePtr g;
  if (prec == SP64) {
    g.p = c->gauge64;
    g.prec = SP64;
    g.c12 = 0;
  } else {
    g.p = c->gauge32;
    g.prec = SP32;
    g.c12 = c->c12;
  }
  return g;
}

// out = D in (or b - D in); optional |out|^2 into *norm_dst
cudaError_t dslash(wd_ctx* c, FieldPtr in, FieldPtr out, int dagger, int epi, FieldPtr b, double* norm_dst,
                   int slot, const int* skip, cudaStream_t st) {
  DslashCall d;
  d.g = c->geom;
  d.u = gauge_for(c, in.prec);
  d.in = in;
  d.out = out;
  d.b = b;
  d.kappa = c->kappa;
  d.dagger = dagger;
  d.epi = epi;
  d.skip = skip;
  d.red = norm_dst ? red_to(c, slot, norm_dst) : no_red();
  d.block = dslash_block(c, in.prec);
  return launch_dslash(d, st);
}

FieldPtr none_field() {
  FieldPtr f;
  f.p = nullptr;
  f.norm = nullptr;
  f.prec = -1;
  return f;
}

// ---------------------------------------------------------------- plain CG (one precision)

cudaError_t plain_prologue(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long cond) {
  cudaError_t e;
  CgScalars* sc = c->sc;
  if ((e = launch_cg_init(sc, 0, st)) != cudaSuccess) return e;
  // r = eta - D x
  if ((e = dslash(c, c->x, c->r, 0, EPI_RESID, c->eta, &sc->rr, TK_DSLASH_A, nullptr, st)) != cudaSuccess) return e;
  // p = D^dag r, gamma = |p|^2
  if ((e = dslash(c, c->r, c->p, 1, EPI_PLAIN, none_field(), &sc->gamma, TK_DSLASH_B, nullptr, st)) != cudaSuccess)
    return e;
  return launch_cg_check(sc, use_cond, cond, st);
}

cudaError_t plain_body(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long cond) {
  cudaError_t e;
  CgScalars* sc = c->sc;
  const int bb = c->block_blas;
  // q = D p, |q|^2
  if ((e = dslash(c, c->p, c->q, 0, EPI_PLAIN, none_field(), &sc->qq, TK_DSLASH_A, &sc->status, st)) != cudaSuccess)
    return e;
  // alpha; r -= alpha q; |r|^2
  if ((e = launch_cg_update_r(c->wprec, c->r, c->q, c->V, sc, c->partials, bb, st)) != cudaSuccess) return e;
  // s = D^dag r, gamma' = |s|^2
  if ((e = dslash(c, c->r, c->s, 1, EPI_PLAIN, none_field(), &sc->gamma_new, TK_DSLASH_B, &sc->status, st)) !=
      cudaSuccess)
    return e;
  // x += alpha p; p = s + beta p; loop condition
  return launch_cg_update_xp(c->wprec, c->x, c->p, c->s, c->V, sc, c->partials, use_cond, cond, bb, st);
}

cudaError_t plain_epilogue(wd_ctx* c, cudaStream_t st) {
  // true residual eta - D x into q
  return dslash(c, c->x, c->q, 0, EPI_RESID, c->eta, &c->sc->rr_true, TK_DSLASH_C, nullptr, st);
}

// ---------------------------------------------------------------- mixed precision CG

cudaError_t mixed_prologue(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long cond) {
  cudaError_t e;
  CgScalars* sc = c->sc;
  const int bb = c->block_blas;
  if ((e = launch_cg_init(sc, 0, st)) != cudaSuccess) return e;
  // r_hi = eta - D x_hi (FP64); x_lo = 0; r_lo = r_hi
  if ((e = dslash(c, c->x64, c->r64, 0, EPI_RESID, c->eta64, &sc->rr_true, TK_DSLASH_C, nullptr, st)) != cudaSuccess)
    return e;
  if ((e = launch_zero(c->x.p, spinor_bytes(c->x.prec, c->V), st)) != cudaSuccess) return e;
  if ((e = launch_mp_convert(c->r64, c->r, c->V, sc, c->partials, 0, nullptr, bb, st)) != cudaSuccess) return e;
  // p = D^dag r_lo
  if ((e = dslash(c, c->r, c->p, 1, EPI_PLAIN, none_field(), &sc->gamma, TK_DSLASH_B, nullptr, st)) != cudaSuccess)
    return e;
  return launch_cg_check(sc, use_cond, cond, st);
}

// reliable update: x_hi += x_lo; x_lo = 0; r_hi = eta - D x_hi (FP64); r_lo = r_hi
cudaError_t mixed_update(wd_ctx* c, cudaStream_t st) {
  cudaError_t e;
  CgScalars* sc = c->sc;
  const int bb = c->block_blas;
  if ((e = launch_mp_accumulate(c->x64, c->x, c->V, nullptr, bb, st)) != cudaSuccess) return e;
  if ((e = dslash(c, c->x64, c->r64, 0, EPI_RESID, c->eta64, &sc->rr_true, TK_DSLASH_C, nullptr, st)) != cudaSuccess)
    return e;
  return launch_mp_convert(c->r64, c->r, c->V, sc, c->partials, 1, nullptr, bb, st);
}

cudaError_t mixed_body_a(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long upd) {
  cudaError_t e;
  CgScalars* sc = c->sc;
  if ((e = dslash(c, c->p, c->q, 0, EPI_PLAIN, none_field(), &sc->qq, TK_DSLASH_A, &sc->status, st)) != cudaSuccess)
    return e;
  return launch_mp_update_rx(c->wprec, c->r, c->q, c->p, c->x, c->V, sc, c->partials, use_cond, upd, c->block_blas, st);
}

cudaError_t mixed_body_b(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long cond) {
  cudaError_t e;
  CgScalars* sc = c->sc;
  if ((e = dslash(c, c->r, c->s, 1, EPI_PLAIN, none_field(), &sc->gamma_new, TK_DSLASH_B, &sc->status, st)) !=
      cudaSuccess)
    return e;
  return launch_mp_update_p(c->wprec, c->p, c->s, c->V, sc, c->partials, use_cond, cond, c->block_blas, st);
}

cudaError_t mixed_epilogue(wd_ctx* c, cudaStream_t st) {
  cudaError_t e;
  if ((e = launch_mp_accumulate(c->x64, c->x, c->V, nullptr, c->block_blas, st)) != cudaSuccess) return e;
  return dslash(c, c->x64, c->r64, 0, EPI_RESID, c->eta64, &c->sc->rr_true, TK_DSLASH_C, nullptr, st);
}

// reliable update with skip flags instead of a conditional node: each kernel checks the flag
cudaError_t mixed_update_flagged(wd_ctx* c, cudaStream_t st) {
  cudaError_t e;
  CgScalars* sc = c->sc;
  const int bb = c->block_blas;
  if ((e = launch_mp_accumulate(c->x64, c->x, c->V, &sc->need_update, bb, st)) != cudaSuccess) return e;
  if ((e = dslash(c, c->x64, c->r64, 0, EPI_RESID, c->eta64, &sc->rr_true, TK_DSLASH_C, &sc->no_update, st)) !=
      cudaSuccess)
    return e;
  return launch_mp_convert(c->r64, c->r, c->V, sc, c->partials, 1, &sc->need_update, bb, st);
}

// ---------------------------------------------------------------- graph construction

wd_status cap_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) return fail(WD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return WD_OK;
}

// Append a conditional node at the current capture point of `st`; the handle must already exist.
wd_status add_conditional(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                          cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t capg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  WD_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &capg, &deps, nullptr, &ndeps));
  if (cs != cudaStreamCaptureStatusActive) return fail(WD_ECUDA, "stream is not capturing");
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = type;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  WD_CUDA(cudaGraphAddNode(&node, capg, deps, nullptr, ndeps, &cp));
  WD_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  *body = cp.conditional.phGraph_out[0];
  return WD_OK;
}

void destroy_graph(wd_ctx* c) {
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->exec = nullptr;
  c->graph = nullptr;
  c->graph_ready = false;
}

// Ends a capture left open by an error so the stream is usable again.
void abort_capture(cudaStream_t st) {
  cudaStreamCaptureStatus cs;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(st, &g);
  }
  cudaGetLastError();
}

// Graph: prologue -> while(loop) { body } -> epilogue -> copy scalars to pinned host memory.
// Mixed precision bodies use a nested if-node for the reliable update when use_if != 0.
wd_status build_graph_impl(wd_ctx* c, int use_if) {
  const bool mixed = is_mixed(c->precision);
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
  WD_CUDA(cudaGraphCreate(&c->graph, 0));
  cudaGraphConditionalHandle loop_h;
  // default 0 at every launch: if no kernel sets the condition, the loop body does not run
  WD_CUDA(cudaGraphConditionalHandleCreate(&loop_h, c->graph, 0, cudaGraphCondAssignDefault));
  cudaGraph_t loop_body = nullptr;
  wd_status st;
  WD_CUDA(cudaStreamBeginCaptureToGraph(c->cap, c->graph, nullptr, nullptr, 0, mode));
  if ((st = cap_check(mixed ? mixed_prologue(c, c->cap, 1, loop_h) : plain_prologue(c, c->cap, 1, loop_h),
                      "prologue")) != WD_OK)
    return st;
  if ((st = add_conditional(c->cap, loop_h, cudaGraphCondTypeWhile, &loop_body)) != WD_OK) return st;
  if ((st = cap_check(mixed ? mixed_epilogue(c, c->cap) : plain_epilogue(c, c->cap), "epilogue")) != WD_OK) return st;
  WD_CUDA(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->cap));
  cudaGraph_t g = nullptr;
  WD_CUDA(cudaStreamEndCapture(c->cap, &g));

  WD_CUDA(cudaStreamBeginCaptureToGraph(c->cap2, loop_body, nullptr, nullptr, 0, mode));
  if (!mixed) {
    if ((st = cap_check(plain_body(c, c->cap2, 1, loop_h), "body")) != WD_OK) return st;
  } else if (use_if) {
    cudaGraphConditionalHandle upd_h;
    WD_CUDA(cudaGraphConditionalHandleCreate(&upd_h, loop_body, 0, cudaGraphCondAssignDefault));
    if ((st = cap_check(mixed_body_a(c, c->cap2, 1, upd_h), "body a")) != WD_OK) return st;
    cudaGraph_t upd_body = nullptr;
    if ((st = add_conditional(c->cap2, upd_h, cudaGraphCondTypeIf, &upd_body)) != WD_OK) return st;
    if ((st = cap_check(mixed_body_b(c, c->cap2, 1, loop_h), "body b")) != WD_OK) return st;
    cudaGraph_t lb = nullptr;
    WD_CUDA(cudaStreamEndCapture(c->cap2, &lb));
    WD_CUDA(cudaStreamBeginCaptureToGraph(c->cap2, upd_body, nullptr, nullptr, 0, mode));
    if ((st = cap_check(mixed_update(c, c->cap2), "update")) != WD_OK) return st;
  } else {
    if ((st = cap_check(mixed_body_a(c, c->cap2, 0, 0), "body a")) != WD_OK) return st;
    if ((st = cap_check(mixed_update_flagged(c, c->cap2), "update")) != WD_OK) return st;
    if ((st = cap_check(mixed_body_b(c, c->cap2, 1, loop_h), "body b")) != WD_OK) return st;
  }
  cudaGraph_t bg = nullptr;
  WD_CUDA(cudaStreamEndCapture(c->cap2, &bg));
  WD_CUDA(cudaGraphInstantiate(&c->exec, c->graph, 0));
  c->graph_ready = true;
  return WD_OK;
}

wd_status build_graph(wd_ctx* c) {
  if (c->graph_ready) return WD_OK;
  wd_status st = build_graph_impl(c, 1);
  if (st == WD_OK) return st;
  abort_capture(c->cap);
  abort_capture(c->cap2);
  destroy_graph(c);
  if (!is_mixed(c->precision)) return st;
  // nested conditional nodes unavailable: fall back to flag-guarded update kernels
  st = build_graph_impl(c, 0);
  if (st != WD_OK) {
    abort_capture(c->cap);
    abort_capture(c->cap2);
    destroy_graph(c);
  }
  return st;
}

// Run one solve attempt without graphs: direct launches, the host reads the status each step.
wd_status run_host_loop(wd_ctx* c) {
  const bool mixed = is_mixed(c->precision);
  CgScalars* sc = c->sc;
  WD_CUDA(mixed ? mixed_prologue(c, c->stream, 0, 0) : plain_prologue(c, c->stream, 0, 0));
  for (;;) {
    WD_CUDA(cudaMemcpyAsync(c->sc_host, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
    WD_CUDA(cudaStreamSynchronize(c->stream));
    if (c->sc_host->status != ST_RUNNING) break;
    if (!mixed) {
      WD_CUDA(plain_body(c, c->stream, 0, 0));
      continue;
    }
    WD_CUDA(mixed_body_a(c, c->stream, 0, 0));
    WD_CUDA(cudaMemcpyAsync(c->sc_host, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
    WD_CUDA(cudaStreamSynchronize(c->stream));
    if (c->sc_host->need_update) WD_CUDA(mixed_update(c, c->stream));
    WD_CUDA(mixed_body_b(c, c->stream, 0, 0));
  }
  WD_CUDA(mixed ? mixed_epilogue(c, c->stream) : plain_epilogue(c, c->stream));
  WD_CUDA(cudaMemcpyAsync(c->sc_host, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  return WD_OK;
}

__global__ void set_params_kernel(CgScalars* sc, double tol2, double delta2, int maxit, double* eta2_src) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc->tol2 = tol2;
    sc->delta2 = delta2;
    sc->maxit = maxit;
    sc->iter = 0;
    sc->updates = 0;
    sc->status = ST_RUNNING;
    sc->need_update = 0;
    sc->no_update = 1;
    for (int i = 0; i < 16; ++i) sc->ticket[i] = 0u;
  }
}

wd_status check_ctx(const wd_ctx* c) {
  if (!c) return fail(WD_EINVAL, "null context");
  return WD_OK;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

const char* wd_last_error(void) { return g_err.c_str(); }

const char* wd_version(void) { return "wdcg 0.1 (sm_103a)"; }

wd_status wd_create(const int dims[4], double kappa, const int boundary[4], int precision, void* cuda_stream,
                    wd_ctx** out) {
  g_err.clear();
  if (!out) return fail(WD_EINVAL, "out is null");
  *out = nullptr;
  if (!dims) return fail(WD_EINVAL, "dims is null");
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 2) return fail(WD_EINVAL, "every lattice extent must be >= 2");
    V *= dims[i];
  }
  if (V > (1LL << 27)) return fail(WD_EINVAL, "volume above 2^27 sites");
  if (!std::isfinite(kappa) || std::fabs(kappa) >= 1.0) return fail(WD_EINVAL, "kappa must be finite with |kappa| < 1");
  int bc[4] = {1, 1, 1, -1};
  if (boundary) {
    for (int i = 0; i < 4; ++i) {
      if (boundary[i] != 1 && boundary[i] != -1) return fail(WD_EINVAL, "boundary entries must be +1 or -1");
      bc[i] = boundary[i];
    }
  }
  int wprec;
  switch (precision) {
    case WD_PREC_F64: wprec = SP64; break;
    case WD_PREC_F32: wprec = SP32; break;
    case WD_PREC_MIXED_F32: wprec = SP32; break;
    case WD_PREC_MIXED_F16: wprec = SP16; break;
    default: return fail(WD_EINVAL, "precision must be one of WD_PREC_*");
  }
  wd_ctx* c = new wd_ctx;
  memset(c, 0, sizeof(wd_ctx));
  for (int i = 0; i < 4; ++i) {
    c->dims[i] = dims[i];
    c->bc[i] = bc[i];
  }
  c->V = (int)V;
  c->precision = precision;
  c->wprec = wprec;
  c->kappa = kappa;
  c->geom.L[0] = dims[0];
  c->geom.L[1] = dims[1];
  c->geom.L[2] = dims[2];
  c->geom.L[3] = dims[3];
  c->geom.stride[0] = 1;
  c->geom.stride[1] = dims[0];
  c->geom.stride[2] = dims[0] * dims[1];
  c->geom.stride[3] = dims[0] * dims[1] * dims[2];
  c->geom.V = (int)V;
  for (int i = 0; i < 4; ++i) c->geom.bc[i] = bc[i];
  c->stream = (cudaStream_t)cuda_stream;
  c->delta = 0.1;
  c->use_graph = 1;
  c->block_blas = 256;
  c->max_restarts = 5;
  wd_status st = WD_OK;
  auto bail = [&](wd_status s) {
    wd_destroy(c);
    return s;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) return bail(fail(WD_ECUDA, "no CUDA device"));
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(WD_ECUDA, "stream creation failed"));
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess)
    return bail(fail(WD_ECUDA, "event creation failed"));
  const bool mixed = is_mixed(precision);
  const int xprec = mixed ? SP32 : wprec;
  if ((st = alloc_field(c, &c->x, xprec)) != WD_OK) return bail(st);
  if ((st = alloc_field(c, &c->r, wprec)) != WD_OK) return bail(st);
  if ((st = alloc_field(c, &c->p, wprec)) != WD_OK) return bail(st);
  if ((st = alloc_field(c, &c->q, wprec)) != WD_OK) return bail(st);
  if ((st = alloc_field(c, &c->s, wprec)) != WD_OK) return bail(st);
  if (!mixed) {
    if ((st = alloc_field(c, &c->eta, wprec)) != WD_OK) return bail(st);
  }
  if (mixed || wprec == SP64) {
    if ((st = alloc_field(c, &c->x64, SP64)) != WD_OK) return bail(st);
    if ((st = alloc_field(c, &c->r64, SP64)) != WD_OK) return bail(st);
    if ((st = alloc_field(c, &c->eta64, SP64)) != WD_OK) return bail(st);
  }
  c->partials_len = (size_t)4 * (size_t)(4 * V / 32 + 64);
  if (cudaMalloc(&c->partials, sizeof(double) * c->partials_len) != cudaSuccess ||
      cudaMalloc(&c->sc, sizeof(CgScalars)) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(WD_ENOMEM, "cudaMalloc of the reduction workspace failed"));
  }
  if (cudaMallocHost(&c->sc_host, sizeof(CgScalars)) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(WD_ENOMEM, "pinned host allocation failed"));
  }
  memset(c->sc_host, 0, sizeof(CgScalars));
  if (cudaMemsetAsync(c->sc, 0, sizeof(CgScalars), c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bail(fail(WD_ECUDA, "workspace initialisation failed"));
  *out = c;
  return WD_OK;
}

void wd_destroy(wd_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  destroy_graph(c);
  free_field(&c->x);
  free_field(&c->r);
  free_field(&c->p);
  free_field(&c->q);
  free_field(&c->s);
  free_field(&c->eta);
  free_field(&c->x64);
  free_field(&c->r64);
  free_field(&c->eta64);
  if (c->gauge64) cudaFree(c->gauge64);
  if (c->gauge32) cudaFree(c->gauge32);
  if (c->staging) cudaFree(c->staging);
  if (c->partials) cudaFree(c->partials);
  if (c->sc) cudaFree(c->sc);
  if (c->sc_host) cudaFreeHost(c->sc_host);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->cap2) cudaStreamDestroy(c->cap2);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
}

wd_status wd_set_option(wd_ctx* c, int key, double value) {
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  switch (key) {
    case WD_OPT_RELIABLE_DELTA:
      if (!(value > 0.0 && value < 1.0)) return fail(WD_EINVAL, "reliable delta must be in (0, 1)");
      c->delta = value;
      return WD_OK;
    case WD_OPT_USE_GRAPH:
      c->use_graph = value != 0.0;
      return WD_OK;
    case WD_OPT_BLOCK_DSLASH:
    case WD_OPT_BLOCK_BLAS: {
      const int b = (int)value;
      if (value != (double)b || (b != 0 && (b < 32 || b > 1024 || b % 32))) return fail(WD_EINVAL, "block size must be 0 or a multiple of 32 in [32, 1024]");
      if (key == WD_OPT_BLOCK_DSLASH)
        c->block_dslash = b;
      else
        c->block_blas = b ? b : 256;
      destroy_graph(c);  // launch shapes are baked into the graph
      return WD_OK;
    }
    case WD_OPT_MAX_RESTARTS:
      if (!(value >= 0 && value <= 100)) return fail(WD_EINVAL, "max restarts must be in [0, 100]");
      c->max_restarts = (int)value;
      return WD_OK;
  }
  return fail(WD_EINVAL, "unknown option");
}

wd_status wd_get_stats(const wd_ctx* c, wd_stats* out) {
  if (!c || !out) return fail(WD_EINVAL, "null argument");
  *out = c->stats;
  return WD_OK;
}

wd_status wd_load_gauge(wd_ctx* c, const double* U, int on_device, int compress12, double* max_unitarity_dev) {
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  if (!U) return fail(WD_EINVAL, "U is null");
  const size_t bytes = (size_t)c->V * 4 * 9 * 16;
  const double* src = U;
  if (!on_device) {
    if (!c->staging && cudaMalloc(&c->staging, bytes) != cudaSuccess) {
      cudaGetLastError();
      c->staging = nullptr;
      return fail(WD_ENOMEM, "cudaMalloc of the gauge staging buffer failed");
    }
    if (cudaMemcpyAsync(c->staging, U, bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      return fail(WD_ECUDA, "host-to-device copy of the gauge field failed");
    src = (const double*)c->staging;
  }
  const bool need64 = c->wprec == SP64 || is_mixed(c->precision);
  const bool need32 = c->wprec != SP64;
  const int c12 = need32 && compress12 ? 1 : 0;
  auto cleanup = [&](wd_status s) { return s; };
  if (need64 && !c->gauge64) {
    if (cudaMalloc(&c->gauge64, (size_t)c->V * 4 * 9 * 16) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(fail(WD_ENOMEM, "cudaMalloc of the FP64 gauge field failed"));
    }
  }
  if (need32) {
    if (c->gauge32 && c->c12 != c12) {
      cudaFree(c->gauge32);
      c->gauge32 = nullptr;
    }
    if (!c->gauge32 && cudaMalloc(&c->gauge32, (size_t)c->V * 4 * (c12 ? 6 : 9) * 8) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(fail(WD_ENOMEM, "cudaMalloc of the FP32 gauge field failed"));
    }
    c->c12 = c12;
  }
  const int gb = 128;
  if (need64) {
    GaugePtr g;
    g.p = c->gauge64;
    g.prec = SP64;
    g.c12 = 0;
    if (launch_gauge_load(src, g, c->V, red_to(c, TK_GAUGE, &c->sc->max_dev), gb, c->stream) != cudaSuccess)
      return cleanup(fail(WD_ECUDA, "gauge load kernel failed to launch"));
  }
  if (need32) {
    GaugePtr g;
    g.p = c->gauge32;
    g.prec = SP32;
    g.c12 = c12;
    // the deviation is measured once (on the FP64 pass when there is one)
    Red r = need64 ? no_red() : red_to(c, TK_GAUGE, &c->sc->max_dev);
    if (launch_gauge_load(src, g, c->V, r, gb, c->stream) != cudaSuccess)
      return cleanup(fail(WD_ECUDA, "gauge load kernel failed to launch"));
  }
  if (cudaMemcpyAsync(c->sc_host, c->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return cleanup(fail(WD_ECUDA, std::string("gauge load failed: ") + cudaGetErrorString(cudaGetLastError())));
  cleanup(WD_OK);
  const double dev = c->sc_host->max_dev;
  if (max_unitarity_dev) *max_unitarity_dev = dev;
  c->gauge_loaded = true;
  if (!(dev < 1e300)) return fail(WD_ENOTUNITARY, "gauge field contains non-finite entries");
  if (c12 && dev > 1e-6) return fail(WD_ENOTUNITARY, "links are not SU(3) to 1e-6; 12-real storage would be wrong");
  return WD_OK;
}

wd_status wd_apply(wd_ctx* c, const void* in, void* out, int dagger) {
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  if (!in || !out) return fail(WD_EINVAL, "null field pointer");
  if (in == out) return fail(WD_EINVAL, "in and out must differ");
  if (!c->gauge_loaded) return fail(WD_ENOGAUGE, "wd_load_gauge has not been called");
  const int bb = c->block_blas;
  if (c->precision == WD_PREC_F32) {
    WD_CUDA(launch_pack_c64((const float*)in, c->q, c->V, bb, c->stream));
    WD_CUDA(dslash(c, c->q, c->s, dagger ? 1 : 0, EPI_PLAIN, none_field(), nullptr, 0, nullptr, c->stream));
    WD_CUDA(launch_unpack_c64(c->s, (float*)out, c->V, bb, c->stream));
  } else {
    FieldPtr a = c->wprec == SP64 ? c->q : c->x64;
    FieldPtr b = c->wprec == SP64 ? c->s : c->r64;
    WD_CUDA(launch_pack((const double*)in, a, c->V, no_red(), bb, c->stream));
    WD_CUDA(dslash(c, a, b, dagger ? 1 : 0, EPI_PLAIN, none_field(), nullptr, 0, nullptr, c->stream));
    WD_CUDA(launch_unpack(b, (double*)out, c->V, bb, c->stream));
  }
  WD_CUDA(cudaStreamSynchronize(c->stream));
  return WD_OK;
}

wd_status cg_solve(wd_ctx* c, const void* src, void* x, double tol, int maxit, int* iters, double* true_rel_res) {
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  if (!src || !x) return fail(WD_EINVAL, "null field pointer");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(WD_EINVAL, "tol must be a positive finite number");
  if (maxit < 0 || maxit > 10000000) return fail(WD_EINVAL, "maxit must be in [0, 10^7]");
  if (!c->gauge_loaded) return fail(WD_ENOGAUGE, "wd_load_gauge has not been called");
  const auto t0 = std::chrono::steady_clock::now();
  const bool mixed = is_mixed(c->precision);
  const int bb = c->block_blas;
  CgScalars* sc = c->sc;
  // inputs into the device layout: eta with ||eta||^2, x = initial guess
  FieldPtr eta = mixed ? c->eta64 : c->eta;
  FieldPtr xs = mixed ? c->x64 : c->x;
  set_params_kernel<<<1, 32, 0, c->stream>>>(sc, tol * tol, c->delta * c->delta, maxit, nullptr);
  WD_CUDA(cudaGetLastError());
  WD_CUDA(launch_pack((const double*)src, eta, c->V, red_to(c, TK_PACK, &sc->eta2), bb, c->stream));
  WD_CUDA(launch_pack((const double*)x, xs, c->V, no_red(), bb, c->stream));
  if (c->use_graph) {
    if ((st = build_graph(c)) != WD_OK) return st;
  }
  int restarts = 0;
  double rel = 0.0;
  int status = ST_RUNNING;
  for (;;) {
    if (c->use_graph) {
      WD_CUDA(cudaGraphLaunch(c->exec, c->stream));
      WD_CUDA(cudaStreamSynchronize(c->stream));
    } else {
      if ((st = run_host_loop(c)) != WD_OK) return st;
    }
    const CgScalars& h = *c->sc_host;
    status = h.status;
    rel = h.eta2 > 0.0 ? std::sqrt(h.rr_true / h.eta2) : std::sqrt(h.rr_true);
    if (!std::isfinite(h.eta2) || !std::isfinite(rel)) status = ST_BREAKDOWN;
    if (status == ST_BREAKDOWN || status == ST_MAXIT) break;
    if (rel <= tol) {
      status = ST_CONVERGED;
      break;
    }
    // recursive residual converged but the true one did not: restart from the true residual
    if (h.iter >= maxit || restarts >= c->max_restarts) {
      status = ST_MAXIT;
      break;
    }
    ++restarts;
  }
  WD_CUDA(launch_unpack(xs, (double*)x, c->V, bb, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  const CgScalars& h = *c->sc_host;
  const auto t1 = std::chrono::steady_clock::now();
  c->stats.iterations = h.iter;
  c->stats.restarts = restarts;
  c->stats.reliable_updates = h.updates;
  c->stats.true_rel_residual = rel;
  c->stats.solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  const int launches = restarts + 1;
  if (mixed) {
    c->stats.dslash_calls_f64 = 2 * launches + h.updates;
    c->stats.dslash_calls = c->stats.dslash_calls_f64 + launches + 2 * h.iter;
  } else {
    c->stats.dslash_calls = 3 * launches + 2 * h.iter;
    c->stats.dslash_calls_f64 = c->wprec == SP64 ? c->stats.dslash_calls : 0;
  }
  if (iters) *iters = h.iter;
  if (true_rel_res) *true_rel_res = rel;
  wd_status ret = WD_OK;
  if (status == ST_BREAKDOWN)
    ret = fail(WD_BREAKDOWN, "CG breakdown: non-finite or non-positive scalar (NaN/Inf in the source or links?)");
  else if (status != ST_CONVERGED)
    ret = fail(WD_NOT_CONVERGED, "maximum iterations reached before the true residual met tol");
  c->stats.status = ret;
  return ret;
}

wd_status wd_time_dslash(wd_ctx* c, int dagger, int launches, double* avg_ms) {
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  if (!avg_ms || launches <= 0) return fail(WD_EINVAL, "bad arguments");
  if (!c->gauge_loaded) return fail(WD_ENOGAUGE, "wd_load_gauge has not been called");
  // the solver's dominant dslash: the working precision one, with its fused norm
  FieldPtr in = c->p, out = c->q;
  WD_CUDA(dslash(c, in, out, dagger, EPI_PLAIN, none_field(), &c->sc->scratch[0], TK_MISC, nullptr, c->stream));
  WD_CUDA(cudaEventRecord(c->ev0, c->stream));
  for (int i = 0; i < launches; ++i)
    WD_CUDA(dslash(c, in, out, dagger, EPI_PLAIN, none_field(), &c->sc->scratch[0], TK_MISC, nullptr, c->stream));
  WD_CUDA(cudaEventRecord(c->ev1, c->stream));
  WD_CUDA(cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  WD_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  *avg_ms = (double)ms / launches;
  return WD_OK;
}

}  // extern "C"
