// C ABI of the Wilson-Dirac CG library: context management, gauge loading, operator application
// and the CG solvers (plain FP64/FP32 and mixed precision with reliable updates).
//
// The CG iteration runs as one CUDA graph per context: a prologue (r = eta - D x, p = D^dag r,
// convergence check), a device-side while node whose body is one CG iteration (the body's last
// kernel sets the loop condition, so the host never polls inside a solve), and an epilogue that
// recomputes the true residual. The host launches the graph, waits once, and relaunches only if
// the recomputed residual has not reached the tolerance (a restart from the true residual).
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

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
  int eo;     // fields stored in parity order; CG on the even-site Schur complement
  int nsolve; // sites the Krylov vectors span: V, or V/2 (even half) for even-odd
  FieldPtr t, t64;  // even-odd: odd-site temporaries of the two-step operator
  // mixed precision: reliable updates in double-float (FP32-pipe) arithmetic
  int use_df;
  int apply_df;  // wd_apply on a mixed context uses the double-float operator (for checks)
  int apply_inner;  // wd_apply / wd_apply_multi on a mixed context use the inner FP32 / FP16 operator
  FieldPtr xdf, rdf, etadf, tdf;
  void* gauge_df;
  FieldPtr x, r, p, q, s, eta;  // plain modes: all in wprec; mixed: r, p, q, s in wprec, x = x_lo (SP32)
  // FP64 operator and outer vectors (FP64 context and mixed modes)
  FieldPtr x64, r64, eta64;
  void* gauge64;
  void* gauge32;
  int c12;
  bool gauge_loaded;

  double* partials;
  size_t partials_len;
  double* loop_partials;   // persistent CG loop: 3 x kLoopMaxGrid block partials
  unsigned* loop_sync;     // persistent CG loop: barrier arrivals, generation, error flag
  long long loop_wait_limit;  // grid-barrier polls before a wait gives up (WD_OPT_LOOP_WAIT_LIMIT)
  double* hist_dev;        // recursive ||r||^2 per iteration (WD_OPT_RESIDUAL_HISTORY entries)
  int hist_cap;
  CgScalars* sc;
  CgScalars* sc_host;  // pinned

  // options
  double delta;
  int use_graph;  // 0 host loop, 1 CUDA graph, 2 persistent kernel (plain CGLS) else graph
  int block_dslash;
  int block_blas;
  int max_restarts;
  int cg_form;  // 0: CGLS on D^dag D; 1: the paper's CG on D D^dag, carried in x
  int time_basis;  // WD_OPT_LOOP_TIME_BASIS: persistent FP64 loop in the basis where gamma_t is diagonal

  // graph
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool graph_ready;

  wd_stats stats;
  cudaEvent_t ev0, ev1;
  void* staging;  // host gauge uploads (kept for reuse)

  // multiple right-hand sides (allocated on first use for mN right-hand sides)
  int mN;
  FieldPtr mx, mr, mp, mq, ms, meta;  // working precision (mixed: mx = x_lo in FP32, meta unused)
  FieldPtr mx64, mr64, meta64;        // FP64 (F64 context: unused; mixed: outer solution/residual)
  FieldPtr mxdf, mrdf, metadf;        // mixed with double-float updates: outer solution, residual, source
  MCgScalars* msc;
  MCgScalars* msc_host;
  double* mpartials;
  size_t mpartials_len;
  int mK, mspb, mgrid;        // tuned launch shape of the working-precision multi-RHS dslash
  int mKT;                    // ... and its right-hand sides per thread (1, 2 or 4)
  int mK64, mspb64, mgrid64;  // ... of the FP64 one (mixed modes)
  cudaGraph_t mgraph;
  cudaGraphExec_t mexec;
  bool mgraph_ready;
  int force_mK, force_mspb;   // launch shape fixed by options (0 = autotuned)
  int force_mKT;
  int tuned_block[4];         // autotuned single-RHS dslash block size per storage precision
  int tuned_var[4];           // ... and kernel variant (FP64: 1 = two threads per site)
  int force_var;              // WD_OPT_DSLASH_VARIANT: 0 tuned, else 1 + variant (FP64)
  int force_sched;            // WD_OPT_DSLASH_SCHEDULE: 0 tuned, else 1, 2 or 3 (FP32 / FP16 lexicographic)
  int loop_block, loop_var;   // launch shape of the persistent FP64 loop (timed on the loop itself)
  bool loop_tuned;
  FieldPtr p2, r2;            // second p and r buffers of the FP64 loop with 4, 8 or 16 lanes per site
  FieldPtr tl;                // FP64 loop in the time-diagonal basis: pre-scaled time links (in an FP64 field)
  int tma;                    // WD_OPT_DSLASH_TMA: stand-alone FP32 12-real operator staged by TMA (tile 1 or 2)
  bool resumable;             // x, r, p and the scalars hold a CG state stopped at maxit (wd_cg_save_state)
  bool standalone;            // the current operator call is wd_apply / wd_time_dslash (not a solve)
  wd_multi_stats mstats;
};

namespace {

size_t spinor_bytes(int prec, int V) {
  switch (prec) {
    case SP64: return (size_t)V * 12 * 16;
    case SP32: return (size_t)V * 12 * 8;
    case SP16: return (size_t)V * 12 * 4;
    case SPDF: return (size_t)V * 12 * 16;
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
  r.cap = (long long)c->partials_len;
  return r;
}

Red no_red() {
  Red r;
  r.partials = nullptr;
  r.ticket = nullptr;
  r.result = nullptr;
  r.cap = 0;
  return r;
}

int dslash_block(const wd_ctx* c, int prec) {
  if (c->block_dslash > 0) return c->block_dslash;
  if (prec >= 0 && prec < 4 && c->tuned_block[prec] > 0) return c->tuned_block[prec];
  return 256;
}

// FP64 single-RHS dslash: lanes per site 1, 2, 4, 8, 16 for variant 0..4
int dslash_variant(const wd_ctx* c, int prec) {
  if (prec != SP64) return 0;
  if (c->force_var) return c->force_var - 1;
  if (c->block_dslash > 0) return 0;
  return c->tuned_block[SP64] > 0 ? c->tuned_var[SP64] : 0;
}

// FP32 / FP16 single-RHS dslash on the lexicographic layout: load schedule 1 (hop by hop), 2 (two
// sites per thread, never tuned: slower wherever measured) or 3 (both hops of a direction loaded
// together; tuned variant 1 of that precision)
int dslash_sched(const wd_ctx* c, int prec) {
  if ((prec != SP32 && prec != SP16) || c->eo) return 1;
  if (c->force_sched) return c->force_sched;
  if (c->block_dslash > 0) return 1;
  return c->tuned_block[prec] > 0 && c->tuned_var[prec] == 1 ? 3 : 1;
}

GaugePtr gauge_for(const wd_ctx* c, int prec) {
  GaugePtr g;
  if (prec == SPDF) {
    g.p = c->gauge_df;
    g.prec = SPDF;
    g.c12 = 0;
  } else if (prec == SP64) {
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
  d.variant = dslash_variant(c, in.prec);
  d.schedule = dslash_sched(c, in.prec);
  d.kappa_dev = &c->sc->kappa;
  d.tma = 0;
  d.err = reinterpret_cast<int*>(c->loop_sync + 3);
  if (c->tma && c->standalone && in.prec == SP32 && c->c12 && epi == EPI_PLAIN && !skip) d.tma = c->tma;
  return launch_dslash(d, st);
}

// After a stand-alone operator call: did a TMA staging wait give up?
wd_status check_tma(wd_ctx* c) {
  if (!c->tma) return WD_OK;
  unsigned f = 0;
  WD_CUDA(cudaMemcpy(&f, c->loop_sync + 3, sizeof(f), cudaMemcpyDeviceToHost));
  if (f) {
    WD_CUDA(cudaMemset(c->loop_sync + 3, 0, sizeof(f)));
    WD_CUDA(cudaMemset(&c->sc->ticket[TK_MISC], 0, sizeof(unsigned)));
    return fail(WD_ECUDA, "TMA-staged dslash: a shared-memory staging wait gave up");
  }
  return WD_OK;
}

const GeomH* eo_geom(const wd_ctx* c) { return c->eo ? &c->geom : nullptr; }

// Even-odd half hopping: out = [b -] ([self] + sign * kappa * H in) on the sites of `parity`.
cudaError_t eo_half(wd_ctx* c, FieldPtr in, FieldPtr out, int parity, double sign, int dagger, const FieldPtr* self,
                    const FieldPtr* b, double* norm_dst, int slot, const int* skip, cudaStream_t st) {
  EoCall e;
  memset(&e, 0, sizeof(e));
  e.g = c->geom;
  e.u = gauge_for(c, in.prec);
  e.in = in;
  e.out = out;
  if (self) e.self = *self;
  if (b) e.b = *b;
  e.parity = parity;
  e.sign = sign;
  e.dagger = dagger;
  e.use_self = self != nullptr;
  e.resid = b != nullptr;
  e.kappa_dev = &c->sc->kappa;
  e.skip = skip;
  e.red = norm_dst ? red_to(c, slot, norm_dst) : no_red();
  e.block = dslash_block(c, in.prec);
  return launch_dslash_eo(e, st);
}

FieldPtr none_field();

// The solver's operator: A = D (lexicographic contexts) or A = M = 1 - kappa^2 H_eo H_oe on the even
// sites (even-odd contexts; two half launches through the odd temporary). out = A in, or
// out = b - A in for EPI_RESID; optional |out|^2 (over the sites the operator acts on).
cudaError_t op(wd_ctx* c, FieldPtr in, FieldPtr out, int dagger, int epi, FieldPtr b, double* norm_dst, int slot,
               const int* skip, cudaStream_t st) {
  if (!c->eo) return dslash(c, in, out, dagger, epi, b, norm_dst, slot, skip, st);
  cudaError_t e;
  FieldPtr t = in.prec == SP64 ? c->t64 : (in.prec == SPDF ? c->tdf : c->t);
  if ((e = eo_half(c, in, t, 1, +1.0, dagger, nullptr, nullptr, nullptr, 0, skip, st)) != cudaSuccess) return e;
  return eo_half(c, t, out, 0, -1.0, dagger, &in, epi == EPI_RESID ? &b : nullptr, norm_dst, slot, skip, st);
}

// out = D in (or D^dagger in) on the whole lattice, whatever the storage order.
cudaError_t full_D(wd_ctx* c, FieldPtr in, FieldPtr out, int dagger, cudaStream_t st) {
  if (!c->eo) return dslash(c, in, out, dagger, EPI_PLAIN, none_field(), nullptr, 0, nullptr, st);
  cudaError_t e;
  if ((e = eo_half(c, in, out, 0, -1.0, dagger, &in, nullptr, nullptr, 0, nullptr, st)) != cudaSuccess) return e;
  return eo_half(c, in, out, 1, -1.0, dagger, &in, nullptr, nullptr, 0, nullptr, st);
}

FieldPtr none_field() {
  FieldPtr f;
  f.p = nullptr;
  f.norm = nullptr;
  f.prec = -1;
  return f;
}

// ---------------------------------------------------------------- plain CG (one precision)

// dst = src (a whole field of the context's volume, norms included)
cudaError_t copy_field(const wd_ctx* c, FieldPtr src, FieldPtr dst, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(dst.p, src.p, spinor_bytes(src.prec, c->V), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess || src.prec != SP16) return e;
  return cudaMemcpyAsync(dst.norm, src.norm, sizeof(float) * (size_t)c->V, cudaMemcpyDeviceToDevice, st);
}

cudaError_t plain_prologue(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long cond) {
  cudaError_t e;
  CgScalars* sc = c->sc;
  if ((e = launch_cg_init(sc, 0, st)) != cudaSuccess) return e;
  // r = eta - D x
  if ((e = op(c, c->x, c->r, 0, EPI_RESID, c->eta, &sc->rr, TK_DSLASH_A, nullptr, st)) != cudaSuccess) return e;
  if (c->cg_form) {
    // the paper's form (CG on D D^dag y = eta, x = D^dag y): p = r, gamma = |r|^2
    if ((e = copy_field(c, c->r, c->p, st)) != cudaSuccess) return e;
    return launch_cg_check(sc, use_cond, cond, st, 1);
  }
  // p = D^dag r, gamma = |p|^2
  if ((e = op(c, c->r, c->p, 1, EPI_PLAIN, none_field(), &sc->gamma, TK_DSLASH_B, nullptr, st)) != cudaSuccess)
    return e;
  return launch_cg_check(sc, use_cond, cond, st);
}

// The paper's iteration (Sec. 2) with x = D^dag y carried directly: s = D^dag p; alpha =
// gamma / |s|^2; x += alpha s; r -= alpha D s; gamma' = |r|^2; p = r + (gamma' / gamma) p.
cudaError_t paper_body(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long cond) {
  cudaError_t e;
  CgScalars* sc = c->sc;
  const int bb = c->block_blas;
  // s = D^dag p, |s|^2 (in the slot the CGLS arrangement uses for |q|^2)
  if ((e = op(c, c->p, c->s, 1, EPI_PLAIN, none_field(), &sc->qq, TK_DSLASH_A, &sc->status, st)) != cudaSuccess)
    return e;
  // q = D s
  if ((e = op(c, c->s, c->q, 0, EPI_PLAIN, none_field(), nullptr, TK_DSLASH_B, &sc->status, st)) != cudaSuccess)
    return e;
  // alpha; r -= alpha q; gamma' = |r|^2
  if ((e = launch_cg_update_r(c->wprec, c->r, c->q, c->nsolve, c->V, sc, c->partials, bb, st, 1)) !=
      cudaSuccess)
    return e;
  // x += alpha s; p = r + beta p; loop condition
  return launch_cg_update_xp(c->wprec, c->x, c->s, c->p, c->r, c->nsolve, c->V, sc, c->partials, use_cond, cond, bb, st);
}

cudaError_t plain_body(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long cond) {
  if (c->cg_form) return paper_body(c, st, use_cond, cond);
  cudaError_t e;
  CgScalars* sc = c->sc;
  const int bb = c->block_blas;
  // q = D p, |q|^2
  if ((e = op(c, c->p, c->q, 0, EPI_PLAIN, none_field(), &sc->qq, TK_DSLASH_A, &sc->status, st)) != cudaSuccess)
    return e;
  // alpha; r -= alpha q; |r|^2
  if ((e = launch_cg_update_r(c->wprec, c->r, c->q, c->nsolve, c->V, sc, c->partials, bb, st)) != cudaSuccess) return e;
  // s = D^dag r, gamma' = |s|^2
  if ((e = op(c, c->r, c->s, 1, EPI_PLAIN, none_field(), &sc->gamma_new, TK_DSLASH_B, &sc->status, st)) !=
      cudaSuccess)
    return e;
  // x += alpha p; p = s + beta p; loop condition
  return launch_cg_update_xp(c->wprec, c->x, c->p, c->p, c->s, c->nsolve, c->V, sc, c->partials, use_cond, cond, bb, st);
}

cudaError_t plain_epilogue(wd_ctx* c, cudaStream_t st) {
  // true residual eta - D x into q (even-odd: b_e - M x_e, which equals the full residual once the
  // odd half is reconstructed below)
  cudaError_t e = op(c, c->x, c->q, 0, EPI_RESID, c->eta, &c->sc->rr_true, TK_DSLASH_C, nullptr, st);
  if (e != cudaSuccess || !c->eo) return e;
  // x_o = eta_o + kappa H_oe x_e
  return eo_half(c, c->x, c->x, 1, +1.0, 0, &c->eta, nullptr, nullptr, 0, nullptr, st);
}

// ---------------------------------------------------------------- mixed precision CG

// Reliable-update residual r_hi = eta - A x_hi, in double-float (FP32 pipes) or in FP64.
cudaError_t mixed_residual(wd_ctx* c, const int* skip, cudaStream_t st) {
  if (c->use_df) return op(c, c->xdf, c->rdf, 0, EPI_RESID, c->etadf, &c->sc->rr_true, TK_DSLASH_C, skip, st);
  return op(c, c->x64, c->r64, 0, EPI_RESID, c->eta64, &c->sc->rr_true, TK_DSLASH_C, skip, st);
}

cudaError_t mixed_accumulate(wd_ctx* c, const int* skip, cudaStream_t st) {
  if (c->use_df) return launch_mp_accumulate_df(c->xdf, c->x, c->nsolve, c->V, skip, c->block_blas, st);
  return launch_mp_accumulate(c->x64, c->x, c->nsolve, c->V, skip, c->block_blas, st);
}

cudaError_t mixed_convert(wd_ctx* c, int count, const int* skip, cudaStream_t st) {
  if (c->use_df)
    return launch_mp_convert_df(c->rdf, c->r, c->nsolve, c->V, c->sc, c->partials, count, skip, c->block_blas, st);
  return launch_mp_convert(c->r64, c->r, c->nsolve, c->V, c->sc, c->partials, count, skip, c->block_blas, st);
}

cudaError_t mixed_prologue(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long cond) {
  cudaError_t e;
  CgScalars* sc = c->sc;
  if ((e = launch_cg_init(sc, 0, st)) != cudaSuccess) return e;
  // r_hi = eta - A x_hi; x_lo = 0; r_lo = r_hi
  if ((e = mixed_residual(c, nullptr, st)) != cudaSuccess) return e;
  if ((e = launch_zero(c->x.p, spinor_bytes(c->x.prec, c->V), st)) != cudaSuccess) return e;
  if ((e = mixed_convert(c, 0, nullptr, st)) != cudaSuccess) return e;
  // p = A^dag r_lo
  if ((e = op(c, c->r, c->p, 1, EPI_PLAIN, none_field(), &sc->gamma, TK_DSLASH_B, nullptr, st)) != cudaSuccess)
    return e;
  return launch_cg_check(sc, use_cond, cond, st);
}

// reliable update: x_hi += x_lo; x_lo = 0; r_hi = eta - A x_hi; r_lo = r_hi
cudaError_t mixed_update(wd_ctx* c, cudaStream_t st) {
  cudaError_t e;
  if ((e = mixed_accumulate(c, nullptr, st)) != cudaSuccess) return e;
  if ((e = mixed_residual(c, nullptr, st)) != cudaSuccess) return e;
  return mixed_convert(c, 1, nullptr, st);
}

cudaError_t mixed_body_a(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long upd) {
  cudaError_t e;
  CgScalars* sc = c->sc;
  if ((e = op(c, c->p, c->q, 0, EPI_PLAIN, none_field(), &sc->qq, TK_DSLASH_A, &sc->status, st)) != cudaSuccess)
    return e;
  return launch_mp_update_rx(c->wprec, c->r, c->q, c->p, c->x, c->nsolve, c->V, sc, c->partials, use_cond, upd,
                             c->block_blas, st);
}

cudaError_t mixed_body_b(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long cond) {
  cudaError_t e;
  CgScalars* sc = c->sc;
  if ((e = op(c, c->r, c->s, 1, EPI_PLAIN, none_field(), &sc->gamma_new, TK_DSLASH_B, &sc->status, st)) !=
      cudaSuccess)
    return e;
  return launch_mp_update_p(c->wprec, c->p, c->s, c->nsolve, c->V, sc, c->partials, use_cond, cond, c->block_blas, st);
}

// Fold the last increment into the solution and recompute the true residual in native FP64
// (double-float solutions are converted first), then rebuild the odd sites for even-odd.
cudaError_t mixed_epilogue(wd_ctx* c, cudaStream_t st) {
  cudaError_t e;
  if ((e = mixed_accumulate(c, nullptr, st)) != cudaSuccess) return e;
  if (c->use_df && (e = launch_convert_f64_df(c->xdf, c->x64, c->V, c->V, 0, c->block_blas, st)) != cudaSuccess)
    return e;
  e = op(c, c->x64, c->r64, 0, EPI_RESID, c->eta64, &c->sc->rr_true, TK_DSLASH_C, nullptr, st);
  if (e != cudaSuccess || !c->eo) return e;
  return eo_half(c, c->x64, c->x64, 1, +1.0, 0, &c->eta64, nullptr, nullptr, 0, nullptr, st);
}

// reliable update with skip flags instead of a conditional node: each kernel checks the flag
cudaError_t mixed_update_flagged(wd_ctx* c, cudaStream_t st) {
  cudaError_t e;
  CgScalars* sc = c->sc;
  if ((e = mixed_accumulate(c, &sc->need_update, st)) != cudaSuccess) return e;
  if ((e = mixed_residual(c, &sc->no_update, st)) != cudaSuccess) return e;
  return mixed_convert(c, 1, &sc->need_update, st);
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
// The plain CGLS loop as one cooperative kernel between the usual prologue and epilogue.
// Volume up to which the persistent loop measured faster than the graph on GB300: plain FP64
// (14^4: 4 %; 16^4 and above: the graph, by 1-5 %) and mixed precision (8^4: 5-8 %, 14^4: 2-3 %;
// 24^3x48 and above: level or the graph). Plain FP32 was faster at every volume (8^4 to 32^4).
constexpr int kPersistentMaxSites = 48000;
// Plain FP64 on the lexicographic layout: up to 16^4, where the loop's launch shape is timed on the
// loop itself (the split of a site over 1 to 16 lanes included) and measured level with the graph or
// faster.
constexpr int kPersistentMaxSitesF64 = 65536;

bool persistent_loop(const wd_ctx* c) {
  // the paper's CG form has a persistent loop on the lexicographic layout (one thread per site)
  if ((c->cg_form && c->eo) || (c->eo && is_mixed(c->precision))) return false;
  if (c->use_graph == 2) return true;
  // even-odd (FP64 14^4: 4 %; FP64 24^4: the graph by 25 %) keeps to the volume limit in FP32 too
  const bool plain32 = !is_mixed(c->precision) && c->wprec == SP32 && !c->eo;
  const bool plain64 = c->precision == WD_PREC_F64 && !c->eo;
  return c->use_graph == 3 && (plain32 || c->V <= (plain64 ? kPersistentMaxSitesF64 : kPersistentMaxSites));
}

}  // namespace

namespace wdk {
// The operators whose default CG loop (WD_OPT_USE_GRAPH = 3) is the persistent kernel, which
// cg_solve_batch shares between problems (mirrors persistent_loop for a context with default options).
bool batch_capable(const int dims[4], int precision) {
  if (precision & WD_EVEN_ODD) return false;
  const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
  switch (precision) {
    case WD_PREC_F32: return true;
    case WD_PREC_F64: return V <= kPersistentMaxSitesF64;
    case WD_PREC_MIXED_F32:
    case WD_PREC_MIXED_F16: return V <= kPersistentMaxSites;
  }
  return false;
}
}  // namespace wdk

namespace {

// Shape of the persistent FP64 loop: options first, then the loop's own timing, else the dslash's.
int loop_block_of(const wd_ctx* c) {
  if (c->block_dslash > 0) return c->block_dslash;
  if (c->cg_form)  // one thread per site; where the dslash tuner split sites over lanes, spread them
    return c->wprec == SP64 && dslash_variant(c, SP64) != 0 ? 64 : dslash_block(c, c->wprec);
  return c->loop_tuned ? c->loop_block : dslash_block(c, c->wprec);
}
int loop_variant_of(const wd_ctx* c) {
  if (c->wprec != SP64 || c->eo || c->cg_form) return 0;  // the paper's loop: one thread per site
  if (c->force_var) return c->force_var - 1;
  return c->loop_tuned ? c->loop_var : dslash_variant(c, c->wprec);
}

// The lane loops alternate p and r between two buffers each.
wd_status ensure_lane_buffers(wd_ctx* c) {
  wd_status st;
  if (!c->p2.p && (st = alloc_field(c, &c->p2, SP64)) != WD_OK) return st;
  if (!c->r2.p && (st = alloc_field(c, &c->r2, SP64)) != WD_OK) return st;
  return WD_OK;
}

// Whether the plain FP64 loop of this launch shape runs in the time-diagonal basis.
bool loop_time_basis(const wd_ctx* c, int variant) {
  return !is_mixed(c->precision) && variant == 0 && c->wprec == SP64 && !c->eo && c->time_basis;
}

// The loop in the time-diagonal basis keeps its pre-scaled time links (9 of an FP64 field's 12
// complex components per site) in a buffer of the context, rewritten by every launch.
wd_status ensure_time_links(wd_ctx* c) {
  return c->tl.p ? WD_OK : alloc_field(c, &c->tl, SP64);
}

// resume: the context holds a restored CG state (x, r, p, gamma, |r|^2, iteration), so the pass
// starts without the prologue and only decides from the scalars whether the loop has work to do.
wd_status run_persistent(wd_ctx* c, double* loop_ms, bool resume = false) {
  const int variant = loop_variant_of(c);
  wd_status st;
  if (variant >= 2 && (st = ensure_lane_buffers(c)) != WD_OK) return st;
  if (loop_time_basis(c, variant) && (st = ensure_time_links(c)) != WD_OK) return st;
  WD_CUDA(resume ? launch_cg_check(c->sc, 0, 0, c->stream, 0) : plain_prologue(c, c->stream, 0, 0));
  CgLoopCall L;
  memset(&L, 0, sizeof(L));
  L.g = c->geom;
  L.u = gauge_for(c, c->wprec);
  L.x = c->x;
  L.r = c->r;
  L.p = c->p;
  L.q = c->q;
  L.s = c->s;
  L.kappa = c->kappa;
  L.kappa_dev = &c->sc->kappa;
  L.sc = c->sc;
  L.partials = c->loop_partials;
  L.bar = c->loop_sync;
  L.err = reinterpret_cast<int*>(c->loop_sync + 2);
  L.block = loop_block_of(c);
  L.max_grid = kLoopMaxGrid;
  L.wait_limit = c->loop_wait_limit;
  L.variant = variant;
  L.time_basis = loop_time_basis(c, variant) ? 1 : 0;
  L.cg_form = c->cg_form;
  L.t = c->t;
  L.p2 = c->p2;
  L.r2 = c->r2;
  L.tl = c->tl;
  WD_CUDA(cudaEventRecord(c->ev0, c->stream));
  WD_CUDA(c->eo ? launch_cg_eo_loop(L, c->stream) : launch_cg_loop(L, c->stream));
  WD_CUDA(cudaEventRecord(c->ev1, c->stream));
  WD_CUDA(plain_epilogue(c, c->stream));
  WD_CUDA(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  unsigned flags[4];
  WD_CUDA(cudaMemcpy(flags, c->loop_sync, sizeof(flags), cudaMemcpyDeviceToHost));
  if (flags[2] != 0) {
    WD_CUDA(cudaMemset(c->loop_sync, 0, sizeof(flags)));
    return fail(WD_ECUDA, "persistent CG loop: a grid barrier wait gave up");
  }
  float ms = 0.f;
  WD_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  *loop_ms += ms;
  return WD_OK;
}

// Mixed precision: the inner loop as a cooperative kernel that returns whenever a reliable update
// is due; the update runs as its separate kernels and the loop resumes in the same iteration.
wd_status run_mixed_persistent(wd_ctx* c, double* loop_ms) {
  WD_CUDA(mixed_prologue(c, c->stream, 0, 0));
  CgLoopCall L;
  memset(&L, 0, sizeof(L));
  L.g = c->geom;
  L.u = gauge_for(c, c->wprec);
  L.x = c->x;
  L.r = c->r;
  L.p = c->p;
  L.q = c->q;
  L.s = c->s;
  L.kappa = c->kappa;
  L.kappa_dev = &c->sc->kappa;
  L.sc = c->sc;
  L.partials = c->loop_partials;
  L.bar = c->loop_sync;
  L.err = reinterpret_cast<int*>(c->loop_sync + 2);
  L.block = dslash_block(c, c->wprec);
  L.max_grid = kLoopMaxGrid;
  L.wait_limit = c->loop_wait_limit;
  for (int launch = 0;; ++launch) {
    L.start_b = launch > 0;
    WD_CUDA(cudaEventRecord(c->ev0, c->stream));
    WD_CUDA(launch_cg_mixed_loop(L, c->stream));
    WD_CUDA(cudaEventRecord(c->ev1, c->stream));
    WD_CUDA(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
    WD_CUDA(cudaStreamSynchronize(c->stream));
    unsigned flags[4];
    WD_CUDA(cudaMemcpy(flags, c->loop_sync, sizeof(flags), cudaMemcpyDeviceToHost));
    if (flags[2] != 0) {
      WD_CUDA(cudaMemset(c->loop_sync, 0, sizeof(flags)));
      return fail(WD_ECUDA, "persistent CG loop: a grid barrier wait gave up");
    }
    float ms = 0.f;
    WD_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    *loop_ms += ms;
    if (!c->sc_host->need_update) break;  // converged, iteration limit or breakdown
    WD_CUDA(mixed_update(c, c->stream));
  }
  WD_CUDA(mixed_epilogue(c, c->stream));
  WD_CUDA(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  return WD_OK;
}

wd_status run_host_loop(wd_ctx* c, bool resume = false) {
  const bool mixed = is_mixed(c->precision);
  CgScalars* sc = c->sc;
  if (resume)  // plain precision only (see run_persistent)
    WD_CUDA(launch_cg_check(sc, 0, 0, c->stream, 0));
  else
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

__global__ void set_params_kernel(CgScalars* sc, double tol2, double delta2, int maxit, double* hist, int hist_len) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc->hist = hist;
    sc->hist_len = hist_len;
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

// Launch shapes chosen by timing are remembered for the life of the process, per device and
// problem shape. The block partials of the fused reductions follow the launch shape, so without
// this two contexts of the same problem (a served request and the same solve alone, say) could
// time their way to different shapes and differ in the last bits; with it they agree bitwise.
using TuneKey = std::array<int, 11>;  // device, kind, storage precision, L[4], eo, c12, nrhs, forced
std::mutex g_tune_mu;
std::map<TuneKey, std::array<int, 2>> g_tune;

TuneKey tune_key(const wd_ctx* c, int kind, int prec, int nrhs, int forced) {
  return TuneKey{c->device, kind, prec, c->dims[0], c->dims[1], c->dims[2], c->dims[3], c->eo, c->c12, nrhs, forced};
}

bool tune_lookup(const TuneKey& k, int* a, int* b) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *a = it->second[0];
  if (b) *b = it->second[1];
  return true;
}

// First writer wins: a context that tuned concurrently with another adopts the stored choice.
void tune_store(const TuneKey& k, int* a, int* b) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto ins = g_tune.emplace(k, std::array<int, 2>{*a, b ? *b : 0});
  *a = ins.first->second[0];
  if (b) *b = ins.first->second[1];
}

// The paper tunes the SYCL workgroup size per device (Sec. 3.1, Fig. 1); here the dslash block
// size is timed per problem shape and precision on first use (CUDA events, the context's own
// fields) and shared with later contexts of the same shape.
wd_status autotune_single(wd_ctx* c) {
  NvtxRange nvtx_("wd:autotune");
  if (c->block_dslash > 0) return WD_OK;
  const int precs[3] = {c->wprec, (is_mixed(c->precision) ? SP64 : -1), (c->use_df ? SPDF : -1)};
  for (int prec : precs) {
    if (prec < 0 || c->tuned_block[prec] > 0) continue;
    const TuneKey key = tune_key(c, 0, prec, 0, 0);
    if (tune_lookup(key, &c->tuned_block[prec], &c->tuned_var[prec])) continue;
    FieldPtr in = prec == c->wprec ? c->p : (prec == SPDF ? c->xdf : c->x64);
    FieldPtr out = prec == c->wprec ? c->q : (prec == SPDF ? c->rdf : c->r64);
    // (block, variant); FP64 on the lexicographic layout also tries two threads per site, and up to
    // 65,536 sites 4, 8 and 16 lanes per site (beyond that every SM sub-partition already holds
    // several warps of the one-thread kernel, which needs the fewest FP64 instructions per site)
    const int cands[15][2] = {{64, 0}, {128, 0}, {256, 0}, {64, 1}, {128, 1}, {256, 1}, {64, 2}, {128, 2},
                              {256, 2}, {64, 3}, {128, 3}, {256, 3}, {64, 4}, {128, 4}, {256, 4}};
    // FP32 / FP16 (lexicographic): variant 1 = both hops of each direction loaded together
    const bool sched = (prec == SP32 || prec == SP16) && !c->eo;
    const int nc = prec == SP64 && !c->eo ? (c->V <= 65536 ? 15 : 6) : (sched ? 6 : 3);
    const int saved_force = c->force_var, saved_sched = c->force_sched;
    c->force_var = 0;
    c->force_sched = 0;
    float best = 1e30f, plain = 1e30f;  // plain: the default shape, 256 threads, one per site
    int best_b = 256, best_v = 0;
    const int reps = prec == SP64 ? 2 : 4;
    for (int k = 0; k < nc; ++k) {
      c->tuned_block[prec] = cands[k][0];
      c->tuned_var[prec] = cands[k][1];
      WD_CUDA(op(c, in, out, 0, EPI_PLAIN, none_field(), &c->sc->scratch[1], TK_MISC, nullptr, c->stream));
      WD_CUDA(cudaEventRecord(c->ev0, c->stream));
      for (int i = 0; i < reps; ++i)
        WD_CUDA(op(c, in, out, 0, EPI_PLAIN, none_field(), &c->sc->scratch[1], TK_MISC, nullptr, c->stream));
      WD_CUDA(cudaEventRecord(c->ev1, c->stream));
      WD_CUDA(cudaEventSynchronize(c->ev1));
      float ms = 0.f;
      WD_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
      if (cands[k][0] == 256 && cands[k][1] == 0) plain = ms;
      if (ms < best) {
        best = ms;
        best_b = cands[k][0];
        best_v = cands[k][1];
      }
    }
    // another shape must beat the default by 3 %: timings within noise keep the default, so that
    // separate processes make the same choice
    if (plain <= best * 1.03f) {
      best_b = 256;
      best_v = 0;
    }
    c->force_var = saved_force;
    c->force_sched = saved_sched;
    tune_store(key, &best_b, &best_v);
    c->tuned_block[prec] = best_b;
    c->tuned_var[prec] = best_v;
  }
  return WD_OK;
}

// The persistent FP64 loop's launch shape (block, lanes per site), timed on the loop itself: a few
// iterations per candidate on the solve's own fields (tolerance 0, so none stops early), CUDA events
// around the loop kernel. The dslash timed alone ranks the candidates differently (at 12^4 the best
// stand-alone kernel made the loop 30 % slower), because the loop's vector phases and barriers
// follow the same grid. Remembered per problem shape like the other choices. The caller restores
// the solve's parameters and its initial guess afterwards.
constexpr int kLoopTuneIters = 6;

wd_status autotune_loop(wd_ctx* c, bool* ran) {
  NvtxRange nvtx_("wd:autotune_loop");
  *ran = false;
  if (c->loop_tuned || c->block_dslash > 0 || c->force_var) return WD_OK;
  const TuneKey key = tune_key(c, 2, SP64, 0, c->time_basis);  // the loop's kernels differ by basis
  int b = 0, v = 0;
  if (tune_lookup(key, &b, &v)) {
    c->loop_block = b;
    c->loop_var = v;
    c->loop_tuned = true;
    return WD_OK;
  }
  const int def_b = dslash_block(c, SP64), def_v = dslash_variant(c, SP64);
  const int nvar = c->V <= kPersistentMaxSitesF64 ? kMaxDslashVariant + 1 : 1;
  float best = 1e30f, dflt = 1e30f;
  int best_b = def_b, best_v = def_v;
  wd_status st;
  *ran = true;  // from here on the context's vectors and scalars are the tuner's
  for (int var = 0; var < nvar; ++var) {
    if (var >= 2 && (st = ensure_lane_buffers(c)) != WD_OK) return st;
    for (int blk = 64; blk <= 256; blk *= 2) {
      c->loop_block = blk;
      c->loop_var = var;
      c->loop_tuned = true;
      float t = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        set_params_kernel<<<1, 32, 0, c->stream>>>(c->sc, 0.0, c->delta * c->delta, kLoopTuneIters, nullptr, 0);
        WD_CUDA(cudaGetLastError());
        double ms = 0.0;
        if ((st = run_persistent(c, &ms)) != WD_OK) {
          c->loop_tuned = false;
          return st;
        }
        if (c->sc_host->iter != kLoopTuneIters) {  // a source the loop cannot iterate on (zero, say)
          c->loop_tuned = false;
          return WD_OK;
        }
        if ((float)ms < t) t = (float)ms;
      }
      if (blk == def_b && var == def_v) dflt = t;
      if (t < best) {
        best = t;
        best_b = blk;
        best_v = var;
      }
    }
  }
  // another shape must beat the stand-alone dslash's choice by 3 %, as in autotune_single
  if (dflt <= best * 1.03f) {
    best_b = def_b;
    best_v = def_v;
  }
  tune_store(key, &best_b, &best_v);
  c->loop_block = best_b;
  c->loop_var = best_v;
  c->loop_tuned = true;
  return WD_OK;
}

// ---------------------------------------------------------------- multiple right-hand sides

void free_multi(wd_ctx* c) {
  if (c->mexec) cudaGraphExecDestroy(c->mexec);
  if (c->mgraph) cudaGraphDestroy(c->mgraph);
  c->mexec = nullptr;
  c->mgraph = nullptr;
  c->mgraph_ready = false;
  FieldPtr* fs[] = {&c->mx,   &c->mr,   &c->mp,   &c->mq,   &c->ms,     &c->meta,
                    &c->mx64, &c->mr64, &c->meta64, &c->mxdf, &c->mrdf, &c->metadf};
  for (FieldPtr* f : fs) free_field(f);
  if (c->mpartials) cudaFree(c->mpartials);
  if (c->msc) cudaFree(c->msc);
  if (c->msc_host) cudaFreeHost(c->msc_host);
  c->mpartials = nullptr;
  c->msc = nullptr;
  c->msc_host = nullptr;
  c->mN = 0;
  c->mK = c->mK64 = 0;
}

wd_status alloc_mfield(wd_ctx* c, FieldPtr* f, int prec, int N) {
  f->prec = prec;
  f->norm = nullptr;
  f->p = nullptr;
  const size_t bytes = spinor_bytes(prec, c->V) * (size_t)N;
  if (cudaMalloc(&f->p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(WD_ENOMEM, "cudaMalloc of a multi-RHS field failed");
  }
  if (cudaMemsetAsync(f->p, 0, bytes, c->stream) != cudaSuccess) return fail(WD_ECUDA, "cudaMemsetAsync failed");
  if (prec == SP16) {
    if (cudaMalloc(&f->norm, sizeof(float) * (size_t)c->V * N) != cudaSuccess) {
      cudaGetLastError();
      return fail(WD_ENOMEM, "cudaMalloc of a multi-RHS norm field failed");
    }
    if (cudaMemsetAsync(f->norm, 0, sizeof(float) * (size_t)c->V * N, c->stream) != cudaSuccess)
      return fail(WD_ECUDA, "cudaMemsetAsync failed");
  }
  return WD_OK;
}

int mgrid_for(const wd_ctx* c, int spb) {
  const long long need = ((long long)c->V + spb - 1) / spb;
  long long cap = (long long)c->sms * 16;
  if (cap > kMaxMultiGrid) cap = kMaxMultiGrid;
  return (int)(need < cap ? need : cap);
}

wd_status ensure_multi(wd_ctx* c, int N) {
  if (c->mN == N) return WD_OK;
  free_multi(c);
  const bool mixed = is_mixed(c->precision);
  const int w = c->wprec;
  wd_status st;
  if ((st = alloc_mfield(c, &c->mx, mixed ? SP32 : w, N)) != WD_OK) return st;
  if ((st = alloc_mfield(c, &c->mr, w, N)) != WD_OK) return st;
  if ((st = alloc_mfield(c, &c->mp, w, N)) != WD_OK) return st;
  if ((st = alloc_mfield(c, &c->mq, w, N)) != WD_OK) return st;
  if ((st = alloc_mfield(c, &c->ms, w, N)) != WD_OK) return st;
  if (!mixed) {
    if ((st = alloc_mfield(c, &c->meta, w, N)) != WD_OK) return st;
  } else {
    if ((st = alloc_mfield(c, &c->mx64, SP64, N)) != WD_OK) return st;
    if ((st = alloc_mfield(c, &c->mr64, SP64, N)) != WD_OK) return st;
    if ((st = alloc_mfield(c, &c->meta64, SP64, N)) != WD_OK) return st;
    if (c->use_df) {
      if ((st = alloc_mfield(c, &c->mxdf, SPDF, N)) != WD_OK) return st;
      if ((st = alloc_mfield(c, &c->mrdf, SPDF, N)) != WD_OK) return st;
      if ((st = alloc_mfield(c, &c->metadf, SPDF, N)) != WD_OK) return st;
    }
  }
  // reduction workspace (block and run partials, run tickets that must start at zero)
  c->mpartials_len = kMultiPartials;
  if (cudaMalloc(&c->mpartials, sizeof(double) * c->mpartials_len) != cudaSuccess ||
      cudaMalloc(&c->msc, sizeof(MCgScalars)) != cudaSuccess) {
    cudaGetLastError();
    return fail(WD_ENOMEM, "cudaMalloc of the multi-RHS reduction workspace failed");
  }
  WD_CUDA(cudaMemsetAsync(c->mpartials, 0, sizeof(double) * c->mpartials_len, c->stream));
  if (cudaMallocHost(&c->msc_host, sizeof(MCgScalars)) != cudaSuccess) {
    cudaGetLastError();
    return fail(WD_ENOMEM, "pinned host allocation failed");
  }
  memset(c->msc_host, 0, sizeof(MCgScalars));
  c->msc_host->nrhs = N;
  WD_CUDA(cudaMemcpyAsync(c->msc, c->msc_host, sizeof(MCgScalars), cudaMemcpyHostToDevice, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  c->mN = N;
  return WD_OK;
}

MDslashCall mcall(wd_ctx* c, FieldPtr in, FieldPtr out, int dagger, int epi, FieldPtr b, double* result, int slot,
                  const int* status) {
  MDslashCall d;
  d.g = c->geom;
  d.u = gauge_for(c, in.prec);
  d.in = in;
  d.out = out;
  d.b = b;
  d.kappa = c->kappa;
  d.dagger = dagger;
  d.epi = epi;
  d.nrhs = c->mN;
  const bool f64 = (in.prec == SP64 || in.prec == SPDF) && c->wprec != SP64;
  d.group = f64 ? c->mK64 : c->mK;
  d.sites_per_block = f64 ? c->mspb64 : c->mspb;
  d.rhs_per_thread = f64 ? 1 : (c->mKT > 0 ? c->mKT : 1);
  d.grid_x = f64 ? c->mgrid64 : c->mgrid;
  d.status = status;
  d.partials = c->mpartials;
  d.tickets = &c->msc->ticket[slot];
  d.result = result;
  d.kappa_dev = &c->sc->kappa;
  return d;
}

cudaError_t mdslash(wd_ctx* c, FieldPtr in, FieldPtr out, int dagger, int epi, FieldPtr b, double* result, int slot,
                    const int* status, cudaStream_t st) {
  return launch_dslash_multi(mcall(c, in, out, dagger, epi, b, result, slot, status), st);
}

// Mean time of one multi-RHS dslash launch of shape (K, spb, KT) on the context's fields.
wd_status time_multi_shape(wd_ctx* c, FieldPtr in, FieldPtr out, int K, int spb, int kt, int reps, float* ms) {
  MDslashCall d = mcall(c, in, out, 0, EPI_PLAIN, none_field(), nullptr, TKM_MISC, nullptr);
  d.group = K;
  d.sites_per_block = spb;
  d.rhs_per_thread = kt;
  d.grid_x = mgrid_for(c, spb);
  WD_CUDA(launch_dslash_multi(d, c->stream));  // warm-up
  WD_CUDA(cudaEventRecord(c->ev0, c->stream));
  for (int i = 0; i < reps; ++i) WD_CUDA(launch_dslash_multi(d, c->stream));
  WD_CUDA(cudaEventRecord(c->ev1, c->stream));
  WD_CUDA(cudaEventSynchronize(c->ev1));
  WD_CUDA(cudaEventElapsedTime(ms, c->ev0, c->ev1));
  *ms /= reps;
  return WD_OK;
}

// Time candidate launch shapes of the multi-RHS dslash on the context's fields; keep the fastest
// (shared with later contexts of the same problem shape, like the single-RHS block size).
// Candidates: K (right-hand sides of a group sharing each link load) among the divisors of nrhs,
// sites per block, and for the FP32 / FP16 working precision KT = 1, 2 or 4 right-hand sides per
// thread (each thread loads and rebuilds a link once for KT of them). K * sites per block <= 256
// (the vector-update kernels run one thread per site and right-hand side on the same shape).
wd_status autotune_multi(wd_ctx* c, FieldPtr in, FieldPtr out, bool f64) {
  NvtxRange nvtx_("wd:autotune_multi");
  const int N = c->mN;
  int bestK = N, bestS = 256 / N, bestT = 1;
  float best = 1e30f;
  const int fixK = c->force_mK, fixS = c->force_mspb, fixT = f64 ? 1 : c->force_mKT;
  const int reps = f64 ? 1 : 3;
  wd_status st;
  const TuneKey key = tune_key(c, 1, in.prec, N, (fixT * 1024 + fixK) * 1024 + fixS);
  int packed = 0;  // sites per block | KT << 16 in the shape cache
  if (tune_lookup(key, &bestK, &packed)) {
    bestS = packed & 0xffff;
    bestT = packed >> 16;
    if (!f64 && (st = time_multi_shape(c, in, out, bestK, bestS, bestT, reps, &best)) != WD_OK) return st;
  } else {
    const bool blocked = !f64 && (in.prec == SP32 || in.prec == SP16);
    for (int K = 1; K <= N; ++K) {
      if (N % K) continue;
      if (fixK && K != fixK) continue;
      const int spbs[] = {4, 8, 16, 32, 64, 128};
      for (int spb : spbs) {
        if (fixS && spb != fixS) continue;
        const int block = K * spb;
        if (block > 256 || block < 64) continue;
        for (int kt = 1; kt <= 4; kt *= 2) {
          if (fixT && kt != fixT) continue;
          if (kt > 1 && (!blocked || K % kt || spb < kt)) continue;
          float ms = 0.f;
          if ((st = time_multi_shape(c, in, out, K, spb, kt, reps, &ms)) != WD_OK) return st;
          if (ms < best) {
            best = ms;
            bestK = K;
            bestS = spb;
            bestT = kt;
          }
        }
      }
    }
    if (best >= 1e29f) return fail(WD_EINVAL, "no valid multi-RHS launch shape for this nrhs and options");
    packed = bestS | (bestT << 16);
    tune_store(key, &bestK, &packed);
    bestS = packed & 0xffff;
    bestT = packed >> 16;
  }
  if (f64) {
    c->mK64 = bestK;
    c->mspb64 = bestS;
    c->mgrid64 = mgrid_for(c, bestS);
  } else {
    c->mK = bestK;
    c->mspb = bestS;
    c->mKT = bestT;
    c->mgrid = mgrid_for(c, bestS);
    c->mstats.dslash_ms = best;
  }
  return WD_OK;
}

wd_status ensure_multi_tuned(wd_ctx* c) {
  wd_status st;
  if (!c->mK) {
    if ((st = autotune_multi(c, c->mp, c->mq, false)) != WD_OK) return st;
  }
  if (is_mixed(c->precision) && !c->mK64) {
    const bool df = c->use_df && c->mxdf.p;
    if ((st = autotune_multi(c, df ? c->mxdf : c->mx64, df ? c->mrdf : c->mr64, true)) != WD_OK) return st;
  }
  c->mstats.group = c->mK;
  c->mstats.sites_per_block = c->mspb;
  c->mstats.rhs_per_thread = c->mKT;
  return WD_OK;
}

cudaError_t mplain_prologue(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long cond) {
  cudaError_t e;
  MCgScalars* sc = c->msc;
  if ((e = launch_mcg_init(sc, st)) != cudaSuccess) return e;
  if ((e = mdslash(c, c->mx, c->mr, 0, EPI_RESID, c->meta, sc->rr, TKM_DSLASH_A, nullptr, st)) != cudaSuccess) return e;
  if ((e = mdslash(c, c->mr, c->mp, 1, EPI_PLAIN, none_field(), sc->gamma, TKM_DSLASH_B, nullptr, st)) != cudaSuccess)
    return e;
  return launch_mcg_check(sc, use_cond, cond, st);
}

cudaError_t mplain_body(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long cond) {
  cudaError_t e;
  MCgScalars* sc = c->msc;
  if ((e = mdslash(c, c->mp, c->mq, 0, EPI_PLAIN, none_field(), sc->qq, TKM_DSLASH_A, sc->status, st)) != cudaSuccess)
    return e;
  if ((e = launch_mcg_update_r(c->wprec, c->mr, c->mq, c->mp, c->mx, c->V, sc, c->mpartials, c->mN, c->mK, c->mspb,
                               c->mgrid, 0, 0, 0, st)) != cudaSuccess)
    return e;
  if ((e = mdslash(c, c->mr, c->ms, 1, EPI_PLAIN, none_field(), sc->gamma_new, TKM_DSLASH_B, sc->status, st)) !=
      cudaSuccess)
    return e;
  return launch_mcg_update_xp(c->wprec, c->mx, c->mp, c->ms, c->V, sc, c->mpartials, c->mN, c->mK, c->mspb, c->mgrid,
                              0, use_cond, cond, st);
}

cudaError_t mplain_epilogue(wd_ctx* c, cudaStream_t st) {
  return mdslash(c, c->mx, c->mq, 0, EPI_RESID, c->meta, c->msc->rr_true, TKM_DSLASH_C, nullptr, st);
}

bool mdf(const wd_ctx* c) { return c->use_df && c->mxdf.p != nullptr; }

cudaError_t mmixed_update(wd_ctx* c, cudaStream_t st) {
  cudaError_t e;
  MCgScalars* sc = c->msc;
  if (mdf(c)) {
    if ((e = launch_macc_df(c->mxdf, c->mx, c->V, c->mN, c->mgrid, st)) != cudaSuccess) return e;
    if ((e = mdslash(c, c->mxdf, c->mrdf, 0, EPI_RESID, c->metadf, sc->rr_true, TKM_DSLASH_C, sc->status, st)) !=
        cudaSuccess)
      return e;
    return launch_mconv_df(c->mrdf, c->mr, c->V, c->mN, c->mgrid, sc, 1, st);
  }
  if ((e = launch_macc(c->mx64, c->mx, c->V, c->mN, c->mgrid, st)) != cudaSuccess) return e;
  if ((e = mdslash(c, c->mx64, c->mr64, 0, EPI_RESID, c->meta64, sc->rr_true, TKM_DSLASH_C, sc->status, st)) !=
      cudaSuccess)
    return e;
  return launch_mconv(c->mr64, c->mr, c->V, c->mN, c->mgrid, sc, 1, st);
}

cudaError_t mmixed_prologue(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long cond) {
  cudaError_t e;
  MCgScalars* sc = c->msc;
  if ((e = launch_mcg_init(sc, st)) != cudaSuccess) return e;
  if (mdf(c)) {
    if ((e = mdslash(c, c->mxdf, c->mrdf, 0, EPI_RESID, c->metadf, sc->rr_true, TKM_DSLASH_C, nullptr, st)) !=
        cudaSuccess)
      return e;
  } else if ((e = mdslash(c, c->mx64, c->mr64, 0, EPI_RESID, c->meta64, sc->rr_true, TKM_DSLASH_C, nullptr, st)) !=
             cudaSuccess) {
    return e;
  }
  if ((e = launch_zero(c->mx.p, spinor_bytes(SP32, c->V) * (size_t)c->mN, st)) != cudaSuccess) return e;
  if (mdf(c)) {
    if ((e = launch_mconv_df(c->mrdf, c->mr, c->V, c->mN, c->mgrid, sc, 0, st)) != cudaSuccess) return e;
  } else if ((e = launch_mconv(c->mr64, c->mr, c->V, c->mN, c->mgrid, sc, 0, st)) != cudaSuccess) {
    return e;
  }
  if ((e = mdslash(c, c->mr, c->mp, 1, EPI_PLAIN, none_field(), sc->gamma, TKM_DSLASH_B, nullptr, st)) != cudaSuccess)
    return e;
  return launch_mcg_check(sc, use_cond, cond, st);
}

cudaError_t mmixed_body_a(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long upd) {
  cudaError_t e;
  MCgScalars* sc = c->msc;
  if ((e = mdslash(c, c->mp, c->mq, 0, EPI_PLAIN, none_field(), sc->qq, TKM_DSLASH_A, sc->status, st)) != cudaSuccess)
    return e;
  return launch_mcg_update_r(c->wprec, c->mr, c->mq, c->mp, c->mx, c->V, sc, c->mpartials, c->mN, c->mK, c->mspb,
                             c->mgrid, 1, use_cond, upd, st);
}

cudaError_t mmixed_body_b(wd_ctx* c, cudaStream_t st, int use_cond, unsigned long long cond) {
  cudaError_t e;
  MCgScalars* sc = c->msc;
  if ((e = mdslash(c, c->mr, c->ms, 1, EPI_PLAIN, none_field(), sc->gamma_new, TKM_DSLASH_B, sc->status, st)) !=
      cudaSuccess)
    return e;
  return launch_mcg_update_xp(c->wprec, c->mx, c->mp, c->ms, c->V, sc, c->mpartials, c->mN, c->mK, c->mspb, c->mgrid,
                              1, use_cond, cond, st);
}

cudaError_t mmixed_epilogue(wd_ctx* c, cudaStream_t st) {
  cudaError_t e;
  if (mdf(c)) {
    if ((e = launch_macc_df(c->mxdf, c->mx, c->V, c->mN, c->mgrid, st)) != cudaSuccess) return e;
    if ((e = launch_mconvert_df(c->mx64, c->mxdf, c->V, c->mN, c->mgrid, 0, st)) != cudaSuccess) return e;
  } else if ((e = launch_macc(c->mx64, c->mx, c->V, c->mN, c->mgrid, st)) != cudaSuccess) {
    return e;
  }
  return mdslash(c, c->mx64, c->mr64, 0, EPI_RESID, c->meta64, c->msc->rr_true, TKM_DSLASH_C, nullptr, st);
}

wd_status build_mgraph(wd_ctx* c) {
  if (c->mgraph_ready) return WD_OK;
  const bool mixed = is_mixed(c->precision);
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
  WD_CUDA(cudaGraphCreate(&c->mgraph, 0));
  cudaGraphConditionalHandle loop_h;
  WD_CUDA(cudaGraphConditionalHandleCreate(&loop_h, c->mgraph, 0, cudaGraphCondAssignDefault));
  cudaGraph_t loop_body = nullptr;
  wd_status st;
  WD_CUDA(cudaStreamBeginCaptureToGraph(c->cap, c->mgraph, nullptr, nullptr, 0, mode));
  if ((st = cap_check(mixed ? mmixed_prologue(c, c->cap, 1, loop_h) : mplain_prologue(c, c->cap, 1, loop_h),
                      "multi prologue")) != WD_OK)
    return st;
  if ((st = add_conditional(c->cap, loop_h, cudaGraphCondTypeWhile, &loop_body)) != WD_OK) return st;
  if ((st = cap_check(mixed ? mmixed_epilogue(c, c->cap) : mplain_epilogue(c, c->cap), "multi epilogue")) != WD_OK)
    return st;
  WD_CUDA(cudaMemcpyAsync(c->msc_host, c->msc, sizeof(MCgScalars), cudaMemcpyDeviceToHost, c->cap));
  cudaGraph_t g = nullptr;
  WD_CUDA(cudaStreamEndCapture(c->cap, &g));
  WD_CUDA(cudaStreamBeginCaptureToGraph(c->cap2, loop_body, nullptr, nullptr, 0, mode));
  if (!mixed) {
    if ((st = cap_check(mplain_body(c, c->cap2, 1, loop_h), "multi body")) != WD_OK) return st;
  } else {
    cudaGraphConditionalHandle upd_h;
    WD_CUDA(cudaGraphConditionalHandleCreate(&upd_h, loop_body, 0, cudaGraphCondAssignDefault));
    if ((st = cap_check(mmixed_body_a(c, c->cap2, 1, upd_h), "multi body a")) != WD_OK) return st;
    cudaGraph_t upd_body = nullptr;
    if ((st = add_conditional(c->cap2, upd_h, cudaGraphCondTypeIf, &upd_body)) != WD_OK) return st;
    if ((st = cap_check(mmixed_body_b(c, c->cap2, 1, loop_h), "multi body b")) != WD_OK) return st;
    cudaGraph_t lb = nullptr;
    WD_CUDA(cudaStreamEndCapture(c->cap2, &lb));
    WD_CUDA(cudaStreamBeginCaptureToGraph(c->cap2, upd_body, nullptr, nullptr, 0, mode));
    if ((st = cap_check(mmixed_update(c, c->cap2), "multi update")) != WD_OK) return st;
  }
  cudaGraph_t bg = nullptr;
  WD_CUDA(cudaStreamEndCapture(c->cap2, &bg));
  WD_CUDA(cudaGraphInstantiate(&c->mexec, c->mgraph, 0));
  c->mgraph_ready = true;
  return WD_OK;
}

wd_status run_mhost_loop(wd_ctx* c) {
  const bool mixed = is_mixed(c->precision);
  MCgScalars* sc = c->msc;
  WD_CUDA(mixed ? mmixed_prologue(c, c->stream, 0, 0) : mplain_prologue(c, c->stream, 0, 0));
  for (;;) {
    WD_CUDA(cudaMemcpyAsync(c->msc_host, sc, sizeof(MCgScalars), cudaMemcpyDeviceToHost, c->stream));
    WD_CUDA(cudaStreamSynchronize(c->stream));
    if (!c->msc_host->any_running) break;
    if (!mixed) {
      WD_CUDA(mplain_body(c, c->stream, 0, 0));
      continue;
    }
    WD_CUDA(mmixed_body_a(c, c->stream, 0, 0));
    WD_CUDA(cudaMemcpyAsync(c->msc_host, sc, sizeof(MCgScalars), cudaMemcpyDeviceToHost, c->stream));
    WD_CUDA(cudaStreamSynchronize(c->stream));
    if (c->msc_host->need_update) WD_CUDA(mmixed_update(c, c->stream));
    WD_CUDA(mmixed_body_b(c, c->stream, 0, 0));
  }
  WD_CUDA(mixed ? mmixed_epilogue(c, c->stream) : mplain_epilogue(c, c->stream));
  WD_CUDA(cudaMemcpyAsync(c->msc_host, sc, sizeof(MCgScalars), cudaMemcpyDeviceToHost, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  return WD_OK;
}

__global__ void mset_params_kernel(MCgScalars* sc, double tol2, double delta2, int maxit) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc->tol2 = tol2;
    sc->delta2 = delta2;
    sc->maxit = maxit;
    sc->iter = 0;
    sc->updates = 0;
    sc->any_running = 0;
    for (int i = 0; i < kMaxRhs; ++i) {
      sc->iters[i] = 0;
      sc->status[i] = ST_RUNNING;
    }
    for (int i = 0; i < 128; ++i) sc->ticket[i] = 0u;
  }
}

// Allocate the gauge copies the context's solver needs; returns the 12-real flag in effect.
wd_status ensure_gauge_buffers(wd_ctx* c, int compress12, bool* need64, bool* need32, int* c12_out) {
  *need64 = c->wprec == SP64 || is_mixed(c->precision);
  *need32 = c->wprec != SP64;
  const int c12 = *need32 && compress12 ? 1 : 0;
  // graphs hold the gauge pointers and the 12-real flag: rebuild them after any change
  if ((*need64 && !c->gauge64) || (*need32 && (!c->gauge32 || c->c12 != c12))) {
    destroy_graph(c);
    if (c->mexec) cudaGraphExecDestroy(c->mexec);
    if (c->mgraph) cudaGraphDestroy(c->mgraph);
    c->mexec = nullptr;
    c->mgraph = nullptr;
    c->mgraph_ready = false;
    c->tuned_block[0] = c->tuned_block[1] = c->tuned_block[2] = c->tuned_block[3] = 0;
    c->mK = c->mK64 = 0;
  }
  if (is_mixed(c->precision) && c->use_df && !c->gauge_df) {
    destroy_graph(c);
    if (cudaMalloc(&c->gauge_df, (size_t)c->V * 4 * 9 * 16) != cudaSuccess) {
      cudaGetLastError();
      c->gauge_df = nullptr;
      return fail(WD_ENOMEM, "cudaMalloc of the double-float gauge field failed");
    }
  }
  if (*need64 && !c->gauge64) {
    if (cudaMalloc(&c->gauge64, (size_t)c->V * 4 * 9 * 16) != cudaSuccess) {
      cudaGetLastError();
      return fail(WD_ENOMEM, "cudaMalloc of the FP64 gauge field failed");
    }
  }
  if (*need32) {
    if (c->gauge32 && c->c12 != c12) {
      cudaFree(c->gauge32);
      c->gauge32 = nullptr;
    }
    if (!c->gauge32 && cudaMalloc(&c->gauge32, (size_t)c->V * 4 * (c12 ? 6 : 9) * 8) != cudaSuccess) {
      cudaGetLastError();
      c->gauge32 = nullptr;
      return fail(WD_ENOMEM, "cudaMalloc of the FP32 gauge field failed");
    }
    c->c12 = c12;
  }
  *c12_out = c12;
  return WD_OK;
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
  const int eo = (precision & WD_EVEN_ODD) ? 1 : 0;
  precision &= ~WD_EVEN_ODD;
  if (eo) {
    for (int i = 0; i < 4; ++i)
      if (dims[i] % 2) return fail(WD_EINVAL, "even-odd preconditioning needs every extent even");
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
  c->eo = eo;
  c->nsolve = eo ? (int)(V / 2) : (int)V;
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
  c->delta = 0.1;  // a reliable update each time |r| has dropped 10x
  c->use_graph = 3;
  c->loop_wait_limit = kLoopWaitLimit;
  c->time_basis = 1;
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
  if (mixed) {
    c->use_df = 1;
    if ((st = alloc_field(c, &c->xdf, SPDF)) != WD_OK) return bail(st);
    if ((st = alloc_field(c, &c->rdf, SPDF)) != WD_OK) return bail(st);
    if ((st = alloc_field(c, &c->etadf, SPDF)) != WD_OK) return bail(st);
    if (eo && (st = alloc_field(c, &c->tdf, SPDF)) != WD_OK) return bail(st);
  }
  if (eo) {
    if ((st = alloc_field(c, &c->t, wprec)) != WD_OK) return bail(st);
    if (mixed && (st = alloc_field(c, &c->t64, SP64)) != WD_OK) return bail(st);
    if (wprec == SP64) c->t64 = c->t;
  }
  // the largest grid of any reduction: the FP64 dslash with 16 lanes per site at 32 threads per
  // block (V / 2 blocks); the vector kernels need at most 12 V / 32, the gauge load 4 V / 128
  c->partials_len = (size_t)(V / 2 + 64);
  if (cudaMalloc(&c->partials, sizeof(double) * c->partials_len) != cudaSuccess ||
      cudaMalloc(&c->sc, sizeof(CgScalars)) != cudaSuccess ||
      cudaMalloc(&c->loop_partials, sizeof(double) * 3 * kLoopMaxGrid) != cudaSuccess ||
      cudaMalloc(&c->loop_sync, 4 * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(WD_ENOMEM, "cudaMalloc of the reduction workspace failed"));
  }
  if (cudaMemsetAsync(c->loop_sync, 0, 4 * sizeof(unsigned), c->stream) != cudaSuccess)
    return bail(fail(WD_ECUDA, "cudaMemsetAsync failed"));
  if (cudaMallocHost(&c->sc_host, sizeof(CgScalars)) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(WD_ENOMEM, "pinned host allocation failed"));
  }
  memset(c->sc_host, 0, sizeof(CgScalars));
  c->sc_host->kappa = kappa;
  if (cudaMemcpyAsync(c->sc, c->sc_host, sizeof(CgScalars), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bail(fail(WD_ECUDA, "workspace initialisation failed"));
  *out = c;
  return WD_OK;
}

void wd_destroy(wd_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  destroy_graph(c);
  free_multi(c);
  free_field(&c->x);
  free_field(&c->r);
  free_field(&c->p);
  free_field(&c->q);
  free_field(&c->s);
  free_field(&c->eta);
  free_field(&c->x64);
  free_field(&c->r64);
  free_field(&c->eta64);
  if (c->t64.p == c->t.p) c->t64.p = nullptr;
  free_field(&c->t);
  free_field(&c->t64);
  free_field(&c->xdf);
  free_field(&c->rdf);
  free_field(&c->etadf);
  free_field(&c->tdf);
  free_field(&c->p2);
  free_field(&c->tl);
  free_field(&c->r2);
  if (c->gauge_df) cudaFree(c->gauge_df);
  if (c->gauge64) cudaFree(c->gauge64);
  if (c->gauge32) cudaFree(c->gauge32);
  if (c->staging) cudaFree(c->staging);
  if (c->partials) cudaFree(c->partials);
  if (c->loop_partials) cudaFree(c->loop_partials);
  if (c->hist_dev) cudaFree(c->hist_dev);
  if (c->loop_sync) cudaFree(c->loop_sync);
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
      if (!(value == 0.0 || value == 1.0 || value == 2.0 || value == 3.0))
        return fail(WD_EINVAL, "loop option must be 0, 1, 2 or 3");
      c->use_graph = (int)value;
      return WD_OK;
    case WD_OPT_BLOCK_DSLASH:
    case WD_OPT_BLOCK_BLAS: {
      const int b = (int)value;
      const int bmax = key == WD_OPT_BLOCK_DSLASH ? 256 : 1024;
      if (value != (double)b || (b != 0 && (b < 32 || b > bmax || b % 32)))
        return fail(WD_EINVAL, "block size must be 0 or a multiple of 32 in [32, 256] (dslash) / [32, 1024] (BLAS)");
      if (key == WD_OPT_BLOCK_DSLASH) {
        c->block_dslash = b;
        c->tuned_block[0] = c->tuned_block[1] = c->tuned_block[2] = c->tuned_block[3] = 0;
        c->loop_tuned = false;
      } else
        c->block_blas = b ? b : 256;
      destroy_graph(c);  // launch shapes are baked into the graph
      return WD_OK;
    }
    case WD_OPT_MULTI_GROUP:
    case WD_OPT_MULTI_SITES:
    case WD_OPT_MULTI_RHS_PER_THREAD: {
      const int v = (int)value;
      if (value != (double)v || v < 0 || v > 256) return fail(WD_EINVAL, "multi-RHS shape option out of range");
      if (key == WD_OPT_MULTI_RHS_PER_THREAD && !(v == 0 || v == 1 || v == 2 || v == 4))
        return fail(WD_EINVAL, "right-hand sides per thread must be 0 (tuned), 1, 2 or 4");
      if (key == WD_OPT_MULTI_GROUP)
        c->force_mK = v;
      else if (key == WD_OPT_MULTI_SITES)
        c->force_mspb = v;
      else
        c->force_mKT = v;
      c->mK = c->mK64 = 0;  // re-tune (or apply the forced shape) on next use
      if (c->mexec) cudaGraphExecDestroy(c->mexec);
      if (c->mgraph) cudaGraphDestroy(c->mgraph);
      c->mexec = nullptr;
      c->mgraph = nullptr;
      c->mgraph_ready = false;
      return WD_OK;
    }
    case WD_OPT_DF_UPDATES: {
      if (!is_mixed(c->precision)) return fail(WD_EINVAL, "double-float updates apply to mixed-precision contexts");
      const int v = value != 0.0;
      if (v && (!c->xdf.p || !c->rdf.p || !c->etadf.p)) return fail(WD_EINVAL, "context has no double-float workspace");
      if (v != c->use_df) {
        c->use_df = v;
        destroy_graph(c);
        free_multi(c);  // multi-RHS workspace is rebuilt with the matching fields on next use
        if (v && c->gauge_loaded && !c->gauge_df) c->gauge_loaded = false;  // needs a reload
      }
      return WD_OK;
    }
    case WD_OPT_APPLY_DF:
      if (!is_mixed(c->precision)) return fail(WD_EINVAL, "double-float operator exists on mixed-precision contexts");
      c->apply_df = value != 0.0;
      return WD_OK;
    case WD_OPT_DSLASH_SCHEDULE: {
      const int v = (int)value;
      if (value != (double)v || v < 0 || v > 3) return fail(WD_EINVAL, "dslash schedule must be 0, 1, 2 or 3");
      if (v >= 2 && (c->wprec == SP64 || c->eo))
        return fail(WD_EINVAL, "load schedules 2 and 3 serve the FP32 / FP16 operator on the lexicographic layout");
      c->force_sched = v;
      destroy_graph(c);
      return WD_OK;
    }
    case WD_OPT_DSLASH_TMA: {
      const int v = (int)value;
      if (value != (double)v || v < 0 || v > 2) return fail(WD_EINVAL, "TMA option must be 0, 1 or 2");
      if (v && (c->wprec != SP32 || c->eo)) return fail(WD_EINVAL, "TMA staging serves the FP32 operator on the lexicographic layout");
      if (v && !tma_dslash_supported(c->geom, v - 1))
        return fail(WD_EINVAL, "TMA staging needs Lx a multiple of 4 up to 64 and Ly, Lz, Lt divisible by the tile");
      c->tma = v;
      return WD_OK;
    }
    case WD_OPT_LOOP_TIME_BASIS:
      if (value != 0.0 && value != 1.0) return fail(WD_EINVAL, "time-basis option must be 0 or 1");
      c->time_basis = (int)value;
      c->loop_tuned = false;  // the loop's launch shape is timed on the kernel it runs
      return WD_OK;
    case WD_OPT_APPLY_INNER:
      if (!is_mixed(c->precision)) return fail(WD_EINVAL, "the inner operator exists on mixed-precision contexts");
      if (value != 0.0 && value != 1.0) return fail(WD_EINVAL, "apply-inner option must be 0 or 1");
      c->apply_inner = value != 0.0;
      return WD_OK;
    case WD_OPT_DSLASH_VARIANT: {
      const int v = (int)value;
      if (value != (double)v || v < 0 || v > kMaxDslashVariant + 1)
        return fail(WD_EINVAL, "dslash variant must be in 0..5");
      if (v >= 2 && !(c->precision == WD_PREC_F64 || is_mixed(c->precision)))
        return fail(WD_EINVAL, "several threads per site is an FP64 dslash variant");
      c->force_var = v;
      c->loop_tuned = false;
      destroy_graph(c);
      return WD_OK;
    }
    case WD_OPT_RESIDUAL_HISTORY: {
      const int n = (int)value;
      if (value != (double)n || n < 0 || n > 10000000) return fail(WD_EINVAL, "history length must be in [0, 10^7]");
      if (n != c->hist_cap) {
        if (c->hist_dev) cudaFree(c->hist_dev);
        c->hist_dev = nullptr;
        c->hist_cap = 0;
        if (n > 0) {
          if (cudaMalloc(&c->hist_dev, sizeof(double) * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            return fail(WD_ENOMEM, "cudaMalloc of the residual history failed");
          }
          c->hist_cap = n;
        }
        destroy_graph(c);  // the graph's parameter kernel holds the history pointer
      }
      return WD_OK;
    }
    case WD_OPT_LOOP_WAIT_LIMIT: {
      if (!(value >= 0.0 && value <= (double)kLoopWaitLimit) || value != std::floor(value))
        return fail(WD_EINVAL, "loop wait limit must be an integer in [0, 2^26]");
      c->loop_wait_limit = value == 0.0 ? kLoopWaitLimit : (long long)value;
      return WD_OK;
    }
    case WD_OPT_CG_FORM: {
      const int v = (int)value;
      if (value != (double)v || v < 0 || v > 1) return fail(WD_EINVAL, "CG form must be 0 or 1");
      if (v && is_mixed(c->precision))
        return fail(WD_EINVAL, "the paper's CG form is available on plain FP64 / FP32 contexts");
      if (v != c->cg_form) {
        c->cg_form = v;
        destroy_graph(c);
      }
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
  NvtxRange nvtx_("wd:load_gauge");
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  c->resumable = false;  // the Krylov fields or the operator change
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
  bool need64 = false, need32 = false;
  int c12 = 0;
  if ((st = ensure_gauge_buffers(c, compress12, &need64, &need32, &c12)) != WD_OK) return st;
  const int gb = 128;
  if (need64) {
    GaugePtr g;
    g.p = c->gauge64;
    g.prec = SP64;
    g.c12 = 0;
    if (launch_gauge_load(src, g, c->V, eo_geom(c), red_to(c, TK_GAUGE, &c->sc->max_dev), gb, c->stream) != cudaSuccess)
      return fail(WD_ECUDA, "gauge load kernel failed to launch");
  }
  if (c->gauge_df) {
    GaugePtr g;
    g.p = c->gauge_df;
    g.prec = SPDF;
    g.c12 = 0;
    if (launch_gauge_load(src, g, c->V, eo_geom(c), no_red(), gb, c->stream) != cudaSuccess)
      return fail(WD_ECUDA, "gauge load kernel failed to launch");
  }
  if (need32) {
    GaugePtr g;
    g.p = c->gauge32;
    g.prec = SP32;
    g.c12 = c12;
    // the deviation is measured once (on the FP64 pass when there is one)
    Red r = need64 ? no_red() : red_to(c, TK_GAUGE, &c->sc->max_dev);
    if (launch_gauge_load(src, g, c->V, eo_geom(c), r, gb, c->stream) != cudaSuccess)
      return fail(WD_ECUDA, "gauge load kernel failed to launch");
  }
  if (cudaMemcpyAsync(c->sc_host, c->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(WD_ECUDA, std::string("gauge load failed: ") + cudaGetErrorString(cudaGetLastError()));
  const double dev = c->sc_host->max_dev;
  if (max_unitarity_dev) *max_unitarity_dev = dev;
  c->gauge_loaded = true;
  if (!(dev < 1e300)) return fail(WD_ENOTUNITARY, "gauge field contains non-finite entries");
  if (c12 && dev > 1e-6) return fail(WD_ENOTUNITARY, "links are not SU(3) to 1e-6; 12-real storage would be wrong");
  return WD_OK;
}

wd_status wd_apply(wd_ctx* c, const void* in, void* out, int dagger) {
  NvtxRange nvtx_("wd:apply");
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  c->resumable = false;  // the Krylov fields or the operator change
  if (!in || !out) return fail(WD_EINVAL, "null field pointer");
  if (in == out) return fail(WD_EINVAL, "in and out must differ");
  if (!c->gauge_loaded) return fail(WD_ENOGAUGE, "wd_load_gauge has not been called");
  if ((st = autotune_single(c)) != WD_OK) return st;
  const int bb = c->block_blas;
  struct Standalone {
    wd_ctx* c;
    ~Standalone() { c->standalone = false; }
  } standalone_{c};
  c->standalone = true;
  if (c->precision == WD_PREC_F32) {
    WD_CUDA(launch_pack_c64((const float*)in, c->q, c->V, eo_geom(c), bb, c->stream));
    WD_CUDA(full_D(c, c->q, c->s, dagger ? 1 : 0, c->stream));
    WD_CUDA(launch_unpack_c64(c->s, (float*)out, c->V, eo_geom(c), bb, c->stream));
  } else if (c->apply_inner) {
    // the inner solver's operator: complex128 rounded into the working precision (FP32, or FP16
    // with its per-site norm), the dslash on the FP32 links, the result widened back
    WD_CUDA(launch_pack((const double*)in, c->p, c->V, eo_geom(c), no_red(), bb, c->stream));
    WD_CUDA(full_D(c, c->p, c->q, dagger ? 1 : 0, c->stream));
    WD_CUDA(launch_unpack(c->q, (double*)out, c->V, eo_geom(c), bb, c->stream));
  } else {
    FieldPtr a = c->wprec == SP64 ? c->q : c->x64;
    FieldPtr b = c->wprec == SP64 ? c->s : c->r64;
    WD_CUDA(launch_pack((const double*)in, a, c->V, eo_geom(c), no_red(), bb, c->stream));
    if (c->apply_df && c->gauge_df) {
      WD_CUDA(launch_convert_f64_df(a, c->xdf, c->V, c->V, 1, bb, c->stream));
      WD_CUDA(full_D(c, c->xdf, c->rdf, dagger ? 1 : 0, c->stream));
      WD_CUDA(launch_convert_f64_df(c->rdf, b, c->V, c->V, 0, bb, c->stream));
    } else {
      WD_CUDA(full_D(c, a, b, dagger ? 1 : 0, c->stream));
    }
    WD_CUDA(launch_unpack(b, (double*)out, c->V, eo_geom(c), bb, c->stream));
  }
  WD_CUDA(cudaStreamSynchronize(c->stream));
  return check_tma(c);
}

}  // extern "C"

// Saved CG state (wd_cg_save_state / cg_resume): this header, then x, r and p in the context's
// device layout (each spinor_bytes(working precision, V) bytes), copied byte for byte.
struct CgStateHeader {
  char magic[8];  // "WDCGST1"
  int dims[4];
  int bc[4];
  int precision;
  int iter;       // iterations done
  double kappa;
  double gamma;   // |D^dag r|^2 of the current direction p
  double rr;      // recursive |r|^2
  unsigned long long field_bytes;
};
constexpr char kStateMagic[8] = {'W', 'D', 'C', 'G', 'S', 'T', '1', 0};

__global__ void set_state_kernel(CgScalars* sc, int iter, double gamma, double rr) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc->iter = iter;
    sc->gamma = gamma;
    sc->rr = rr;
    sc->status = ST_RUNNING;
  }
}

namespace {

// One solve's progress, shared by cg_solve and cg_solve_batch.
struct Solve {
  const void* src;
  void* x;
  const unsigned char* state;  // cg_resume: the saved state (header, then x, r, p); null for cg_solve
  bool resume_pass;            // the next pass continues the restored state (no prologue)
  double tol;
  int maxit;
  bool persistent;
  bool done;
  int status;
  int restarts;
  double rel;
  double loop_ms;
  std::chrono::steady_clock::time_point t0;
};

// Checks, the inputs into the device layout (eta with ||eta||^2, x = initial guess), launch-shape
// tuning and the graph.
wd_status solve_begin(wd_ctx* c, Solve& v) {
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  if (!v.src || !v.x) return fail(WD_EINVAL, "null field pointer");
  if (!(v.tol > 0.0) || !std::isfinite(v.tol)) return fail(WD_EINVAL, "tol must be a positive finite number");
  if (v.maxit < 0 || v.maxit > 10000000) return fail(WD_EINVAL, "maxit must be in [0, 10^7]");
  if (!c->gauge_loaded) return fail(WD_ENOGAUGE, "wd_load_gauge has not been called");
  c->resumable = false;
  v.t0 = std::chrono::steady_clock::now();
  v.done = false;
  v.resume_pass = false;
  v.status = ST_RUNNING;
  v.restarts = 0;
  v.rel = 0.0;
  v.loop_ms = 0.0;
  const bool mixed = is_mixed(c->precision);
  const int bb = c->block_blas;
  CgScalars* sc = c->sc;
  FieldPtr eta = mixed ? c->eta64 : c->eta;
  FieldPtr xs = mixed ? c->x64 : c->x;
  set_params_kernel<<<1, 32, 0, c->stream>>>(sc, v.tol * v.tol, c->delta * c->delta, v.maxit, c->hist_dev, c->hist_cap);
  WD_CUDA(cudaGetLastError());
  WD_CUDA(launch_pack((const double*)v.src, eta, c->V, eo_geom(c), red_to(c, TK_PACK, &sc->eta2), bb, c->stream));
  const size_t fb = spinor_bytes(c->wprec, c->V);
  const unsigned char* saved = v.state ? v.state + sizeof(CgStateHeader) : nullptr;  // x, r, p
  if (saved)
    WD_CUDA(cudaMemcpyAsync(xs.p, saved, fb, cudaMemcpyHostToDevice, c->stream));
  else
    WD_CUDA(launch_pack((const double*)v.x, xs, c->V, eo_geom(c), no_red(), bb, c->stream));
  if (c->eo) {
    // Schur source on the even sites, in place: b_e = eta_e + kappa H_eo eta_o (eta_o is kept for
    // the reconstruction x_o = eta_o + kappa H_oe x_e)
    WD_CUDA(eo_half(c, eta, eta, 0, +1.0, 0, &eta, nullptr, nullptr, 0, nullptr, c->stream));
  }
  if (mixed && c->use_df) {
    WD_CUDA(launch_convert_f64_df(c->eta64, c->etadf, c->V, c->V, 1, bb, c->stream));
    WD_CUDA(launch_convert_f64_df(c->x64, c->xdf, c->V, c->V, 1, bb, c->stream));
  }
  if ((st = autotune_single(c)) != WD_OK) return st;
  v.persistent = persistent_loop(c);
  if (v.persistent && c->precision == WD_PREC_F64 && !c->eo && !c->cg_form) {
    bool ran = false;
    if ((st = autotune_loop(c, &ran)) != WD_OK) return st;
    if (ran) {  // the tuner iterated on this solve's fields: restore its parameters and initial guess
      set_params_kernel<<<1, 32, 0, c->stream>>>(sc, v.tol * v.tol, c->delta * c->delta, v.maxit, c->hist_dev,
                                                 c->hist_cap);
      WD_CUDA(cudaGetLastError());
      if (saved)
        WD_CUDA(cudaMemcpyAsync(xs.p, saved, fb, cudaMemcpyHostToDevice, c->stream));
      else
        WD_CUDA(launch_pack((const double*)v.x, xs, c->V, eo_geom(c), no_red(), bb, c->stream));
    }
  }
  if (c->use_graph && !v.persistent) {
    if ((st = build_graph(c)) != WD_OK) return st;
  }
  if (saved) {  // the rest of the saved state, after any tuning that iterated on the context's fields
    const CgStateHeader* h = reinterpret_cast<const CgStateHeader*>(v.state);
    WD_CUDA(cudaMemcpyAsync(c->r.p, saved + fb, fb, cudaMemcpyHostToDevice, c->stream));
    WD_CUDA(cudaMemcpyAsync(c->p.p, saved + 2 * fb, fb, cudaMemcpyHostToDevice, c->stream));
    set_state_kernel<<<1, 32, 0, c->stream>>>(sc, h->iter, h->gamma, h->rr);
    WD_CUDA(cudaGetLastError());
    WD_CUDA(cudaStreamSynchronize(c->stream));  // the caller's host buffer may be reused on return
    v.resume_pass = true;
  }
  return WD_OK;
}

// After a pass (the scalars are in sc_host): converged, out of iterations, broken down, or a restart
// from the true residual.
void solve_judge(wd_ctx* c, Solve& v) {
  const CgScalars& h = *c->sc_host;
  int status = h.status;
  v.rel = h.eta2 > 0.0 ? std::sqrt(h.rr_true / h.eta2) : std::sqrt(h.rr_true);
  if (!std::isfinite(h.eta2) || !std::isfinite(v.rel)) status = ST_BREAKDOWN;
  v.done = true;
  if (status == ST_BREAKDOWN || status == ST_MAXIT) {
    v.status = status;
  } else if (v.rel <= v.tol) {
    v.status = ST_CONVERGED;
  } else if (h.iter >= v.maxit || v.restarts >= c->max_restarts) {
    // recursive residual converged but the true one did not, and no restart is left
    v.status = ST_MAXIT;
  } else {
    ++v.restarts;  // restart from the true residual
    v.done = false;
  }
}

wd_status solve_pass(wd_ctx* c, Solve& v) {
  wd_status st;
  const bool resume = v.resume_pass;  // plain precision only; the graph holds the prologue, so a
  v.resume_pass = false;              // resumed first pass runs its kernels from the host
  if (v.persistent) {
    if ((st = is_mixed(c->precision) ? run_mixed_persistent(c, &v.loop_ms) : run_persistent(c, &v.loop_ms, resume)) !=
        WD_OK)
      return st;
  } else if (c->use_graph && !resume) {
    WD_CUDA(cudaGraphLaunch(c->exec, c->stream));
    WD_CUDA(cudaStreamSynchronize(c->stream));
  } else {
    if ((st = run_host_loop(c, resume)) != WD_OK) return st;
  }
  solve_judge(c, v);
  return WD_OK;
}

// The solution back to the caller's layout, statistics, the status.
wd_status solve_end(wd_ctx* c, Solve& v, int* iters, double* true_rel_res) {
  const bool mixed = is_mixed(c->precision);
  FieldPtr xs = mixed ? c->x64 : c->x;
  WD_CUDA(launch_unpack(xs, (double*)v.x, c->V, eo_geom(c), c->block_blas, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  const CgScalars& h = *c->sc_host;
  const auto t1 = std::chrono::steady_clock::now();
  // a plain CG loop that stopped at maxit leaves x, r, p and the scalars ready for the next iteration
  c->resumable = !mixed && v.status == ST_MAXIT && h.status == ST_MAXIT;
  c->stats.iterations = h.iter;
  c->stats.restarts = v.restarts;
  c->stats.loop_mode = v.persistent ? 2 : (c->use_graph ? 1 : 0);
  c->stats.loop_lanes = v.persistent ? lanes_of_variant(loop_variant_of(c)) : 0;
  c->stats.loop_ms = v.loop_ms;
  c->stats.reliable_updates = h.updates;
  c->stats.true_rel_residual = v.rel;
  c->stats.solve_ms = std::chrono::duration<double, std::milli>(t1 - v.t0).count();
  const int launches = v.restarts + 1;
  if (mixed) {
    c->stats.dslash_calls_f64 = 2 * launches + h.updates;
    c->stats.dslash_calls = c->stats.dslash_calls_f64 + launches + 2 * h.iter;
  } else {
    c->stats.dslash_calls = 3 * launches + 2 * h.iter;
    c->stats.dslash_calls_f64 = c->wprec == SP64 ? c->stats.dslash_calls : 0;
  }
  if (iters) *iters = h.iter;
  if (true_rel_res) *true_rel_res = v.rel;
  wd_status ret = WD_OK;
  if (v.status == ST_BREAKDOWN)
    ret = fail(WD_BREAKDOWN, "CG breakdown: non-finite or non-positive scalar (NaN/Inf in the source or links?)");
  else if (v.status != ST_CONVERGED)
    ret = fail(WD_NOT_CONVERGED, "maximum iterations reached before the true residual met tol");
  c->stats.status = ret;
  return ret;
}

// ---------------------------------------------------------------- batched solves
//
// Several contexts of one problem shape (lattice, boundary, precision, launch shape) whose CG loop
// is the persistent kernel: each pass runs their prologues, ONE cooperative launch of the loop for
// all of them (each problem on its own blocks, with its own barrier counter, scalars and fields,
// and the grid it has alone), then their epilogues. Every problem thus computes exactly what its
// solve alone computes, in the same order. Launches that cannot keep all blocks resident are split.

CgLoopCall loop_call(wd_ctx* c, int start_b) {
  CgLoopCall L;
  memset(&L, 0, sizeof(L));
  L.g = c->geom;
  L.u = gauge_for(c, c->wprec);
  L.x = c->x;
  L.r = c->r;
  L.p = c->p;
  L.q = c->q;
  L.s = c->s;
  L.kappa = c->kappa;
  L.kappa_dev = &c->sc->kappa;
  L.sc = c->sc;
  L.partials = c->loop_partials;
  L.bar = c->loop_sync;
  L.err = reinterpret_cast<int*>(c->loop_sync + 2);
  L.block = is_mixed(c->precision) ? dslash_block(c, c->wprec) : loop_block_of(c);
  L.max_grid = kLoopMaxGrid;
  L.wait_limit = c->loop_wait_limit;
  L.variant = is_mixed(c->precision) ? 0 : loop_variant_of(c);
  L.time_basis = loop_time_basis(c, L.variant) ? 1 : 0;
  L.cg_form = c->cg_form;
  L.t = c->t;
  L.p2 = c->p2;
  L.r2 = c->r2;
  L.tl = c->tl;
  L.start_b = start_b;
  return L;
}

// Launch the loops of calls[0 .. n), in batches of at most kMaxBatch, halving any batch whose blocks
// cannot all be resident.
cudaError_t launch_loops(const CgLoopCall* calls, int n, bool mixed, cudaStream_t st) {
  for (int i = 0; i < n;) {
    int m = std::min(n - i, kMaxBatch);
    for (;;) {
      cudaError_t e = mixed ? launch_cg_mixed_loop_n(calls + i, m, st) : launch_cg_loop_n(calls + i, m, st);
      if (e == cudaErrorCooperativeLaunchTooLarge && m > 1) {
        cudaGetLastError();
        m = (m + 1) / 2;
        continue;
      }
      if (e != cudaSuccess) return e;
      break;
    }
    i += m;
  }
  return cudaSuccess;
}

wd_status check_loop_errors(wd_ctx* const* cs, int n) {
  bool failed = false;
  for (int i = 0; i < n; ++i) {
    unsigned flags[4];
    WD_CUDA(cudaMemcpy(flags, cs[i]->loop_sync, sizeof(flags), cudaMemcpyDeviceToHost));
    if (flags[2] != 0) {
      WD_CUDA(cudaMemset(cs[i]->loop_sync, 0, sizeof(flags)));
      failed = true;
    }
  }
  if (failed) return fail(WD_ECUDA, "persistent CG loop: a grid barrier wait gave up");
  return WD_OK;
}

// One pass over the contexts cs[0 .. n) (all persistent, same shape) on stream st.
wd_status batch_pass(wd_ctx* const* cs, int n, cudaStream_t st, double* loop_ms) {
  const bool mixed = is_mixed(cs[0]->precision);
  wd_status r;
  std::vector<CgLoopCall> calls(n);
  for (int i = 0; i < n; ++i) {
    wd_ctx* c = cs[i];
    if (!mixed && loop_variant_of(c) >= 2 && (r = ensure_lane_buffers(c)) != WD_OK) return r;
    if (loop_time_basis(c, loop_variant_of(c)) && (r = ensure_time_links(c)) != WD_OK) return r;
    WD_CUDA(mixed ? mixed_prologue(c, st, 0, 0) : plain_prologue(c, st, 0, 0));
    calls[i] = loop_call(c, 0);
  }
  cudaEvent_t e0 = cs[0]->ev0, e1 = cs[0]->ev1;
  std::vector<wd_ctx*> active(cs, cs + n);
  for (int launch = 0; !active.empty(); ++launch) {
    std::vector<CgLoopCall> now;
    for (wd_ctx* c : active) now.push_back(loop_call(c, launch > 0));
    WD_CUDA(cudaEventRecord(e0, st));
    WD_CUDA(launch_loops(now.data(), (int)now.size(), mixed, st));
    WD_CUDA(cudaEventRecord(e1, st));
    for (wd_ctx* c : active) WD_CUDA(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    WD_CUDA(cudaStreamSynchronize(st));
    if ((r = check_loop_errors(active.data(), (int)active.size())) != WD_OK) return r;
    float ms = 0.f;
    WD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    *loop_ms += ms;
    if (!mixed) break;
    // mixed precision: the problems whose reliable update is due get it and resume together
    std::vector<wd_ctx*> next;
    for (wd_ctx* c : active)
      if (c->sc_host->need_update) {
        WD_CUDA(mixed_update(c, st));
        next.push_back(c);
      }
    active.swap(next);
  }
  for (int i = 0; i < n; ++i) {
    wd_ctx* c = cs[i];
    WD_CUDA(mixed ? mixed_epilogue(c, st) : plain_epilogue(c, st));
    WD_CUDA(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
  }
  WD_CUDA(cudaStreamSynchronize(st));
  return WD_OK;
}

// Contexts that can share loop launches: persistent loop on the lexicographic layout (mixed
// precision) or any layout the plain loop serves, identical problem shape and launch shape.
bool batchable(wd_ctx* const* cs, const Solve* vs, int n) {
  const wd_ctx* a = cs[0];
  if (!vs[0].persistent || a->eo || a->cg_form) return false;
  for (int i = 1; i < n; ++i) {
    const wd_ctx* b = cs[i];
    if (!vs[i].persistent || b->eo || b->cg_form || b->precision != a->precision || b->c12 != a->c12 ||
        memcmp(&b->geom, &a->geom, sizeof(GeomH)) != 0 || b->use_df != a->use_df ||
        dslash_block(b, b->wprec) != dslash_block(a, a->wprec) || loop_block_of(b) != loop_block_of(a) ||
        loop_variant_of(b) != loop_variant_of(a) || b->device != a->device)
      return false;
  }
  return true;
}

}  // namespace

extern "C" {

wd_status cg_solve(wd_ctx* c, const void* src, void* x, double tol, int maxit, int* iters, double* true_rel_res) {
  NvtxRange nvtx_("wd:cg_solve");
  Solve v;
  v.src = src;
  v.x = x;
  v.state = nullptr;
  v.tol = tol;
  v.maxit = maxit;
  wd_status st;
  if ((st = solve_begin(c, v)) != WD_OK) return st;
  while (!v.done)
    if ((st = solve_pass(c, v)) != WD_OK) return st;
  return solve_end(c, v, iters, true_rel_res);
}

wd_status wd_cg_state_size(const wd_ctx* c, size_t* bytes) {
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  if (!bytes) return fail(WD_EINVAL, "bytes is null");
  if (is_mixed(c->precision)) return fail(WD_EINVAL, "CG states are saved for plain FP64 or FP32 contexts only");
  *bytes = sizeof(CgStateHeader) + 3 * spinor_bytes(c->wprec, c->V);
  return WD_OK;
}

wd_status wd_cg_save_state(wd_ctx* c, void* host, size_t bytes) {
  NvtxRange nvtx_("wd:cg_save_state");
  wd_status st;
  size_t need = 0;
  if ((st = wd_cg_state_size(c, &need)) != WD_OK) return st;
  if (!host) return fail(WD_EINVAL, "host buffer is null");
  if (bytes < need) return fail(WD_EINVAL, "host buffer smaller than wd_cg_state_size");
  if (!c->resumable)
    return fail(WD_EINVAL, "no resumable CG state: the last solve on this context did not stop at maxit, or a "
                           "later call changed its fields or operator");
  CgStateHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kStateMagic, sizeof(h.magic));
  memcpy(h.dims, c->dims, sizeof(h.dims));
  memcpy(h.bc, c->bc, sizeof(h.bc));
  h.precision = c->precision;
  h.iter = c->sc_host->iter;
  h.kappa = c->kappa;
  h.gamma = c->sc_host->gamma;
  h.rr = c->sc_host->rr;
  h.field_bytes = spinor_bytes(c->wprec, c->V);
  unsigned char* out = static_cast<unsigned char*>(host);
  memcpy(out, &h, sizeof(h));
  const FieldPtr* fs[3] = {&c->x, &c->r, &c->p};
  for (int i = 0; i < 3; ++i)
    WD_CUDA(cudaMemcpyAsync(out + sizeof(h) + i * h.field_bytes, fs[i]->p, h.field_bytes, cudaMemcpyDeviceToHost,
                            c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  return WD_OK;
}

wd_status cg_resume(wd_ctx* c, const void* state, size_t bytes, const void* src, void* x, double tol, int maxit,
                    int* iters, double* true_rel_res) {
  NvtxRange nvtx_("wd:cg_resume");
  wd_status st;
  size_t need = 0;
  if ((st = wd_cg_state_size(c, &need)) != WD_OK) return st;
  if (!state || bytes < need) return fail(WD_EINVAL, "state is null or smaller than wd_cg_state_size");
  CgStateHeader h;
  memcpy(&h, state, sizeof(h));
  if (memcmp(h.magic, kStateMagic, sizeof(h.magic)) != 0) return fail(WD_EINVAL, "not a saved CG state");
  if (memcmp(h.dims, c->dims, sizeof(h.dims)) != 0 || memcmp(h.bc, c->bc, sizeof(h.bc)) != 0 ||
      h.precision != c->precision || h.field_bytes != spinor_bytes(c->wprec, c->V))
    return fail(WD_EINVAL, "the saved state belongs to another lattice, boundary or precision");
  if (h.kappa != c->kappa) return fail(WD_EINVAL, "the saved state was taken with another kappa");
  if (h.iter < 0) return fail(WD_EINVAL, "corrupt saved state");
  Solve v;
  v.src = src;
  v.x = x;
  v.state = static_cast<const unsigned char*>(state);
  v.tol = tol;
  v.maxit = maxit;
  if ((st = solve_begin(c, v)) != WD_OK) return st;
  while (!v.done)
    if ((st = solve_pass(c, v)) != WD_OK) return st;
  return solve_end(c, v, iters, true_rel_res);
}

wd_status cg_solve_batch(wd_ctx* const* ctxs, int n, const void* const* srcs, void* const* xs, const double* tols,
                         int maxit, int* iters, double* true_rel_res, int* statuses) {
  NvtxRange nvtx_("wd:cg_solve_batch");
  if (!ctxs || !srcs || !xs || !tols || n < 1 || n > 64) return fail(WD_EINVAL, "null array or n outside [1, 64]");
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return fail(WD_EINVAL, "null context");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(WD_EINVAL, "a context appears twice in the batch");
  }
  std::vector<Solve> vs(n);
  wd_status st;
  for (int i = 0; i < n; ++i) {
    vs[i].src = srcs[i];
    vs[i].x = xs[i];
    vs[i].state = nullptr;
    vs[i].tol = tols[i];
    vs[i].maxit = maxit;
    if ((st = solve_begin(ctxs[i], vs[i])) != WD_OK) return st;
  }
  wd_status ret = WD_OK;
  if (n > 1 && batchable(ctxs, vs.data(), n)) {
    // every context's own queued work (inputs, tuning) first, then the batch on the first one's stream
    for (int i = 0; i < n; ++i) WD_CUDA(cudaStreamSynchronize(ctxs[i]->stream));
    cudaStream_t s0 = ctxs[0]->stream;
    for (;;) {
      std::vector<wd_ctx*> run;
      std::vector<int> idx;
      for (int i = 0; i < n; ++i)
        if (!vs[i].done) {
          run.push_back(ctxs[i]);
          idx.push_back(i);
        }
      if (run.empty()) break;
      double ms = 0.0;
      if ((st = batch_pass(run.data(), (int)run.size(), s0, &ms)) != WD_OK) return st;
      for (size_t k = 0; k < run.size(); ++k) {
        vs[idx[k]].loop_ms += ms;
        solve_judge(run[k], vs[idx[k]]);
      }
    }
  } else {  // one after another, each as cg_solve would run it
    for (int i = 0; i < n; ++i)
      while (!vs[i].done)
        if ((st = solve_pass(ctxs[i], vs[i])) != WD_OK) return st;
  }
  for (int i = 0; i < n; ++i) {
    const wd_status r = solve_end(ctxs[i], vs[i], iters ? iters + i : nullptr, true_rel_res ? true_rel_res + i : nullptr);
    if (statuses) statuses[i] = r;
    if (r == WD_BREAKDOWN || (r == WD_NOT_CONVERGED && ret == WD_OK)) ret = r;
  }
  if (ret == WD_BREAKDOWN) fail(WD_BREAKDOWN, "CG breakdown in at least one problem of the batch");
  else if (ret == WD_NOT_CONVERGED) fail(WD_NOT_CONVERGED, "at least one problem of the batch did not converge");
  return ret;
}

wd_status wd_get_residual_history(const wd_ctx* c, double* out, int max_entries, int* count) {
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  if (!out || !count || max_entries < 0) return fail(WD_EINVAL, "null argument or negative length");
  int n = c->stats.iterations;
  if (n > c->hist_cap) n = c->hist_cap;
  if (n > max_entries) n = max_entries;
  *count = n;
  if (n == 0) return WD_OK;
  WD_CUDA(cudaMemcpy(out, c->hist_dev, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost));
  const double eta2 = c->sc_host->eta2;
  for (int i = 0; i < n; ++i) out[i] = eta2 > 0.0 ? std::sqrt(out[i] / eta2) : std::sqrt(out[i]);
  return WD_OK;
}

wd_status wd_time_dslash(wd_ctx* c, int dagger, int launches, double* avg_ms) {
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  c->resumable = false;  // the Krylov fields or the operator change
  if (!avg_ms || launches <= 0) return fail(WD_EINVAL, "bad arguments");
  if (!c->gauge_loaded) return fail(WD_ENOGAUGE, "wd_load_gauge has not been called");
  if ((st = autotune_single(c)) != WD_OK) return st;
  // the solver's dominant dslash: the working precision one, with its fused norm
  FieldPtr in = c->p, out = c->q;
  struct Standalone {
    wd_ctx* c;
    ~Standalone() { c->standalone = false; }
  } standalone_{c};
  c->standalone = true;
  WD_CUDA(op(c, in, out, dagger, EPI_PLAIN, none_field(), &c->sc->scratch[0], TK_MISC, nullptr, c->stream));
  WD_CUDA(cudaEventRecord(c->ev0, c->stream));
  for (int i = 0; i < launches; ++i)
    WD_CUDA(op(c, in, out, dagger, EPI_PLAIN, none_field(), &c->sc->scratch[0], TK_MISC, nullptr, c->stream));
  WD_CUDA(cudaEventRecord(c->ev1, c->stream));
  WD_CUDA(cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  WD_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  *avg_ms = (double)ms / launches;
  return check_tma(c);
}

wd_status wd_get_multi_stats(const wd_ctx* c, wd_multi_stats* out) {
  if (!c || !out) return fail(WD_EINVAL, "null argument");
  *out = c->mstats;
  return WD_OK;
}

wd_status wd_apply_multi(wd_ctx* c, const double* in, double* out, int nrhs, int dagger) {
  NvtxRange nvtx_("wd:apply_multi");
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  c->resumable = false;
  if (!in || !out || in == out) return fail(WD_EINVAL, "null or aliased field pointer");
  if (nrhs < 1 || nrhs > kMaxRhs) return fail(WD_EINVAL, "nrhs must be in [1, 16]");
  if (c->eo) return fail(WD_EINVAL, "multi-RHS calls need a context without WD_EVEN_ODD");
  if (!c->gauge_loaded) return fail(WD_ENOGAUGE, "wd_load_gauge has not been called");
  if ((st = ensure_multi(c, nrhs)) != WD_OK) return st;
  if ((st = ensure_multi_tuned(c)) != WD_OK) return st;
  const bool mixed = is_mixed(c->precision);
  const bool f64op = mixed && !c->apply_inner;  // mixed: FP64 operator unless the inner one is asked for
  FieldPtr a = f64op ? c->mx64 : (mixed ? c->mp : c->mq);
  FieldPtr b = f64op ? c->mr64 : (mixed ? c->mq : c->ms);
  const int grid = f64op ? c->mgrid64 : c->mgrid;
  WD_CUDA(launch_mpack(in, a, c->V, nrhs, grid, nullptr, nullptr, nullptr, c->stream));
  WD_CUDA(mdslash(c, a, b, dagger ? 1 : 0, EPI_PLAIN, none_field(), nullptr, TKM_MISC, nullptr, c->stream));
  WD_CUDA(launch_munpack(b, out, c->V, nrhs, grid, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  c->mstats.nrhs = nrhs;
  return WD_OK;
}

wd_status cg_solve_multi(wd_ctx* c, const double* src, double* x, int nrhs, double tol, int maxit, int* iters,
                         double* true_rel_res) {
  NvtxRange nvtx_("wd:cg_solve_multi");
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  c->resumable = false;
  if (!src || !x) return fail(WD_EINVAL, "null field pointer");
  if (nrhs < 1 || nrhs > kMaxRhs) return fail(WD_EINVAL, "nrhs must be in [1, 16]");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(WD_EINVAL, "tol must be a positive finite number");
  if (maxit < 0 || maxit > 10000000) return fail(WD_EINVAL, "maxit must be in [0, 10^7]");
  if (c->eo) return fail(WD_EINVAL, "multi-RHS calls need a context without WD_EVEN_ODD");
  if (c->cg_form) return fail(WD_EINVAL, "the paper's CG form (WD_OPT_CG_FORM = 1) solves one right-hand side");
  if (!c->gauge_loaded) return fail(WD_ENOGAUGE, "wd_load_gauge has not been called");
  const auto t0 = std::chrono::steady_clock::now();
  if ((st = ensure_multi(c, nrhs)) != WD_OK) return st;
  if ((st = ensure_multi_tuned(c)) != WD_OK) return st;
  const bool mixed = is_mixed(c->precision);
  MCgScalars* sc = c->msc;
  FieldPtr eta = mixed ? c->meta64 : c->meta;
  FieldPtr xs = mixed ? c->mx64 : c->mx;
  mset_params_kernel<<<1, 32, 0, c->stream>>>(sc, tol * tol, c->delta * c->delta, maxit);
  WD_CUDA(cudaGetLastError());
  WD_CUDA(launch_mpack(src, eta, c->V, nrhs, c->mgrid, c->mpartials, &sc->ticket[TKM_PACK], sc->eta2, c->stream));
  WD_CUDA(launch_mpack(x, xs, c->V, nrhs, c->mgrid, nullptr, nullptr, nullptr, c->stream));
  if (mixed && mdf(c)) {
    WD_CUDA(launch_mconvert_df(c->meta64, c->metadf, c->V, nrhs, c->mgrid, 1, c->stream));
    WD_CUDA(launch_mconvert_df(c->mx64, c->mxdf, c->V, nrhs, c->mgrid, 1, c->stream));
  }
  if (c->use_graph) {
    if ((st = build_mgraph(c)) != WD_OK) {
      abort_capture(c->cap);
      abort_capture(c->cap2);
      if (c->mexec) cudaGraphExecDestroy(c->mexec);
      if (c->mgraph) cudaGraphDestroy(c->mgraph);
      c->mexec = nullptr;
      c->mgraph = nullptr;
      return st;
    }
  }
  int restarts = 0;
  bool any_break = false, any_maxit = false, all_conv = false;
  for (;;) {
    if (c->use_graph) {
      WD_CUDA(cudaGraphLaunch(c->mexec, c->stream));
      WD_CUDA(cudaStreamSynchronize(c->stream));
    } else {
      if ((st = run_mhost_loop(c)) != WD_OK) return st;
    }
    const MCgScalars& h = *c->msc_host;
    any_break = any_maxit = false;
    all_conv = true;
    for (int r = 0; r < nrhs; ++r) {
      const double rel = h.eta2[r] > 0.0 ? std::sqrt(h.rr_true[r] / h.eta2[r]) : std::sqrt(h.rr_true[r]);
      if (h.status[r] == ST_BREAKDOWN || !std::isfinite(rel) || !std::isfinite(h.eta2[r])) {
        any_break = true;
        all_conv = false;
      } else if (rel > tol) {
        all_conv = false;
        if (h.status[r] == ST_MAXIT) any_maxit = true;
      }
    }
    if (all_conv || any_break || any_maxit) break;
    if (h.iter >= maxit || restarts >= c->max_restarts) {
      any_maxit = true;
      break;
    }
    ++restarts;
  }
  WD_CUDA(launch_munpack(xs, x, c->V, nrhs, c->mgrid, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  const MCgScalars& h = *c->msc_host;
  for (int r = 0; r < nrhs; ++r) {
    const double rel = h.eta2[r] > 0.0 ? std::sqrt(h.rr_true[r] / h.eta2[r]) : std::sqrt(h.rr_true[r]);
    if (iters) iters[r] = h.iters[r];
    if (true_rel_res) true_rel_res[r] = rel;
  }
  const auto t1 = std::chrono::steady_clock::now();
  c->mstats.nrhs = nrhs;
  c->mstats.iterations = h.iter;
  c->mstats.restarts = restarts;
  c->mstats.reliable_updates = h.updates;
  c->mstats.solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  wd_status ret = WD_OK;
  if (any_break)
    ret = fail(WD_BREAKDOWN, "CG breakdown in at least one right-hand side (NaN/Inf in a source?)");
  else if (!all_conv)
    ret = fail(WD_NOT_CONVERGED, "maximum iterations reached before every right-hand side met tol");
  c->mstats.status = ret;
  return ret;
}

wd_status wd_generate_gauge(wd_ctx* c, double eps, unsigned long long seed, int compress12, double* U_out) {
  NvtxRange nvtx_("wd:generate_gauge");
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  c->resumable = false;
  if (!std::isfinite(eps)) return fail(WD_EINVAL, "eps must be finite");
  bool need64 = false, need32 = false;
  int c12 = 0;
  if ((st = ensure_gauge_buffers(c, compress12, &need64, &need32, &c12)) != WD_OK) return st;
  WD_CUDA(launch_gen_gauge(c->V, eo_geom(c), eps, seed, need64 ? c->gauge64 : nullptr, need32 ? c->gauge32 : nullptr, c12, U_out, c->gauge_df,
                           c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  c->gauge_loaded = true;
  return WD_OK;
}

wd_status wd_generate_source(wd_ctx* c, unsigned long long seed, double* out) {
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  if (!out) return fail(WD_EINVAL, "out is null");
  WD_CUDA(launch_gen_source(c->V, seed, out, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  return WD_OK;
}

wd_status wd_set_kappa(wd_ctx* c, double kappa) {
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  c->resumable = false;  // the Krylov fields or the operator change
  if (!std::isfinite(kappa) || std::fabs(kappa) >= 1.0) return fail(WD_EINVAL, "kappa must be finite with |kappa| < 1");
  WD_CUDA(cudaStreamSynchronize(c->stream));
  c->kappa = kappa;
  c->sc_host->kappa = kappa;
  WD_CUDA(cudaMemcpyAsync(&c->sc->kappa, &c->sc_host->kappa, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  return WD_OK;
}

wd_status wd_coo_build(wd_ctx* c, const double* U, int* row, int* col, double* val, long long capacity,
                       long long* nnz) {
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  if (!U || !row || !col || !val || !nnz) return fail(WD_EINVAL, "null argument");
  const long long need = 49LL * 12LL * c->V;
  *nnz = need;
  if (capacity < need) return fail(WD_EINVAL, "capacity below 49 * 12 * V entries");
  if (12LL * c->V > 0x7fffffffLL) return fail(WD_EINVAL, "volume too large for 32-bit COO indices");
  WD_CUDA(launch_coo_build(c->geom, U, c->kappa, row, col, val, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  return WD_OK;
}

wd_status wd_coo_spmv(wd_ctx* c, long long nnz, const int* row, const int* col, const double* val, const double* in,
                      double* out) {
  wd_status st;
  if ((st = check_ctx(c)) != WD_OK) return st;
  if (!row || !col || !val || !in || !out || in == out || nnz < 0) return fail(WD_EINVAL, "bad argument");
  WD_CUDA(launch_coo_spmv(nnz, row, col, val, in, out, 12LL * c->V, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  return WD_OK;
}

}  // extern "C"
