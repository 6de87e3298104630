// Persistent cooperative CG loops: plain (lexicographic), mixed-precision inner loop and even-odd.
#include <type_traits>

#include "wd_stencil.cuh"

namespace wdk {

// ---------------------------------------------------------------- persistent CG loop
//
// At the paper's volumes every kernel of a CG iteration costs a launch and a grid-reduction tail
// of several microseconds, comparable to its work. This kernel runs the whole CGLS loop (the four
// phases of each iteration) in one cooperative launch: the grid is one wave of resident blocks,
// the phases are separated by a grid barrier, and each norm is summed by every block from the
// block partials in one fixed order, so all blocks hold the same scalars and the results are
// reproducible. The launch is cooperative, so all blocks are resident and the barrier always
// completes; its wait is still bounded: past the limit the kernel records an error and stops.

struct LoopSync {
  unsigned long long* ctr;  // arrivals since the launch began (zeroed by the host before each launch)
  int* err;                 // set to 1 when a barrier wait gave up
  long long limit;          // polls (64 ns sleep each) before a wait gives up
};

// Arrival with release and acquire semantics at GPU scope (the block's writes, ordered before it by
// the __syncthreads that precedes, become visible to every block that later acquires the counter),
// and the acquiring read of the pollers. No separate fence instruction is needed.
__device__ __forceinline__ unsigned long long arrive_acq_rel(unsigned long long* p) {
  unsigned long long old;
  asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], 1;" : "=l"(old) : "l"(p) : "memory");
  return old;
}

__device__ __forceinline__ unsigned long long load_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// All blocks arrive, then continue. Returns false (everywhere, eventually) if a wait gave up.
// One monotonic 64-bit counter: barrier number k of the launch completes when the counter reaches
// k * gridDim.x, so a waiter sees the last arrival's own atomic (no second release step), and the
// last block to arrive does not wait at all. Thread 0 of each block arrives and polls; the
// __syncthreads on either side carry the ordering to the rest of the block.
__device__ __forceinline__ bool grid_barrier(const LoopSync& y) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long G = gridDim.x;
    const unsigned long long arrived = arrive_acq_rel(y.ctr);
    const unsigned long long target = (arrived / G + 1) * G;
    int good = 1;
    if (arrived + 1 != target) {
      long long spins = 0;
      while (load_acquire(y.ctr) < target) {
        if (++spins > y.limit || *(volatile int*)y.err) {
          atomicExch(y.err, 1);
          good = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    ok = good && !*(volatile int*)y.err;
  }
  __syncthreads();
  return ok;
}

// The sum of G block partials by the first warp, in one fixed order: lane l adds partials l, l + 32,
// l + 64, ... in turn, then a shuffle tree. AHEAD: up to 256 partials, the lane's loads are issued
// together ahead of the additions, whose order is kept (same bits). Measured per loop kernel: the
// one-thread-per-site FP64 loop gains with it (14^4 11.57 -> 11.45 ms, 16^4 22.60 -> 22.41 ms), the
// FP64 loop with 4 to 16 lanes per site loses (8^4 at 64-thread blocks 3.00 -> 3.10 ms, 4^4 with
// 8 lanes 1.70 -> 1.78 ms), so the others keep the plain strided sum.
template <bool AHEAD>
__device__ __forceinline__ double lane_sum(const double* partials, int G) {
  double a = 0.0;
  if constexpr (AHEAD) {
    constexpr int kAhead = 8;
    double x[kAhead];
#pragma unroll
    for (int k = 0; k < kAhead; ++k) {
      const int b = threadIdx.x + 32 * k;
      x[k] = b < G ? __ldcg(partials + b) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < kAhead; ++k)
      if (threadIdx.x + 32 * k < G) a += x[k];
    for (int b = threadIdx.x + 32 * kAhead; b < G; b += 32) a += __ldcg(partials + b);
  } else {
    for (int b = threadIdx.x; b < G; b += 32) a += __ldcg(partials + b);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
  return a;
}

// Sum over the grid of one value per thread: block partial, barrier, then every block sums the
// partials in the same order (lanes stride over them, then a fixed shuffle tree).
template <bool AHEAD = false>
__device__ __forceinline__ bool loop_sum(double v, double* partials, const LoopSync& y, double* out) {
  __shared__ double smem[32];
  __shared__ double total;
  double w[1] = {v};
  block_reduce<OpSum, 1>(w, smem);
  if (threadIdx.x == 0) partials[blockIdx.x] = w[0];  // released by the barrier's arrival
  if (!grid_barrier(y)) return false;
  if (threadIdx.x < 32) {
    const double a = lane_sum<AHEAD>(partials, gridDim.x);
    if (threadIdx.x == 0) total = a;
  }
  __syncthreads();
  *out = total;
  return true;
}

// Two sums behind one barrier (partials: two regions of gridDim.x).
__device__ __forceinline__ bool loop_sum2(double v0, double v1, double* partials, const LoopSync& y, double* o0,
                                          double* o1) {
  __shared__ double smem[64];
  __shared__ double total[2];
  const int G = gridDim.x;
  double w[2] = {v0, v1};
  block_reduce<OpSum, 2>(w, smem);
  if (threadIdx.x == 0) {  // released by the barrier's arrival
    partials[blockIdx.x] = w[0];
    partials[G + blockIdx.x] = w[1];
  }
  if (!grid_barrier(y)) return false;
  if (threadIdx.x < 32) {
    double a0 = 0.0, a1 = 0.0;
    for (int b = threadIdx.x; b < G; b += 32) {
      a0 += __ldcg(partials + b);
      a1 += __ldcg(partials + G + b);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      a0 += __shfl_down_sync(0xffffffffu, a0, off);
      a1 += __shfl_down_sync(0xffffffffu, a1, off);
    }
    if (threadIdx.x == 0) {
      total[0] = a0;
      total[1] = a1;
    }
  }
  __syncthreads();
  *o0 = total[0];
  *o1 = total[1];
  return true;
}

template <int SP, bool C12>
struct LoopArgs {
  DslashArgs<SP, C12> dq;  // q = D p
  DslashArgs<SP, C12> ds;  // s = D^dag r
  SpinorRef<SP> x, r, p, q, s;
  double2* tl;             // FP64 loop in the time-diagonal basis: pre-scaled time links [9][V]
  int n;                   // sites
  CgScalars* sc;
  double* partials;        // 3 x gridDim.x
  LoopSync y;
};

// The dslash phases of the loop: one thread per site, (FP64) two lanes per site, or (FP64, one
// thread per site, DT) the operator in the basis where gamma_t is diagonal (hop_t_dirac).
template <int SP, bool C12, bool DAG, int LANES, bool DT = false>
__device__ __forceinline__ double loop_dslash(const DslashArgs<SP, C12>& d, const double2* tl, int n, int t0,
                                              int tstep) {
  if constexpr (SP == P64 && LANES == 2) {
    return pair_sites<C12, DAG, EPI_PLAIN>(d);
  } else if constexpr (DT) {
    static_assert(SP == P64 && !C12 && LANES == 1, "the time-diagonal basis serves the FP64 one-thread loop");
    double v = 0.0;
    for (int i = t0; i < n; i += tstep) {
      Cx<double> acc[12];
      v += dslash_site_dirac_t<DAG>(d, tl, i, acc);
    }
    return v;
  } else {
    double v = 0.0;
    for (int i = t0; i < n; i += tstep) v += dslash_site<SP, C12, DAG, EPI_PLAIN>(d, i);
    return v;
  }
}

// One site of a dslash phase whose output stays in registers (the loop with one site per thread).
template <int SP, bool C12, bool DAG, bool DT>
__device__ __forceinline__ double loop_dslash_site(const DslashArgs<SP, C12>& d, const double2* tl, int i,
                                                   Cx<typename RealOf<SP>::type> (&out)[12]) {
  if constexpr (DT)
    return dslash_site_dirac_t<DAG>(d, tl, i, out);
  else
    return dslash_site_out<SP, C12, DAG, EPI_PLAIN>(d, i, out);
}

// A batch of independent loops in one cooperative launch: blockIdx.y selects the problem, whose
// blocks run exactly the body (and the grid, gridDim.x) of its launch alone, with its own barrier
// counter, scalars and fields, so each result is bitwise the one of a launch of its own.
constexpr int kLoopBatch = kMaxBatch;
template <typename Args>
struct LoopBatch {
  Args a[kLoopBatch];
};
// The batch kernels read their arguments with a runtime index (blockIdx.y), so the pointers and
// geometry live in registers rather than in the constant bank: they get the register budget of
// two blocks per SM instead of three (FP32 / FP16), which the small volumes they serve leave free.
template <int SP>
struct BatchMinBlocks {
  static constexpr int value = SP == P64 ? 1 : 2;
};

// DT (FP64, one thread per site): the loop runs in the spin basis psi' = T psi of hop_t_dirac.
// x, r, p and s enter it in place before the first iteration (a grid barrier follows, since the
// first dslash reads p at neighbours) and leave it, with q, when the loop ends; each thread
// transforms only the sites it updates itself, whose last writes are its own. T = sqrt(2) x a
// unitary, so every norm in the basis is twice the chiral one: gamma and |r|^2 enter doubled and
// leave halved (exact scalings), alpha and beta are unchanged, and the iterates are T times the
// chiral ones up to rounding.
template <int SP, bool C12, int LANES, bool DT = false>
__device__ __forceinline__ void cg_loop_body(const LoopArgs<SP, C12>& a) {
  typedef typename RealOf<SP>::type R;
  CgScalars* sc = a.sc;
  if (sc->status != ST_RUNNING) return;  // uniform over the grid
  const int n = a.n, V = a.dq.g.V, G = gridDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, tstep = G * blockDim.x;
  constexpr bool AH = SP == P64 && LANES == 1;  // see lane_sum
  const double nscale = DT ? 2.0 : 1.0;  // |T v|^2 / |v|^2
  double gamma = sc->gamma * nscale, rr = sc->rr * nscale;
  const double tol2e = sc->tol2 * sc->eta2 * nscale;
  int iter = sc->iter, status = ST_RUNNING;
  const int maxit = sc->maxit;
  double alpha = 0.0, beta = 0.0;
  bool run = true;
  if constexpr (DT) {
    for (int i = t0; i < n; i += tstep) {
      dirac_t_basis<false>(a.x, i, V);
      dirac_t_basis<false>(a.r, i, V);
      dirac_t_basis<false>(a.p, i, V);
      dirac_t_basis<false>(a.s, i, V);
      scale_time_link(a.dq, a.tl, i);
    }
    run = grid_barrier(a.y);  // p and the time links everywhere before D p reads its neighbours
  }
  // One site per thread (FP64, the grid covers the lattice): the dslash outputs q and s stay in
  // registers for the vector phase after the next barrier instead of being read back from the L2
  // (they are still stored: the fields are the loop's state). The arithmetic and its order are those
  // of the general path, and FP64 fields store the register values unrounded, so both give the same
  // bits. Loading r, x and p before the barrier as well measured slower (spills at 255 registers).
  // The two paths are separate instantiations, so neither keeps the other's values live.
  auto iterate = [&](auto one_tag) {
    constexpr bool ONE = decltype(one_tag)::value;
    const bool mine = t0 < n;
    while (run) {
      // q = D p, |q|^2
      Cx<R> qv[12];
      double v = 0.0;
      if constexpr (ONE) {
        if (mine) v = loop_dslash_site<SP, C12, false, DT>(a.dq, a.tl, t0, qv);
      } else {
        v = loop_dslash<SP, C12, false, LANES, DT>(a.dq, a.tl, n, t0, tstep);
      }
      double qq;
      if (!loop_sum<AH>(v, a.partials, a.y, &qq)) break;
      if (!(qq > 0.0 && isfinite(qq) && isfinite(gamma))) {
        status = ST_BREAKDOWN;
        break;
      }
      alpha = gamma / qq;
      const R ar = (R)alpha;
      // r -= alpha q, |r|^2
      v = 0.0;
      for (int i = t0; i < n; i += tstep) {
        Cx<R> rv[12];
        load_spinor(a.r, i, V, rv);
        if constexpr (!ONE) load_spinor(a.q, i, V, qv);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          rv[c].re = fma(-ar, qv[c].re, rv[c].re);
          rv[c].im = fma(-ar, qv[c].im, rv[c].im);
        }
        store_spinor(a.r, i, V, rv);
        v += norm2_site(rv);
      }
      if (!loop_sum<AH>(v, a.partials + G, a.y, &rr)) break;
      if (blockIdx.x == 0 && threadIdx.x == 0) record_residual(sc, iter, rr / nscale);
      if (!isfinite(rr)) {
        status = ST_BREAKDOWN;
        break;
      }
      const bool conv = rr <= tol2e;
      // s = D^dag r, |s|^2 (not needed once converged)
      double gnew = 0.0;
      Cx<R> sv[12];
      if (!conv) {
        if constexpr (ONE) {
          v = 0.0;
          if (mine) v = loop_dslash_site<SP, C12, true, DT>(a.ds, a.tl, t0, sv);
        } else {
          v = loop_dslash<SP, C12, true, LANES, DT>(a.ds, a.tl, n, t0, tstep);
        }
        if (!loop_sum<AH>(v, a.partials + 2 * G, a.y, &gnew)) break;
      }
      const bool do_p = !conv && isfinite(gnew) && gamma > 0.0;
      beta = do_p ? gnew / gamma : 0.0;
      const R br = (R)beta;
      // x += alpha p; p = s + beta p
      for (int i = t0; i < n; i += tstep) {
        Cx<R> xv[12], pv[12];
        load_spinor(a.x, i, V, xv);
        load_spinor(a.p, i, V, pv);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          xv[c].re = fma(ar, pv[c].re, xv[c].re);
          xv[c].im = fma(ar, pv[c].im, xv[c].im);
        }
        store_spinor(a.x, i, V, xv);
        if (do_p) {
          if constexpr (!ONE) load_spinor(a.s, i, V, sv);
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            pv[c].re = fma(br, pv[c].re, sv[c].re);
            pv[c].im = fma(br, pv[c].im, sv[c].im);
          }
          store_spinor(a.p, i, V, pv);
        }
      }
      iter += 1;
      if (conv) {
        status = ST_CONVERGED;
        break;
      }
      if (!do_p) {
        status = ST_BREAKDOWN;
        break;
      }
      gamma = gnew;
      if (iter >= maxit) {
        status = ST_MAXIT;
        break;
      }
      if (!grid_barrier(a.y)) break;  // p complete before the next dslash reads its neighbours
    }
  };
  if constexpr (SP == P64 && LANES == 1) {
    if (n <= tstep)
      iterate(std::true_type{});
    else
      iterate(std::false_type{});
  } else {
    iterate(std::false_type{});
  }
  if constexpr (DT) {
    // every neighbour read of this launch is behind the last barrier all blocks passed
    for (int i = t0; i < n; i += tstep) {
      dirac_t_basis<true>(a.x, i, V);
      dirac_t_basis<true>(a.r, i, V);
      dirac_t_basis<true>(a.p, i, V);
      dirac_t_basis<true>(a.s, i, V);
      dirac_t_basis<true>(a.q, i, V);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const bool failed = *(volatile int*)a.y.err != 0;
    sc->status = failed ? ST_BREAKDOWN : status;
    sc->iter = iter;
    sc->gamma = gamma / nscale;
    sc->rr = rr / nscale;
    sc->alpha = alpha;
    sc->beta = beta;
  }
}

template <int SP, bool C12, int LANES, bool DT>
__global__ void __launch_bounds__(kDslashMaxThreads, DslashMinBlocks<SP>::value) cg_loop_kernel(const LoopArgs<SP, C12> a) {
  cg_loop_body<SP, C12, LANES, DT>(a);
}

template <int SP, bool C12, int LANES, bool DT>
__global__ void __launch_bounds__(kDslashMaxThreads, BatchMinBlocks<SP>::value)
    cg_loop_batch_kernel(const __grid_constant__ LoopBatch<LoopArgs<SP, C12>> b) {
  cg_loop_body<SP, C12, LANES, DT>(b.a[blockIdx.y]);
}

// The paper's CG (Sec. 2: CG on D D^dag psi = eta, carried in x = D^dag psi) as one persistent
// launch. Its iteration needs three grid barriers where CGLS needs four: alpha comes from the first
// operator's output, so the second operator and both vector updates share one phase.
//   A: s = D^dag p, |s|^2;                                  barrier; alpha = |r|^2 / |s|^2
//   B: q = D s and, at the same site, x += alpha s, r -= alpha q, |r|^2
//                                                          barrier; beta = |r'|^2 / |r|^2, convergence
//   C: p = r + beta p;                                      barrier (p complete before A reads it)
// gamma holds |r|^2 here. The vector arithmetic is that of the graph's kernels (fma(alpha, s, x),
// fma(-alpha, q, r), fma(beta, p, r)). DT: the spin basis of cg_loop_body, entered and left the
// same way. ds reads p and writes s; dq reads s and writes q (paper_loop_args).
template <int SP, bool C12, bool DT>
__device__ __forceinline__ void cg_paper_loop_body(const LoopArgs<SP, C12>& a) {
  typedef typename RealOf<SP>::type R;
  CgScalars* sc = a.sc;
  if (sc->status != ST_RUNNING) return;  // uniform over the grid
  const int n = a.n, V = a.dq.g.V, G = gridDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, tstep = G * blockDim.x;
  constexpr bool AH = SP == P64;  // see lane_sum
  const double nscale = DT ? 2.0 : 1.0;
  double gamma = sc->gamma * nscale, rr = sc->rr * nscale;
  const double tol2e = sc->tol2 * sc->eta2 * nscale;
  int iter = sc->iter, status = ST_RUNNING;
  const int maxit = sc->maxit;
  double alpha = 0.0, beta = 0.0;
  bool run = true;
  if constexpr (DT) {
    for (int i = t0; i < n; i += tstep) {
      dirac_t_basis<false>(a.x, i, V);
      dirac_t_basis<false>(a.r, i, V);
      dirac_t_basis<false>(a.p, i, V);
      scale_time_link(a.dq, a.tl, i);
    }
    run = grid_barrier(a.y);  // p and the time links everywhere before D^dag p reads them
  }
  // FP64, one site per thread: r stays in registers from B to C (the FP32 kernel's register budget
  // of three blocks per SM has no room for it)
  constexpr bool KEEP = SP == P64;
  const bool one = KEEP && n <= tstep;
  while (run) {
    // A: s = D^dag p, |s|^2
    double v = loop_dslash<SP, C12, true, 1, DT>(a.ds, a.tl, n, t0, tstep);
    double ss;
    if (!loop_sum<AH>(v, a.partials, a.y, &ss)) break;
    if (!(ss > 0.0 && isfinite(ss) && isfinite(gamma))) {
      status = ST_BREAKDOWN;
      break;
    }
    alpha = gamma / ss;
    const R ar = (R)alpha;
    // B: q = D s; x += alpha s; r -= alpha q; |r|^2
    v = 0.0;
    Cx<R> rkeep[12];
    for (int i = t0; i < n; i += tstep) {
      Cx<R> qv[12], sv[12], xv[12], rv[12];
      loop_dslash_site<SP, C12, false, DT>(a.dq, a.tl, i, qv);
      load_spinor(a.s, i, V, sv);
      load_spinor(a.x, i, V, xv);
      load_spinor(a.r, i, V, rv);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        xv[c].re = fma(ar, sv[c].re, xv[c].re);
        xv[c].im = fma(ar, sv[c].im, xv[c].im);
        rv[c].re = fma(-ar, qv[c].re, rv[c].re);
        rv[c].im = fma(-ar, qv[c].im, rv[c].im);
      }
      store_spinor(a.x, i, V, xv);
      store_spinor(a.r, i, V, rv);
      v += norm2_site(rv);
      if constexpr (KEEP) {
#pragma unroll
        for (int c = 0; c < 12; ++c) rkeep[c] = rv[c];
      }
    }
    double rnew;
    if (!loop_sum<AH>(v, a.partials + G, a.y, &rnew)) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) record_residual(sc, iter, rnew / nscale);
    if (!isfinite(rnew)) {
      status = ST_BREAKDOWN;
      break;
    }
    iter += 1;
    if (rnew <= tol2e) {
      rr = rnew;
      gamma = rnew;
      status = ST_CONVERGED;
      break;
    }
    if (!(gamma > 0.0)) {
      status = ST_BREAKDOWN;
      break;
    }
    beta = rnew / gamma;
    gamma = rnew;
    rr = rnew;
    const R br = (R)beta;
    // C: p = r + beta p
    for (int i = t0; i < n; i += tstep) {
      Cx<R> pv[12], rv[12];
      load_spinor(a.p, i, V, pv);
      if (KEEP && one) {
#pragma unroll
        for (int c = 0; c < 12; ++c) rv[c] = rkeep[c];
      } else {
        load_spinor(a.r, i, V, rv);
      }
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        pv[c].re = fma(br, pv[c].re, rv[c].re);
        pv[c].im = fma(br, pv[c].im, rv[c].im);
      }
      store_spinor(a.p, i, V, pv);
    }
    if (iter >= maxit) {
      status = ST_MAXIT;
      break;
    }
    if (!grid_barrier(a.y)) break;  // p complete before A reads its neighbours
  }
  if constexpr (DT) {
    // every neighbour read of this launch is behind the last barrier all blocks passed
    for (int i = t0; i < n; i += tstep) {
      dirac_t_basis<true>(a.x, i, V);
      dirac_t_basis<true>(a.r, i, V);
      dirac_t_basis<true>(a.p, i, V);
      dirac_t_basis<true>(a.s, i, V);
      dirac_t_basis<true>(a.q, i, V);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const bool failed = *(volatile int*)a.y.err != 0;
    sc->status = failed ? ST_BREAKDOWN : status;
    sc->iter = iter;
    sc->gamma = gamma / nscale;
    sc->rr = rr / nscale;
    sc->alpha = alpha;
    sc->beta = beta;
  }
}

template <int SP, bool C12, bool DT>
__global__ void __launch_bounds__(kDslashMaxThreads, DslashMinBlocks<SP>::value)
    cg_paper_loop_kernel(const LoopArgs<SP, C12> a) {
  cg_paper_loop_body<SP, C12, DT>(a);
}

template <int SP, bool C12, bool DT>
__global__ void __launch_bounds__(kDslashMaxThreads, BatchMinBlocks<SP>::value)
    cg_paper_loop_batch_kernel(const __grid_constant__ LoopBatch<LoopArgs<SP, C12>> b) {
  cg_paper_loop_body<SP, C12, DT>(b.a[blockIdx.y]);
}

// The inner loop of the mixed-precision solver (FP32 or FP16 vectors, x_lo in FP32) in one
// cooperative launch. Phase A: q = D p, |q|^2; r_lo -= alpha q, x_lo += alpha p, |r_lo|^2, and
// the reliable-update test. Phase B: s = D^dag r_lo, |s|^2; p = s + beta p. The kernel starts at A
// (or at B right after a reliable update) and returns as soon as an update is due or the loop
// ends, leaving the same scalars and flags as the separate kernels of the graph solver.
template <int SPW, bool C12>
struct MixedLoopArgs {
  DslashArgs<SPW, C12> dq;  // q = D p
  DslashArgs<SPW, C12> ds;  // s = D^dag r
  SpinorRef<SPW> r, p, q, s;
  SpinorRef<P32> xlo;
  int n;
  int start_b;
  CgScalars* sc;
  double* partials;  // 3 x gridDim.x
  LoopSync y;
};

template <int SPW, bool C12>
__device__ __forceinline__ void cg_mixed_loop_body(const MixedLoopArgs<SPW, C12>& a) {
  CgScalars* sc = a.sc;
  const int st_in = sc->status;
  if (st_in != ST_RUNNING && !(a.start_b && st_in == ST_CONVERGED)) return;  // uniform over the grid
  const int n = a.n, V = a.dq.g.V, G = gridDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, tstep = G * blockDim.x;
  double gamma = sc->gamma, rr = sc->rr, alpha = sc->alpha, beta = sc->beta;
  const double tol2e = sc->tol2 * sc->eta2, d2ref = sc->delta2 * sc->rr_ref;
  int iter = sc->iter, status = st_in, need = 0;
  const int maxit = sc->maxit;
  bool phase_b = a.start_b != 0;
  for (;;) {
    if (phase_b) {
      // s = D^dag r_lo, gamma' = |s|^2 (skipped once the last update converged)
      double gnew = 0.0;
      if (status == ST_RUNNING) {
        double v = 0.0;
        for (int i = t0; i < n; i += tstep) v += dslash_site<SPW, C12, true, EPI_PLAIN>(a.ds, i);
        if (!loop_sum(v, a.partials + 2 * G, a.y, &gnew)) break;
      }
      const bool do_p = status == ST_RUNNING && isfinite(gnew) && gamma > 0.0;
      beta = do_p ? gnew / gamma : 0.0;
      const float bf = (float)beta;
      if (do_p) {
        for (int i = t0; i < n; i += tstep) {
          Cx<float> pv[12], sv[12];
          load_spinor(a.p, i, V, pv);
          load_spinor(a.s, i, V, sv);
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            pv[c].re = fmaf(bf, pv[c].re, sv[c].re);
            pv[c].im = fmaf(bf, pv[c].im, sv[c].im);
          }
          store_spinor(a.p, i, V, pv);
        }
      }
      iter += 1;  // the iteration whose r update ran, including one that converged in its update
      if (status != ST_RUNNING) break;
      if (!do_p) {
        status = ST_BREAKDOWN;
        break;
      }
      gamma = gnew;
      if (iter >= maxit) {
        status = ST_MAXIT;
        break;
      }
      if (!grid_barrier(a.y)) break;  // p complete before the next dslash reads its neighbours
    }
    phase_b = true;
    // q = D p, |q|^2
    double v = 0.0;
    for (int i = t0; i < n; i += tstep) v += dslash_site<SPW, C12, false, EPI_PLAIN>(a.dq, i);
    double qq;
    if (!loop_sum(v, a.partials, a.y, &qq)) break;
    if (!(qq > 0.0 && isfinite(qq) && isfinite(gamma))) {
      status = ST_BREAKDOWN;
      break;
    }
    alpha = gamma / qq;
    const float af = (float)alpha;
    // r_lo -= alpha q; x_lo += alpha p; |r_lo|^2
    v = 0.0;
    for (int i = t0; i < n; i += tstep) {
      Cx<float> rv[12], qv[12], pv[12], xv[12];
      load_spinor(a.r, i, V, rv);
      load_spinor(a.q, i, V, qv);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        rv[c].re = fmaf(-af, qv[c].re, rv[c].re);
        rv[c].im = fmaf(-af, qv[c].im, rv[c].im);
      }
      store_spinor(a.r, i, V, rv);
      v += norm2_site(rv);
      load_spinor(a.p, i, V, pv);
      load_spinor(a.xlo, i, V, xv);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        xv[c].re = fmaf(af, pv[c].re, xv[c].re);
        xv[c].im = fmaf(af, pv[c].im, xv[c].im);
      }
      store_spinor(a.xlo, i, V, xv);
    }
    if (!loop_sum(v, a.partials + G, a.y, &rr)) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) record_residual(sc, iter, rr);
    if (!isfinite(rr)) {
      status = ST_BREAKDOWN;
      break;
    }
    need = (rr <= d2ref) || (rr <= tol2e);
    if (need) break;  // the reliable update runs outside; the loop resumes at phase B
    if (!grid_barrier(a.y)) break;  // r complete before D^dag reads its neighbours
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const bool failed = *(volatile int*)a.y.err != 0;
    sc->status = failed ? ST_BREAKDOWN : status;
    sc->iter = iter;
    sc->gamma = gamma;
    sc->rr = rr;
    sc->alpha = alpha;
    sc->beta = beta;
    sc->need_update = need;
    sc->no_update = !need;
  }
}

template <int SPW, bool C12>
__global__ void __launch_bounds__(kDslashMaxThreads, DslashMinBlocks<SPW>::value)
    cg_mixed_loop_kernel(const MixedLoopArgs<SPW, C12> a) {
  cg_mixed_loop_body<SPW, C12>(a);
}

template <int SPW, bool C12>
__global__ void __launch_bounds__(kDslashMaxThreads, BatchMinBlocks<SPW>::value)
    cg_mixed_loop_batch_kernel(const __grid_constant__ LoopBatch<MixedLoopArgs<SPW, C12>> b) {
  cg_mixed_loop_body<SPW, C12>(b.a[blockIdx.y]);
}

template <int SPW, bool C12>
static MixedLoopArgs<SPW, C12> mixed_loop_args(const CgLoopCall& c) {
  MixedLoopArgs<SPW, C12> a;
  for (DslashArgs<SPW, C12>* d : {&a.dq, &a.ds}) {
    memcpy(&d->g, &c.g, sizeof(Geom));
    d->u.p = reinterpret_cast<decltype(d->u.p)>(c.u.p);
    d->mkappa = (float)(-c.kappa);
    d->kappa_dev = c.kappa_dev;
    d->skip = nullptr;
    d->partials = nullptr;
    d->ticket = nullptr;
    d->result = nullptr;
  }
  a.dq.in = make_ref<SPW>(c.p, c.g.V);
  a.dq.out = make_ref<SPW>(c.q, c.g.V);
  a.dq.b = make_ref<SPW>(FieldPtr{}, c.g.V);
  a.ds.in = make_ref<SPW>(c.r, c.g.V);
  a.ds.out = make_ref<SPW>(c.s, c.g.V);
  a.ds.b = a.dq.b;
  a.r = make_ref<SPW>(c.r, c.g.V);
  a.p = make_ref<SPW>(c.p, c.g.V);
  a.q = make_ref<SPW>(c.q, c.g.V);
  a.s = make_ref<SPW>(c.s, c.g.V);
  a.xlo = make_ref<P32>(c.x, c.g.V);
  a.n = c.g.V;
  a.start_b = c.start_b;
  a.sc = c.sc;
  a.partials = c.partials;
  a.y.ctr = reinterpret_cast<unsigned long long*>(c.bar);
  a.y.limit = c.wait_limit;
  a.y.err = c.err;
  return a;
}

// Grid of the loop over `threads` threads: one wave of resident blocks of the single-problem kernel,
// or fewer when the sites do not fill it. A batch uses the same grid per problem.
static int loop_grid(const void* single_kernel, int threads, const CgLoopCall& c) {
  int grid = resident_blocks(single_kernel, c.block);
  const int need = grid_for(threads, c.block);
  if (need < grid) grid = need;
  if (grid > c.max_grid) grid = c.max_grid;
  return grid;
}

// One problem: the single kernel with its arguments in parameter space. Several: the batch kernel
// on a (grid, n) grid, when all n * grid blocks can be resident at once (else the launch is refused
// with cudaErrorCooperativeLaunchTooLarge and the caller splits the batch).
template <typename Args, typename KS, typename KB>
static cudaError_t loop_launch(KS single, KB batch, Args (*make)(const CgLoopCall&), const CgLoopCall* cs, int n,
                               int threads, cudaStream_t st) {
  const CgLoopCall& c0 = cs[0];
  const int grid = loop_grid(reinterpret_cast<const void*>(single), threads, c0);
  for (int i = 0; i < n; ++i) {  // barrier count of this launch
    cudaError_t e = cudaMemsetAsync(cs[i].bar, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  if (n == 1) {
    Args a = make(c0);
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(single), dim3(grid), dim3(c0.block), args, 0, st);
  }
  if (n > kLoopBatch) return cudaErrorInvalidValue;
  if ((long long)grid * n > resident_blocks(reinterpret_cast<const void*>(batch), c0.block))
    return cudaErrorCooperativeLaunchTooLarge;
  LoopBatch<Args> b;
  memset(&b, 0, sizeof(b));
  for (int i = 0; i < n; ++i) b.a[i] = make(cs[i]);
  void* args[] = {&b};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(batch), dim3(grid, n), dim3(c0.block), args, 0, st);
}

// Every call of a batch must describe the same problem shape (lattice, precisions, launch shape).
static bool same_shape(const CgLoopCall* cs, int n) {
  for (int i = 1; i < n; ++i) {
    const CgLoopCall &a = cs[0], &b = cs[i];
    if (memcmp(&a.g, &b.g, sizeof(GeomH)) != 0 || a.block != b.block || a.variant != b.variant ||
        a.max_grid != b.max_grid || a.u.prec != b.u.prec || a.u.c12 != b.u.c12 || a.r.prec != b.r.prec ||
        a.x.prec != b.x.prec || a.time_basis != b.time_basis || a.cg_form != b.cg_form)
      return false;
  }
  return true;
}

cudaError_t launch_cg_mixed_loop_n(const CgLoopCall* cs, int n, cudaStream_t st) {
  if (n < 1 || !same_shape(cs, n)) return cudaErrorInvalidValue;
  const CgLoopCall& c = cs[0];
  if (c.block <= 0 || c.block > kDslashMaxThreads || c.block % 32 || c.max_grid < 1) return cudaErrorInvalidValue;
  for (int i = 0; i < n; ++i) {
    const CgLoopCall& d = cs[i];
    if (d.x.prec != SP32 || d.u.prec != SP32 || d.p.prec != d.r.prec || d.q.prec != d.r.prec || d.s.prec != d.r.prec)
      return cudaErrorInvalidValue;
  }
  const int th = c.g.V;
  if (c.r.prec == SP32) {
    if (c.u.c12)
      return loop_launch(cg_mixed_loop_kernel<P32, true>, cg_mixed_loop_batch_kernel<P32, true>, mixed_loop_args<P32, true>, cs, n, th, st);
    return loop_launch(cg_mixed_loop_kernel<P32, false>, cg_mixed_loop_batch_kernel<P32, false>, mixed_loop_args<P32, false>, cs, n, th, st);
  }
  if (c.r.prec == SP16) {
    if (c.u.c12)
      return loop_launch(cg_mixed_loop_kernel<P16, true>, cg_mixed_loop_batch_kernel<P16, true>, mixed_loop_args<P16, true>, cs, n, th, st);
    return loop_launch(cg_mixed_loop_kernel<P16, false>, cg_mixed_loop_batch_kernel<P16, false>, mixed_loop_args<P16, false>, cs, n, th, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_cg_mixed_loop(const CgLoopCall& c, cudaStream_t st) { return launch_cg_mixed_loop_n(&c, 1, st); }

template <int SP, bool C12>
static LoopArgs<SP, C12> plain_loop_args(const CgLoopCall& c) {
  LoopArgs<SP, C12> a;
  for (DslashArgs<SP, C12>* d : {&a.dq, &a.ds}) {
    memcpy(&d->g, &c.g, sizeof(Geom));
    d->u.p = reinterpret_cast<decltype(d->u.p)>(c.u.p);
    d->mkappa = (typename RealOf<SP>::type)(-c.kappa);
    d->kappa_dev = c.kappa_dev;
    d->skip = nullptr;
    d->partials = nullptr;
    d->ticket = nullptr;
    d->result = nullptr;
  }
  a.dq.in = make_ref<SP>(c.p, c.g.V);
  a.dq.out = make_ref<SP>(c.q, c.g.V);
  a.dq.b = make_ref<SP>(FieldPtr{}, c.g.V);
  a.ds.in = make_ref<SP>(c.r, c.g.V);
  a.ds.out = make_ref<SP>(c.s, c.g.V);
  a.ds.b = a.dq.b;
  a.x = make_ref<SP>(c.x, c.g.V);
  a.r = make_ref<SP>(c.r, c.g.V);
  a.p = make_ref<SP>(c.p, c.g.V);
  a.q = make_ref<SP>(c.q, c.g.V);
  a.s = make_ref<SP>(c.s, c.g.V);
  a.tl = reinterpret_cast<double2*>(c.tl.p);
  a.n = c.g.V;
  a.sc = c.sc;
  a.partials = c.partials;
  a.y.ctr = reinterpret_cast<unsigned long long*>(c.bar);
  a.y.limit = c.wait_limit;
  a.y.err = c.err;
  return a;
}

// The paper's loop: D^dag reads p into s, D reads s into q.
template <int SP, bool C12>
static LoopArgs<SP, C12> paper_loop_args(const CgLoopCall& c) {
  LoopArgs<SP, C12> a = plain_loop_args<SP, C12>(c);
  a.ds.in = make_ref<SP>(c.p, c.g.V);
  a.ds.out = make_ref<SP>(c.s, c.g.V);
  a.dq.in = make_ref<SP>(c.s, c.g.V);
  a.dq.out = make_ref<SP>(c.q, c.g.V);
  return a;
}

template <int SP, bool C12, bool DT = false>
static cudaError_t paper_loop_launch_t(const CgLoopCall* cs, int n, cudaStream_t st) {
  return loop_launch(cg_paper_loop_kernel<SP, C12, DT>, cg_paper_loop_batch_kernel<SP, C12, DT>,
                     paper_loop_args<SP, C12>, cs, n, cs[0].g.V, st);
}

template <int SP, bool C12, int LANES, bool DT = false>
static cudaError_t loop_launch_t(const CgLoopCall* cs, int n, cudaStream_t st) {
  return loop_launch(cg_loop_kernel<SP, C12, LANES, DT>, cg_loop_batch_kernel<SP, C12, LANES, DT>,
                     plain_loop_args<SP, C12>, cs, n, LANES * cs[0].g.V, st);
}

// ---------------------------------------------------------------- persistent CG loop, FP64 lanes
//
// At the paper's small volumes (up to 16^4) the FP64 loop is bound by latency: each grid barrier
// costs a few microseconds, as much as a phase's arithmetic. With 4, 8 or 16 lanes per site the
// iteration is fused into two passes and two barriers instead of four:
//   A: p_k = s + beta p_{k-1} formed at every neighbour it is read at (p_0 as the prologue left it),
//      q = D p_k, |q|^2; the site's p_k is stored;                          barrier, alpha = gamma/|q|^2
//   B: r_k = r_{k-1} - alpha q formed likewise, s = D^dag r_k, |s|^2, |r_k|^2; x += alpha p_k;
//      the site's r_k is stored;                                            barrier, beta, convergence
// p and r alternate between two buffers, so no pass overwrites a field another lane still reads at a
// neighbour; the vector arithmetic (fma(beta, p, s), fma(-alpha, q, r)) is that of the four-phase
// loop, and the scalars and stopping rule are the same.
struct LanesLoopArgs {
  Geom g;
  GaugeRef<double, false> u;
  const double* kappa_dev;
  double2 *x, *p0, *p1, *r0, *r1, *q, *s;
  CgScalars* sc;
  double* partials;  // 3 x gridDim.x
  LoopSync y;
};

template <int L>
__device__ __forceinline__ void cg_loop_lanes_body(const LanesLoopArgs& a) {
  CgScalars* sc = a.sc;
  if (sc->status != ST_RUNNING) return;  // uniform over the grid
  const int G = gridDim.x;
  double gamma = sc->gamma, rr = sc->rr;
  const double tol2e = sc->tol2 * sc->eta2;
  int iter = sc->iter, status = ST_RUNNING;
  const int maxit = sc->maxit;
  double alpha = 0.0, beta = 0.0;
  const double mk = -*a.kappa_dev;
  int pi = 0, ri = 0;  // which of the two buffers holds p_{k-1} / r_{k-1} (selects, not indexing)
  bool first = true;
  for (;;) {
    // A: q = D p_k, |q|^2
    double nq = 0.0, nw = 0.0;
    if (first) {
      const FusedPass f = {pi ? a.p1 : a.p0, nullptr, 0.0, nullptr, a.q, nullptr, nullptr, 0.0};
      lanes_fused_sites<L, false, false>(a.g, a.u, mk, f, nq, nw);
    } else {
      const FusedPass f = {a.s, pi ? a.p1 : a.p0, beta, pi ? a.p0 : a.p1, a.q, nullptr, nullptr, 0.0};
      lanes_fused_sites<L, false, true>(a.g, a.u, mk, f, nq, nw);
      pi ^= 1;
    }
    first = false;
    double qq;
    if (!loop_sum(nq, a.partials, a.y, &qq)) break;
    if (!(qq > 0.0 && isfinite(qq) && isfinite(gamma))) {
      status = ST_BREAKDOWN;
      break;
    }
    alpha = gamma / qq;
    // B: s = D^dag r_k, |s|^2, |r_k|^2; x += alpha p_k
    double ns = 0.0, nr = 0.0;
    {
      const FusedPass f = {ri ? a.r1 : a.r0, a.q, -alpha, ri ? a.r0 : a.r1, a.s, a.x, pi ? a.p1 : a.p0, alpha};
      lanes_fused_sites<L, true, true>(a.g, a.u, mk, f, ns, nr);
      ri ^= 1;
    }
    double gnew;
    if (!loop_sum2(ns, nr, a.partials + G, a.y, &gnew, &rr)) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) record_residual(sc, iter, rr);
    if (!isfinite(rr)) {
      status = ST_BREAKDOWN;
      break;
    }
    iter += 1;
    if (rr <= tol2e) {
      status = ST_CONVERGED;
      break;
    }
    if (!(isfinite(gnew) && gamma > 0.0)) {
      status = ST_BREAKDOWN;
      break;
    }
    beta = gnew / gamma;
    gamma = gnew;
    if (iter >= maxit) {
      status = ST_MAXIT;
      break;
    }
  }
  if (status == ST_MAXIT) {
    // Stopped between iterations: leave the state every loop starts from, p_k = s + beta p_{k-1} in
    // p0 and r_k in r0 (the same fma the next pass would form), so that a later launch can continue
    // it (cg_resume). Each thread rewrites only the reals it reads; the last barrier ended every
    // neighbour read.
    const double* pold = reinterpret_cast<const double*>(pi ? a.p1 : a.p0);
    const double* rcur = reinterpret_cast<const double*>(a.r1);
    const double* sv = reinterpret_cast<const double*>(a.s);
    double* p0 = reinterpret_cast<double*>(a.p0);
    double* r0 = reinterpret_cast<double*>(a.r0);
    const int ne = 24 * a.g.V;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
      p0[e] = fma(beta, pold[e], sv[e]);
      if (ri) r0[e] = rcur[e];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const bool failed = *(volatile int*)a.y.err != 0;
    sc->status = failed ? ST_BREAKDOWN : status;
    sc->iter = iter;
    sc->gamma = gamma;
    sc->rr = rr;
    sc->alpha = alpha;
    sc->beta = beta;
  }
}

template <int L>
__global__ void __launch_bounds__(kDslashMaxThreads) cg_loop_lanes_kernel(const LanesLoopArgs a) {
  cg_loop_lanes_body<L>(a);
}

template <int L>
__global__ void __launch_bounds__(kDslashMaxThreads) cg_loop_lanes_batch_kernel(const __grid_constant__ LoopBatch<LanesLoopArgs> b) {
  cg_loop_lanes_body<L>(b.a[blockIdx.y]);
}

static LanesLoopArgs lanes_loop_args(const CgLoopCall& c) {
  LanesLoopArgs a;
  memcpy(&a.g, &c.g, sizeof(Geom));
  a.u.p = reinterpret_cast<const double2*>(c.u.p);
  a.kappa_dev = c.kappa_dev;
  a.x = reinterpret_cast<double2*>(c.x.p);
  a.p0 = reinterpret_cast<double2*>(c.p.p);
  a.p1 = reinterpret_cast<double2*>(c.p2.p);
  a.r0 = reinterpret_cast<double2*>(c.r.p);
  a.r1 = reinterpret_cast<double2*>(c.r2.p);
  a.q = reinterpret_cast<double2*>(c.q.p);
  a.s = reinterpret_cast<double2*>(c.s.p);
  a.sc = c.sc;
  a.partials = c.partials;
  a.y.ctr = reinterpret_cast<unsigned long long*>(c.bar);
  a.y.limit = c.wait_limit;
  a.y.err = c.err;
  return a;
}

template <int L>
static cudaError_t lanes_loop_launch_t(const CgLoopCall* cs, int n, cudaStream_t st) {
  return loop_launch(cg_loop_lanes_kernel<L>, cg_loop_lanes_batch_kernel<L>, lanes_loop_args, cs, n, L * cs[0].g.V, st);
}

cudaError_t launch_cg_loop_n(const CgLoopCall* cs, int n, cudaStream_t st) {
  if (n < 1 || !same_shape(cs, n)) return cudaErrorInvalidValue;
  const CgLoopCall& c = cs[0];
  if (c.block <= 0 || c.block > kDslashMaxThreads || c.block % 32 || c.max_grid < 1) return cudaErrorInvalidValue;
  for (int i = 0; i < n; ++i) {
    const CgLoopCall& d = cs[i];
    if (d.x.prec != d.r.prec || d.p.prec != d.r.prec || d.q.prec != d.r.prec || d.s.prec != d.r.prec)
      return cudaErrorInvalidValue;
    if (d.r.prec == SP64 && d.variant >= 2 &&
        (!d.p2.p || !d.r2.p || d.p2.prec != SP64 || d.r2.prec != SP64))
      return cudaErrorInvalidValue;
    if (d.r.prec == SP64 && d.variant == 0 && d.time_basis && !d.tl.p) return cudaErrorInvalidValue;
  }
  if (c.cg_form) {  // one thread per site, the paper's CG form
    if (c.variant != 0) return cudaErrorInvalidValue;
    if (c.r.prec == SP64 && c.u.prec == SP64)
      return c.time_basis ? paper_loop_launch_t<P64, false, true>(cs, n, st) : paper_loop_launch_t<P64, false>(cs, n, st);
    if (c.r.prec == SP32 && c.u.prec == SP32)
      return c.u.c12 ? paper_loop_launch_t<P32, true>(cs, n, st) : paper_loop_launch_t<P32, false>(cs, n, st);
    return cudaErrorInvalidValue;
  }
  if (c.r.prec == SP64) {
    if (c.u.prec != SP64) return cudaErrorInvalidValue;
    switch (c.variant) {
      case 0: return c.time_basis ? loop_launch_t<P64, false, 1, true>(cs, n, st) : loop_launch_t<P64, false, 1>(cs, n, st);
      case 1: return loop_launch_t<P64, false, 2>(cs, n, st);
      case 2: return lanes_loop_launch_t<4>(cs, n, st);
      case 3: return lanes_loop_launch_t<8>(cs, n, st);
      case 4: return lanes_loop_launch_t<16>(cs, n, st);
    }
    return cudaErrorInvalidValue;
  }
  if (c.r.prec == SP32 && c.u.prec == SP32)
    return c.u.c12 ? loop_launch_t<P32, true, 1>(cs, n, st) : loop_launch_t<P32, false, 1>(cs, n, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_cg_loop(const CgLoopCall& c, cudaStream_t st) { return launch_cg_loop_n(&c, 1, st); }

// ---------------------------------------------------------------- persistent CG loop, even-odd
//
// The plain CGLS loop on M = 1 - kappa^2 H_eo H_oe over the even sites, in one cooperative launch:
// each application of M (or M^dag) is two half-lattice passes through the odd temporary t with a
// grid barrier between them; the vector updates run over the even half. Six barriers per
// iteration; the scalars and the stopping rule are those of the lexicographic loop.
template <int SP, bool C12>
struct EoLoopArgs {
  EoArgs<SP, C12> pt, tq, rt, ts;  // t = kappa H_oe p; q = p - kappa H_eo t; the same with H^dag for r -> s
  SpinorRef<SP> x, r, p, q, s;
  int n;                           // even sites (V / 2)
  CgScalars* sc;
  double* partials;
  LoopSync y;
};

template <int SP, bool C12>
__global__ void __launch_bounds__(kDslashMaxThreads, DslashMinBlocks<SP>::value)
    cg_eo_loop_kernel(const EoLoopArgs<SP, C12> a) {
  typedef typename RealOf<SP>::type R;
  CgScalars* sc = a.sc;
  if (sc->status != ST_RUNNING) return;  // uniform over the grid
  const int n = a.n, V = a.pt.e.g.V, G = gridDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, tstep = G * blockDim.x;
  double gamma = sc->gamma, rr = sc->rr;
  const double tol2e = sc->tol2 * sc->eta2;
  int iter = sc->iter, status = ST_RUNNING;
  const int maxit = sc->maxit;
  double alpha = 0.0, beta = 0.0;
  for (;;) {
    // q = M p, |q|^2
    for (int i = t0; i < n; i += tstep) (void)eo_site<SP, C12, false, false, false>(a.pt, i);
    if (!grid_barrier(a.y)) break;
    double v = 0.0;
    for (int i = t0; i < n; i += tstep) v += eo_site<SP, C12, false, true, false>(a.tq, i);
    double qq;
    if (!loop_sum(v, a.partials, a.y, &qq)) break;
    if (!(qq > 0.0 && isfinite(qq) && isfinite(gamma))) {
      status = ST_BREAKDOWN;
      break;
    }
    alpha = gamma / qq;
    const R ar = (R)alpha;
    // r -= alpha q, |r|^2
    v = 0.0;
    for (int i = t0; i < n; i += tstep) {
      Cx<R> rv[12], qv[12];
      load_spinor(a.r, i, V, rv);
      load_spinor(a.q, i, V, qv);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        rv[c].re = fma(-ar, qv[c].re, rv[c].re);
        rv[c].im = fma(-ar, qv[c].im, rv[c].im);
      }
      store_spinor(a.r, i, V, rv);
      v += norm2_site(rv);
    }
    if (!loop_sum(v, a.partials + G, a.y, &rr)) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) record_residual(sc, iter, rr);
    if (!isfinite(rr)) {
      status = ST_BREAKDOWN;
      break;
    }
    const bool conv = rr <= tol2e;
    // s = M^dag r, |s|^2 (not needed once converged)
    double gnew = 0.0;
    if (!conv) {
      for (int i = t0; i < n; i += tstep) (void)eo_site<SP, C12, true, false, false>(a.rt, i);
      if (!grid_barrier(a.y)) break;
      v = 0.0;
      for (int i = t0; i < n; i += tstep) v += eo_site<SP, C12, true, true, false>(a.ts, i);
      if (!loop_sum(v, a.partials + 2 * G, a.y, &gnew)) break;
    }
    const bool do_p = !conv && isfinite(gnew) && gamma > 0.0;
    beta = do_p ? gnew / gamma : 0.0;
    const R br = (R)beta;
    // x += alpha p; p = s + beta p
    for (int i = t0; i < n; i += tstep) {
      Cx<R> xv[12], pv[12];
      load_spinor(a.x, i, V, xv);
      load_spinor(a.p, i, V, pv);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        xv[c].re = fma(ar, pv[c].re, xv[c].re);
        xv[c].im = fma(ar, pv[c].im, xv[c].im);
      }
      store_spinor(a.x, i, V, xv);
      if (do_p) {
        Cx<R> sv[12];
        load_spinor(a.s, i, V, sv);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          pv[c].re = fma(br, pv[c].re, sv[c].re);
          pv[c].im = fma(br, pv[c].im, sv[c].im);
        }
        store_spinor(a.p, i, V, pv);
      }
    }
    iter += 1;
    if (conv) {
      status = ST_CONVERGED;
      break;
    }
    if (!do_p) {
      status = ST_BREAKDOWN;
      break;
    }
    gamma = gnew;
    if (iter >= maxit) {
      status = ST_MAXIT;
      break;
    }
    if (!grid_barrier(a.y)) break;  // p complete before the next pass reads its neighbours
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const bool failed = *(volatile int*)a.y.err != 0;
    sc->status = failed ? ST_BREAKDOWN : status;
    sc->iter = iter;
    sc->gamma = gamma;
    sc->rr = rr;
    sc->alpha = alpha;
    sc->beta = beta;
  }
}

template <int SP, bool C12>
static void eo_args(EoArgs<SP, C12>& e, const CgLoopCall& c, FieldPtr in, FieldPtr out, const FieldPtr* self,
                    int parity, double sign) {
  memset(&e, 0, sizeof(e));
  memcpy(&e.e.g, &c.g, sizeof(Geom));
  e.e.parity = parity;
  e.e.sign = sign;
  e.e.kappa_dev = c.kappa_dev;
  e.u.p = reinterpret_cast<decltype(e.u.p)>(c.u.p);
  e.in = make_ref<SP>(in, c.g.V);
  e.out = make_ref<SP>(out, c.g.V);
  if (self) e.self = make_ref<SP>(*self, c.g.V);
}

template <int SP, bool C12>
static cudaError_t eo_loop_launch_t(const CgLoopCall& c, cudaStream_t st) {
  EoLoopArgs<SP, C12> a;
  eo_args(a.pt, c, c.p, c.t, nullptr, 1, +1.0);
  eo_args(a.tq, c, c.t, c.q, &c.p, 0, -1.0);
  eo_args(a.rt, c, c.r, c.t, nullptr, 1, +1.0);
  eo_args(a.ts, c, c.t, c.s, &c.r, 0, -1.0);
  a.x = make_ref<SP>(c.x, c.g.V);
  a.r = make_ref<SP>(c.r, c.g.V);
  a.p = make_ref<SP>(c.p, c.g.V);
  a.q = make_ref<SP>(c.q, c.g.V);
  a.s = make_ref<SP>(c.s, c.g.V);
  a.n = c.g.V / 2;
  a.sc = c.sc;
  a.partials = c.partials;
  a.y.ctr = reinterpret_cast<unsigned long long*>(c.bar);
  a.y.limit = c.wait_limit;
  a.y.err = c.err;
  auto k = cg_eo_loop_kernel<SP, C12>;
  int grid = resident_blocks(reinterpret_cast<const void*>(k), c.block);
  const int need = grid_for(c.g.V / 2, c.block);
  if (need < grid) grid = need;
  if (grid > c.max_grid) grid = c.max_grid;
  void* args[] = {&a};
  cudaError_t e = cudaMemsetAsync(c.bar, 0, sizeof(unsigned long long), st);  // barrier count of this launch
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k), dim3(grid), dim3(c.block), args, 0, st);
}

cudaError_t launch_cg_eo_loop(const CgLoopCall& c, cudaStream_t st) {
  if (c.block <= 0 || c.block > kDslashMaxThreads || c.block % 32 || c.max_grid < 1 || !c.t.p) return cudaErrorInvalidValue;
  if (c.x.prec != c.r.prec || c.p.prec != c.r.prec || c.q.prec != c.r.prec || c.s.prec != c.r.prec ||
      c.t.prec != c.r.prec)
    return cudaErrorInvalidValue;
  if (c.r.prec == SP64) {
    if (c.u.prec != SP64) return cudaErrorInvalidValue;
    return eo_loop_launch_t<P64, false>(c, st);
  }
  if (c.r.prec == SP32 && c.u.prec == SP32)
    return c.u.c12 ? eo_loop_launch_t<P32, true>(c, st) : eo_loop_launch_t<P32, false>(c, st);
  return cudaErrorInvalidValue;
}

}  // namespace wdk
