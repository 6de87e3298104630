// The Wilson-Dirac hopping kernel (dslash) of Eq. (1), for every storage precision.
//
// One thread per site n. For each of the 8 hops it loads the neighbour spinor, projects it to a
// half-spinor with (1 -/+ gamma_mu) (chiral basis, see wd_device.cuh), multiplies the two colour
// vectors by U_mu(n) or U_mu(n - mu)^dagger, reconstructs the four spins and accumulates with
// the factor -kappa * boundary phase. The accumulator starts from psi(n), so the diagonal term of
// D costs nothing extra. Epilogues: out = D in (EPI_PLAIN) or out = b - D in (EPI_RESID), with an
// optional fused ||out||^2 (deterministic grid reduction).
//
// Arithmetic per site: 8 x (12 projection adds + 72 SU(3) FMA/MUL + 24 reconstruction FMA)
// = 864 FP instructions for 1320 hopping flops + 48 diagonal flops (the usual convention counts
// 1320). Bytes per site at minimum: 1 spinor in + 1 out + 4 links.
#include "wd_device.cuh"
#include "wd_internal.h"

namespace wdk {

template <int SP>
struct RealOf {
  typedef float type;
};
template <>
struct RealOf<P64> {
  typedef double type;
};
template <>
struct RealOf<PDF> {
  typedef dfloat type;
};

// device view of a field (hi/lo halves for double-float)
template <int SP>
__host__ SpinorRef<SP> make_ref(FieldPtr f, int V) {
  SpinorRef<SP> r;
  if constexpr (SP == PDF) {
    r.hi = reinterpret_cast<float4*>(f.p);
    r.lo = f.p ? reinterpret_cast<float4*>(f.p) + (size_t)6 * V : nullptr;
  } else {
    r.p = reinterpret_cast<decltype(r.p)>(f.p);
    if constexpr (SP == P16) r.norm = f.norm;
  }
  return r;
}

template <int SP, bool C12>
struct DslashArgs {
  Geom g;
  GaugeRef<typename RealOf<SP>::type, C12> u;
  SpinorRef<SP> in, out, b;
  typename RealOf<SP>::type mkappa;  // -kappa (used when kappa_dev is null)
  const double* kappa_dev;
  const int* skip;
  double* partials;
  unsigned* ticket;
  double* result;
};

template <int MU, int S_FWD, int SP, bool C12, typename R>
__device__ __forceinline__ void hop_pair(const DslashArgs<SP, C12>& a, R mk, int s, const int (&c)[4],
                                         Cx<R> (&acc)[12]) {
  const int V = a.g.V;
  // forward hop n -> n + mu with U_mu(n)
  {
    const bool wrap = c[MU] == a.g.L[MU] - 1;
    const int nb = wrap ? s - (a.g.L[MU] - 1) * a.g.stride[MU] : s + a.g.stride[MU];
    Cx<R> psi[12];
    const R k = load_hop_spinor(a.in, nb, V, psi, (wrap && a.g.bc[MU] < 0) ? -mk : mk);
    Cx<R> h[6];
    spin_project<MU, S_FWD>(psi, h);
    Cx<R> u[9];
    load_link(a.u, MU, s, V, u);
    Cx<R> chi[6];
    su3_mul(u, h, chi);
    spin_reconstruct<MU, S_FWD>(acc, chi, k);
  }
  // backward hop n -> n - mu with U_mu(n - mu)^dagger and the opposite projector
  {
    const bool wrap = c[MU] == 0;
    const int nb = wrap ? s + (a.g.L[MU] - 1) * a.g.stride[MU] : s - a.g.stride[MU];
    Cx<R> psi[12];
    const R k = load_hop_spinor(a.in, nb, V, psi, (wrap && a.g.bc[MU] < 0) ? -mk : mk);
    Cx<R> h[6];
    spin_project<MU, -S_FWD>(psi, h);
    Cx<R> u[9];
    load_link(a.u, MU, nb, V, u);
    Cx<R> chi[6];
    su3_dag_mul(u, h, chi);
    spin_reconstruct<MU, -S_FWD>(acc, chi, k);
  }
}

// All 8 hops in a runtime loop (one copy of the per-hop code): for double-float arithmetic, whose
// unrolled form overflows the instruction cache.
template <int SF, int SP, bool C12, typename R>
__device__ __forceinline__ void hops_rt(const DslashArgs<SP, C12>& a, R mk, int s, const int (&c)[4], Cx<R> (&acc)[12]) {
  const int V = a.g.V;
#pragma unroll 1
  for (int hop = 0; hop < 8; ++hop) {
    const int mu = hop >> 1, dir = hop & 1;
    const int cm = mu == 0 ? c[0] : (mu == 1 ? c[1] : (mu == 2 ? c[2] : c[3]));
    const int L = a.g.L[mu], st = a.g.stride[mu];
    const bool wrap = dir == 0 ? cm == L - 1 : cm == 0;
    const int nb = dir == 0 ? (wrap ? s - (L - 1) * st : s + st) : (wrap ? s + (L - 1) * st : s - st);
    const R k = (wrap && a.g.bc[mu] < 0) ? -mk : mk;
    const int S = dir == 0 ? SF : -SF;
    Cx<R> psi[12], h[6], u[9], chi[6];
    load_spinor(a.in, nb, V, psi);
    spin_project_rt(mu, S, psi, h);
    load_link(a.u, mu, dir == 0 ? s : nb, V, u);
    if (dir == 0)
      su3_mul(u, h, chi);
    else
      su3_dag_mul(u, h, chi);
    spin_reconstruct_rt(mu, S, acc, chi, k);
  }
}

// One site of out = D in (or b - D in); returns |out(s)|^2.
template <int SP, bool C12, bool DAG, int EPI>
__device__ __forceinline__ double dslash_site(const DslashArgs<SP, C12>& a, int s) {
  typedef typename RealOf<SP>::type R;
  const int V = a.g.V;
  int c[4];
  {
    int r = s;
    c[0] = r % a.g.L[0];
    r /= a.g.L[0];
    c[1] = r % a.g.L[1];
    r /= a.g.L[1];
    c[2] = r % a.g.L[2];
    c[3] = r / a.g.L[2];
  }
  const R mk = a.kappa_dev ? (R)(-*a.kappa_dev) : a.mkappa;
  Cx<R> acc[12];
  load_spinor(a.in, s, V, acc);
  // D: forward (1 - gamma), backward (1 + gamma); D^dagger: the reverse
  constexpr int SF = DAG ? +1 : -1;
  if constexpr (SP == PDF) {
    hops_rt<SF>(a, mk, s, c, acc);
  } else {
    hop_pair<0, SF>(a, mk, s, c, acc);
    hop_pair<1, SF>(a, mk, s, c, acc);
    hop_pair<2, SF>(a, mk, s, c, acc);
    hop_pair<3, SF>(a, mk, s, c, acc);
  }
  if (EPI == EPI_RESID) {
    Cx<R> bv[12];
    load_spinor(a.b, s, V, bv);
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = cx<R>(bv[i].re - acc[i].re, bv[i].im - acc[i].im);
  }
  store_spinor(a.out, s, V, acc);
  return norm2_site(acc);
}

// Occupancy: the kernel is latency-bound at large volumes (memory-level parallelism comes from
// resident warps), so registers are capped for 3 blocks of 256 threads per SM in FP32/FP16
// (24 warps) and 2 in FP64 (whose FP64 pipe saturates with few warps).
constexpr int kDslashMaxThreads = 256;
template <int SP>
struct DslashMinBlocks {
  static constexpr int value = SP == P64 ? 2 : (SP == PDF ? 1 : 3);
};

template <int SP, bool C12, bool DAG, int EPI, bool NORM>
__global__ void __launch_bounds__(kDslashMaxThreads, DslashMinBlocks<SP>::value)
    dslash_kernel(const DslashArgs<SP, C12> a) {
  if (a.skip != nullptr && *a.skip != 0) return;  // uniform over the grid
  const int V = a.g.V;
  double n2 = 0.0;
  // grid-stride over sites: the launch is one wave of resident blocks, so the fused norm has one
  // partial per resident block and no block waits in a queue
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += gridDim.x * blockDim.x) {
    const double v = dslash_site<SP, C12, DAG, EPI>(a, s);
    if (NORM) n2 += v;
  }
  if (NORM) {
    double v[1] = {n2}, tot[1];
    if (grid_reduce<OpSum, 1>(v, a.partials, a.ticket, tot) && threadIdx.x == 0) *a.result = tot[0];
  }
}

// ---------------------------------------------------------------- FP64: two threads per site
//
// The FP64 dslash is bound by the FP64 pipe. At the paper's volumes (14^4 = 38,416 sites) one
// thread per site leaves 8 warps per SM, too few to keep that pipe fed through the load and
// dependency latencies. Here lanes 2i and 2i+1 share a site: lane h projects only the half-spinor
// row h, multiplies it by the link and reconstructs it, so both lanes run the same instructions
// (no divergence) and together execute the same FP64 operations as one thread of dslash_kernel.
// Row h of (1 -/+ gamma_mu) pairs upper spin h with lower spin 2 + pi(h), pi(h) = 1 - h for x, y
// (B_mu off-diagonal) and h for z, t, with the coefficient B_mu[h][pi(h)] = sigma * i^e; the
// reconstructed row feeds upper spin h and lower spin 2 + pi(h) with S conj(B_mu[h][pi(h)]).
// Lane h accumulates its upper spin, its own lower spin 2 + h (z, t hops) and the partner's
// lower spin (x, y hops), which the lanes exchange with one shuffle at the end.

__device__ __forceinline__ Cx<double> shfl_xor_cx(Cx<double> z, int m) {
  return cx(__shfl_xor_sync(0xffffffffu, z.re, m), __shfl_xor_sync(0xffffffffu, z.im, m));
}

template <int MU, int DIR, int SF, bool C12>
__device__ __forceinline__ void pair_hop(const DslashArgs<P64, C12>& a, double mk, int s, const int (&c)[4], int hl,
                                         Cx<double> (&au)[3], Cx<double> (&ald)[3], Cx<double> (&alo)[3]) {
  constexpr int S = DIR == 0 ? SF : -SF;  // projector sign: forward (1 + SF gamma), backward the opposite
  constexpr int E = (MU == 0 || MU == 2) ? 1 : 0;
  const int V = a.g.V;
  bool wrap;
  int nb;
  if (DIR == 0) {
    wrap = c[MU] == a.g.L[MU] - 1;
    nb = wrap ? s - (a.g.L[MU] - 1) * a.g.stride[MU] : s + a.g.stride[MU];
  } else {
    wrap = c[MU] == 0;
    nb = wrap ? s + (a.g.L[MU] - 1) * a.g.stride[MU] : s - a.g.stride[MU];
  }
  const double k = (wrap && a.g.bc[MU] < 0) ? -mk : mk;
  // sigma: B_mu[h][pi(h)] = sigma i^E
  const double sigma = MU == 0 ? -1.0 : (MU == 3 ? 1.0 : (hl ? 1.0 : -1.0));
  const double ssig = S > 0 ? sigma : -sigma;
  const int lower = (MU < 2) ? 3 - hl : 2 + hl;  // spin paired with upper spin hl
  Cx<double> hh[3];
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    const double2 pu = __ldg(a.in.p + (size_t)(3 * hl + col) * V + nb);
    const double2 pl = __ldg(a.in.p + (size_t)(3 * lower + col) * V + nb);
    if (E == 0)
      hh[col] = cx(fma(ssig, pl.x, pu.x), fma(ssig, pl.y, pu.y));
    else  // i z = (-z.im, z.re)
      hh[col] = cx(fma(-ssig, pl.y, pu.x), fma(ssig, pl.x, pu.y));
  }
  Cx<double> u[9];
  load_link(a.u, MU, DIR == 0 ? s : nb, V, u);
  Cx<double> chi[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    Cx<double> u0, u1, u2;
    if (DIR == 0) {
      u0 = u[3 * r];
      u1 = u[3 * r + 1];
      u2 = u[3 * r + 2];
    } else {
      u0 = conj_(u[r]);
      u1 = conj_(u[3 + r]);
      u2 = conj_(u[6 + r]);
    }
    double re = u0.re * hh[0].re;
    re = fma(-u0.im, hh[0].im, re);
    re = fma(u1.re, hh[1].re, re);
    re = fma(-u1.im, hh[1].im, re);
    re = fma(u2.re, hh[2].re, re);
    re = fma(-u2.im, hh[2].im, re);
    double im = u0.re * hh[0].im;
    im = fma(u0.im, hh[0].re, im);
    im = fma(u1.re, hh[1].im, im);
    im = fma(u1.im, hh[1].re, im);
    im = fma(u2.re, hh[2].im, im);
    im = fma(u2.im, hh[2].re, im);
    chi[r] = cx(re, im);
  }
  // upper spin hl += k chi; lower spin 2 + pi(hl) += k S conj(sigma i^E) chi = k S sigma (-i)^E chi
  const double kl = k * ssig;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    au[r].re = fma(k, chi[r].re, au[r].re);
    au[r].im = fma(k, chi[r].im, au[r].im);
    Cx<double>& t = (MU < 2) ? alo[r] : ald[r];
    if (E == 0) {
      t.re = fma(kl, chi[r].re, t.re);
      t.im = fma(kl, chi[r].im, t.im);
    } else {  // (-i) z = (z.im, -z.re)
      t.re = fma(kl, chi[r].im, t.re);
      t.im = fma(-kl, chi[r].re, t.im);
    }
  }
}

// All sites of out = D in (or b - D in) with two lanes per site, over the whole grid (grid-stride
// on the warp's first site); returns this thread's share of |out|^2.
template <bool C12, bool DAG, int EPI>
__device__ __forceinline__ double pair_sites(const DslashArgs<P64, C12>& a) {
  const int V = a.g.V;
  const int hl = threadIdx.x & 1;
  double n2 = 0.0;
  const int step = (gridDim.x * blockDim.x) >> 1;
  // The loop runs on the warp's first site, so all 32 lanes take the same trips and meet at the
  // full-warp shuffle below; lanes past the last site recompute the warp's first site and store
  // nothing.
  for (int s0 = (blockIdx.x * blockDim.x + (threadIdx.x & ~31)) >> 1; s0 < V; s0 += step) {
    const int sl = s0 + ((threadIdx.x & 31) >> 1);
    const bool live = sl < V;
    const int s = live ? sl : s0;
    int c[4];
    {
      int r = s;
      c[0] = r % a.g.L[0];
      r /= a.g.L[0];
      c[1] = r % a.g.L[1];
      r /= a.g.L[1];
      c[2] = r % a.g.L[2];
      c[3] = r / a.g.L[2];
    }
    const double mk = a.kappa_dev ? -*a.kappa_dev : a.mkappa;
    Cx<double> au[3], ald[3], alo[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      const double2 pu = __ldg(a.in.p + (size_t)(3 * hl + col) * V + s);
      const double2 pl = __ldg(a.in.p + (size_t)(3 * (2 + hl) + col) * V + s);
      au[col] = cx(pu.x, pu.y);
      ald[col] = cx(pl.x, pl.y);
      alo[col] = cx(0.0, 0.0);
    }
    constexpr int SF = DAG ? +1 : -1;
    pair_hop<0, 0, SF>(a, mk, s, c, hl, au, ald, alo);
    pair_hop<0, 1, SF>(a, mk, s, c, hl, au, ald, alo);
    pair_hop<1, 0, SF>(a, mk, s, c, hl, au, ald, alo);
    pair_hop<1, 1, SF>(a, mk, s, c, hl, au, ald, alo);
    pair_hop<2, 0, SF>(a, mk, s, c, hl, au, ald, alo);
    pair_hop<2, 1, SF>(a, mk, s, c, hl, au, ald, alo);
    pair_hop<3, 0, SF>(a, mk, s, c, hl, au, ald, alo);
    pair_hop<3, 1, SF>(a, mk, s, c, hl, au, ald, alo);
    // lower spin 2 + hl: own z, t part + the partner's x, y part
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      const Cx<double> o = shfl_xor_cx(alo[col], 1);
      ald[col] = cx(ald[col].re + o.re, ald[col].im + o.im);
    }
    if (!live) continue;  // after the shuffle: the loop condition is warp-uniform
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      Cx<double> up = au[col], lo = ald[col];
      if (EPI == EPI_RESID) {
        const double2 bu = __ldg(a.b.p + (size_t)(3 * hl + col) * V + s);
        const double2 bl = __ldg(a.b.p + (size_t)(3 * (2 + hl) + col) * V + s);
        up = cx(bu.x - up.re, bu.y - up.im);
        lo = cx(bl.x - lo.re, bl.y - lo.im);
      }
      a.out.p[(size_t)(3 * hl + col) * V + s] = make_double2(up.re, up.im);
      a.out.p[(size_t)(3 * (2 + hl) + col) * V + s] = make_double2(lo.re, lo.im);
      n2 = fma(up.re, up.re, n2);
      n2 = fma(up.im, up.im, n2);
      n2 = fma(lo.re, lo.re, n2);
      n2 = fma(lo.im, lo.im, n2);
    }
  }
  return n2;
}

template <bool C12, bool DAG, int EPI, bool NORM>
__global__ void __launch_bounds__(kDslashMaxThreads, 2) dslash_pair_kernel(const DslashArgs<P64, C12> a) {
  if (a.skip != nullptr && *a.skip != 0) return;  // uniform over the grid
  const double n2 = pair_sites<C12, DAG, EPI>(a);
  if (NORM) {
    double v[1] = {n2}, tot[1];
    if (grid_reduce<OpSum, 1>(v, a.partials, a.ticket, tot) && threadIdx.x == 0) *a.result = tot[0];
  }
}

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
  unsigned* bar;  // [0] arrivals, [1] generation
  int* err;       // set to 1 when a barrier wait gave up
};

constexpr long long kBarrierSpinLimit = 1LL << 26;  // x 64 ns sleep: about 4 s

// All blocks arrive, then continue. Returns false (everywhere, eventually) if a wait gave up.
__device__ __forceinline__ bool grid_barrier(const LoopSync& y) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = y.bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(y.bar, 1u);
    int good = 1;
    if (arrived == gridDim.x - 1) {
      y.bar[0] = 0u;
      __threadfence();
      atomicAdd(y.bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g0) {
        if (++spins > kBarrierSpinLimit || *(volatile int*)y.err) {
          atomicExch(y.err, 1);
          good = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = good && !*(volatile int*)y.err;
  }
  __syncthreads();
  return ok;
}

// Sum over the grid of one value per thread: block partial, barrier, then every block sums the
// partials in the same order (lanes stride over them, then a fixed shuffle tree).
__device__ __forceinline__ bool loop_sum(double v, double* partials, const LoopSync& y, double* out) {
  __shared__ double smem[32];
  __shared__ double total;
  double w[1] = {v};
  block_reduce<OpSum, 1>(w, smem);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = w[0];
    __threadfence();
  }
  if (!grid_barrier(y)) return false;
  if (threadIdx.x < 32) {
    double a = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) a += __ldcg(partials + b);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (threadIdx.x == 0) total = a;
  }
  __syncthreads();
  *out = total;
  return true;
}

template <int SP, bool C12>
struct LoopArgs {
  DslashArgs<SP, C12> dq;  // q = D p
  DslashArgs<SP, C12> ds;  // s = D^dag r
  SpinorRef<SP> x, r, p, q, s;
  int n;                   // sites
  CgScalars* sc;
  double* partials;        // 3 x gridDim.x
  LoopSync y;
};

// The dslash phases of the loop: one thread per site, or (FP64, PAIR) two lanes per site.
template <int SP, bool C12, bool DAG, bool PAIR>
__device__ __forceinline__ double loop_dslash(const DslashArgs<SP, C12>& d, int n, int t0, int tstep) {
  if constexpr (SP == P64 && PAIR) {
    return pair_sites<C12, DAG, EPI_PLAIN>(d);
  } else {
    double v = 0.0;
    for (int i = t0; i < n; i += tstep) v += dslash_site<SP, C12, DAG, EPI_PLAIN>(d, i);
    return v;
  }
}

template <int SP, bool C12, bool PAIR>
__global__ void __launch_bounds__(kDslashMaxThreads, DslashMinBlocks<SP>::value) cg_loop_kernel(const LoopArgs<SP, C12> a) {
  typedef typename RealOf<SP>::type R;
  CgScalars* sc = a.sc;
  if (sc->status != ST_RUNNING) return;  // uniform over the grid
  const int n = a.n, V = a.dq.g.V, G = gridDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, tstep = G * blockDim.x;
  double gamma = sc->gamma, rr = sc->rr;
  const double tol2e = sc->tol2 * sc->eta2;
  int iter = sc->iter, status = ST_RUNNING;
  const int maxit = sc->maxit;
  double alpha = 0.0, beta = 0.0;
  for (;;) {
    // q = D p, |q|^2
    double v = loop_dslash<SP, C12, false, PAIR>(a.dq, n, t0, tstep);
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
    if (!isfinite(rr)) {
      status = ST_BREAKDOWN;
      break;
    }
    const bool conv = rr <= tol2e;
    // s = D^dag r, |s|^2 (not needed once converged)
    double gnew = 0.0;
    if (!conv) {
      v = loop_dslash<SP, C12, true, PAIR>(a.ds, n, t0, tstep);
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
    if (!grid_barrier(a.y)) break;  // p complete before the next dslash reads its neighbours
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
__global__ void __launch_bounds__(kDslashMaxThreads, DslashMinBlocks<SPW>::value)
    cg_mixed_loop_kernel(const MixedLoopArgs<SPW, C12> a) {
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
static cudaError_t mixed_loop_launch_t(const CgLoopCall& c, cudaStream_t st) {
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
  a.y.bar = c.bar;
  a.y.err = c.err;
  auto k = cg_mixed_loop_kernel<SPW, C12>;
  int grid = resident_blocks(reinterpret_cast<const void*>(k), c.block);
  const int need = grid_for(c.g.V, c.block);
  if (need < grid) grid = need;
  if (grid > c.max_grid) grid = c.max_grid;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k), dim3(grid), dim3(c.block), args, 0, st);
}

cudaError_t launch_cg_mixed_loop(const CgLoopCall& c, cudaStream_t st) {
  if (c.block <= 0 || c.block > kDslashMaxThreads || c.block % 32 || c.max_grid < 1) return cudaErrorInvalidValue;
  if (c.x.prec != SP32 || c.u.prec != SP32 || c.p.prec != c.r.prec || c.q.prec != c.r.prec || c.s.prec != c.r.prec)
    return cudaErrorInvalidValue;
  if (c.r.prec == SP32) return c.u.c12 ? mixed_loop_launch_t<P32, true>(c, st) : mixed_loop_launch_t<P32, false>(c, st);
  if (c.r.prec == SP16) return c.u.c12 ? mixed_loop_launch_t<P16, true>(c, st) : mixed_loop_launch_t<P16, false>(c, st);
  return cudaErrorInvalidValue;
}

template <int SP, bool C12, bool PAIR>
static cudaError_t loop_launch_t(const CgLoopCall& c, cudaStream_t st) {
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
  a.n = c.g.V;
  a.sc = c.sc;
  a.partials = c.partials;
  a.y.bar = c.bar;
  a.y.err = c.err;
  auto k = cg_loop_kernel<SP, C12, PAIR>;
  int grid = resident_blocks(reinterpret_cast<const void*>(k), c.block);
  const int need = grid_for(PAIR ? 2 * c.g.V : c.g.V, c.block);
  if (need < grid) grid = need;
  if (grid > c.max_grid) grid = c.max_grid;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k), dim3(grid), dim3(c.block), args, 0, st);
}

cudaError_t launch_cg_loop(const CgLoopCall& c, cudaStream_t st) {
  if (c.block <= 0 || c.block > kDslashMaxThreads || c.block % 32 || c.max_grid < 1) return cudaErrorInvalidValue;
  if (c.x.prec != c.r.prec || c.p.prec != c.r.prec || c.q.prec != c.r.prec || c.s.prec != c.r.prec)
    return cudaErrorInvalidValue;
  if (c.r.prec == SP64) {
    if (c.u.prec != SP64) return cudaErrorInvalidValue;
    return c.variant == 1 ? loop_launch_t<P64, false, true>(c, st) : loop_launch_t<P64, false, false>(c, st);
  }
  if (c.r.prec == SP32 && c.u.prec == SP32)
    return c.u.c12 ? loop_launch_t<P32, true, false>(c, st) : loop_launch_t<P32, false, false>(c, st);
  return cudaErrorInvalidValue;
}

template <int SP, bool C12, bool DAG, int EPI>
static cudaError_t launch_t(const DslashCall& c, cudaStream_t st) {
  DslashArgs<SP, C12> a;
  static_assert(sizeof(GeomH) == sizeof(Geom), "geometry mirror");
  memcpy(&a.g, &c.g, sizeof(Geom));
  a.u.p = reinterpret_cast<decltype(a.u.p)>(c.u.p);
  a.in = make_ref<SP>(c.in, c.g.V);
  a.out = make_ref<SP>(c.out, c.g.V);
  a.b = make_ref<SP>(c.b, c.g.V);
  a.mkappa = (typename RealOf<SP>::type)(-c.kappa);
  a.kappa_dev = c.kappa_dev;
  a.skip = c.skip;
  a.partials = c.red.partials;
  a.ticket = c.red.ticket;
  a.result = c.red.result;
  if constexpr (SP == P64 && !C12) {
    if (c.variant == 1) {  // two lanes per site
      if (c.red.result) {
        auto k = dslash_pair_kernel<C12, DAG, EPI, true>;
        k<<<stride_grid(k, 2 * c.g.V, c.block), c.block, 0, st>>>(a);
      } else {
        auto k = dslash_pair_kernel<C12, DAG, EPI, false>;
        k<<<stride_grid(k, 2 * c.g.V, c.block), c.block, 0, st>>>(a);
      }
      return cudaGetLastError();
    }
  }
  if (c.red.result) {
    auto k = dslash_kernel<SP, C12, DAG, EPI, true>;
    k<<<stride_grid(k, c.g.V, c.block), c.block, 0, st>>>(a);
  } else {
    auto k = dslash_kernel<SP, C12, DAG, EPI, false>;
    k<<<stride_grid(k, c.g.V, c.block), c.block, 0, st>>>(a);
  }
  return cudaGetLastError();
}

template <int SP, bool C12>
static cudaError_t launch_p(const DslashCall& c, cudaStream_t st) {
  if (c.dagger) {
    return c.epi == EPI_RESID ? launch_t<SP, C12, true, EPI_RESID>(c, st) : launch_t<SP, C12, true, EPI_PLAIN>(c, st);
  }
  return c.epi == EPI_RESID ? launch_t<SP, C12, false, EPI_RESID>(c, st) : launch_t<SP, C12, false, EPI_PLAIN>(c, st);
}

cudaError_t launch_dslash(const DslashCall& c, cudaStream_t st) {
  if (c.block <= 0 || c.block > kDslashMaxThreads || c.block % 32) return cudaErrorInvalidValue;
  if (c.variant != 0 && (c.variant != 1 || c.in.prec != SP64)) return cudaErrorInvalidValue;
  if (c.in.prec == SPDF) {
    if (c.u.prec != SPDF) return cudaErrorInvalidValue;
    return launch_p<PDF, false>(c, st);
  }
  if (c.in.prec == SP64) {
    if (c.u.prec != SP64) return cudaErrorInvalidValue;
    return launch_p<P64, false>(c, st);
  }
  if (c.u.prec != SP32) return cudaErrorInvalidValue;
  if (c.in.prec == SP32) return c.u.c12 ? launch_p<P32, true>(c, st) : launch_p<P32, false>(c, st);
  if (c.in.prec == SP16) return c.u.c12 ? launch_p<P16, true>(c, st) : launch_p<P16, false>(c, st);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- even-odd (Schur) hopping
//
// With all extents even, sites split into parities p = (x + y + z + t) mod 2 and the hopping term
// H of D = 1 - kappa H only connects opposite parities. An even-odd context stores every field in
// parity order: site (x, y, z, t) of parity p sits at s = p * V/2 + (x/2 + Lx/2 (y + Ly (z + Lz t))).
// The half kernel computes, for every site of output parity p,
//   out = [b -] ([self] + c * H in)           c = sign * kappa (kappa read from device memory)
// with `in` read on parity 1 - p. M = 1 - kappa^2 H_eo H_oe on the even sites is two launches:
// t_o = kappa H_oe x_e, then M x_e = x_e - kappa H_eo t_o.

struct EoArgsBase {
  Geom g;
  int parity;         // output parity
  double sign;        // c = sign * kappa
  const double* kappa_dev;
  const int* skip;
  double* partials;
  unsigned* ticket;
  double* result;
};

template <int SP, bool C12>
struct EoArgs {
  EoArgsBase e;
  GaugeRef<typename RealOf<SP>::type, C12> u;
  SpinorRef<SP> in, out, self, b;
};

// full coordinates of half index i of parity p
__device__ __forceinline__ void eo_coords(const Geom& g, int i, int p, int (&c)[4]) {
  const int lxh = g.L[0] >> 1;
  int r = i;
  const int xh = r % lxh;
  r /= lxh;
  c[1] = r % g.L[1];
  r /= g.L[1];
  c[2] = r % g.L[2];
  c[3] = r / g.L[2];
  c[0] = 2 * xh + ((c[1] + c[2] + c[3] + p) & 1);
}

__device__ __forceinline__ int eo_index(const Geom& g, const int (&c)[4]) {
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  return par * (g.V >> 1) + (c[0] >> 1) + (g.L[0] >> 1) * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}

template <int MU, int SF, int SP, bool C12, typename R>
__device__ __forceinline__ void eo_hop_pair(const EoArgs<SP, C12>& a, R k0, int s, const int (&c)[4],
                                            Cx<R> (&acc)[12]) {
  const int V = a.e.g.V;
  {
    int n[4] = {c[0], c[1], c[2], c[3]};
    const bool wrap = n[MU] == a.e.g.L[MU] - 1;
    n[MU] = wrap ? 0 : n[MU] + 1;
    const int nb = eo_index(a.e.g, n);
    Cx<R> psi[12], h[6], u[9], chi[6];
    const R k = load_hop_spinor(a.in, nb, V, psi, (wrap && a.e.g.bc[MU] < 0) ? -k0 : k0);
    spin_project<MU, SF>(psi, h);
    load_link(a.u, MU, s, V, u);
    su3_mul(u, h, chi);
    spin_reconstruct<MU, SF>(acc, chi, k);
  }
  {
    int n[4] = {c[0], c[1], c[2], c[3]};
    const bool wrap = n[MU] == 0;
    n[MU] = wrap ? a.e.g.L[MU] - 1 : n[MU] - 1;
    const int nb = eo_index(a.e.g, n);
    Cx<R> psi[12], h[6], u[9], chi[6];
    const R k = load_hop_spinor(a.in, nb, V, psi, (wrap && a.e.g.bc[MU] < 0) ? -k0 : k0);
    spin_project<MU, -SF>(psi, h);
    load_link(a.u, MU, nb, V, u);
    su3_dag_mul(u, h, chi);
    spin_reconstruct<MU, -SF>(acc, chi, k);
  }
}

template <int SF, int SP, bool C12, typename R>
__device__ __forceinline__ void eo_hops_rt(const EoArgs<SP, C12>& a, R k0, int s, const int (&c)[4],
                                           Cx<R> (&acc)[12]) {
  const int V = a.e.g.V;
#pragma unroll 1
  for (int hop = 0; hop < 8; ++hop) {
    const int mu = hop >> 1, dir = hop & 1;
    int n[4] = {c[0], c[1], c[2], c[3]};
    const int L = a.e.g.L[mu];
    const int cm = mu == 0 ? c[0] : (mu == 1 ? c[1] : (mu == 2 ? c[2] : c[3]));
    const bool wrap = dir == 0 ? cm == L - 1 : cm == 0;
    const int nm = dir == 0 ? (wrap ? 0 : cm + 1) : (wrap ? L - 1 : cm - 1);
    if (mu == 0) n[0] = nm; else if (mu == 1) n[1] = nm; else if (mu == 2) n[2] = nm; else n[3] = nm;
    const int nb = eo_index(a.e.g, n);
    const R k = (wrap && a.e.g.bc[mu] < 0) ? -k0 : k0;
    const int S = dir == 0 ? SF : -SF;
    Cx<R> psi[12], h[6], u[9], chi[6];
    load_spinor(a.in, nb, V, psi);
    spin_project_rt(mu, S, psi, h);
    load_link(a.u, mu, dir == 0 ? s : nb, V, u);
    if (dir == 0)
      su3_mul(u, h, chi);
    else
      su3_dag_mul(u, h, chi);
    spin_reconstruct_rt(mu, S, acc, chi, k);
  }
}

// Half-site i of the output parity: out = [b -] ([self] + c * H in); returns |out|^2.
template <int SP, bool C12, bool DAG, bool SELF, bool RESID>
__device__ __forceinline__ double eo_site(const EoArgs<SP, C12>& a, int i) {
  typedef typename RealOf<SP>::type R;
  const int Vh = a.e.g.V >> 1, V = a.e.g.V;
  const int p = a.e.parity;
  int c[4];
  eo_coords(a.e.g, i, p, c);
  const int s = p * Vh + i;
  const R k0 = (R)(a.e.sign * *a.e.kappa_dev);
  Cx<R> acc[12];
  if (SELF) {
    load_spinor(a.self, s, V, acc);
  } else {
#pragma unroll
    for (int j = 0; j < 12; ++j) acc[j] = cx<R>(0, 0);
  }
  constexpr int SF = DAG ? +1 : -1;
  if constexpr (SP == PDF) {
    eo_hops_rt<SF>(a, k0, s, c, acc);
  } else {
    eo_hop_pair<0, SF>(a, k0, s, c, acc);
    eo_hop_pair<1, SF>(a, k0, s, c, acc);
    eo_hop_pair<2, SF>(a, k0, s, c, acc);
    eo_hop_pair<3, SF>(a, k0, s, c, acc);
  }
  if (RESID) {
    Cx<R> bv[12];
    load_spinor(a.b, s, V, bv);
#pragma unroll
    for (int j = 0; j < 12; ++j) acc[j] = cx<R>(bv[j].re - acc[j].re, bv[j].im - acc[j].im);
  }
  store_spinor(a.out, s, V, acc);
  return norm2_site(acc);
}

template <int SP, bool C12, bool DAG, bool SELF, bool RESID, bool NORM>
__global__ void __launch_bounds__(kDslashMaxThreads, DslashMinBlocks<SP>::value)
    dslash_eo_kernel(const EoArgs<SP, C12> a) {
  if (a.e.skip != nullptr && *a.e.skip != 0) return;
  const int Vh = a.e.g.V >> 1;
  double n2 = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    const double v = eo_site<SP, C12, DAG, SELF, RESID>(a, i);
    if (NORM) n2 += v;
  }
  if (NORM) {
    double v[1] = {n2}, tot[1];
    if (grid_reduce<OpSum, 1>(v, a.e.partials, a.e.ticket, tot) && threadIdx.x == 0) *a.e.result = tot[0];
  }
}

template <int SP, bool C12, bool DAG, bool SELF, bool RESID>
static cudaError_t eo_launch_t(const EoCall& c, cudaStream_t st) {
  EoArgs<SP, C12> a;
  memcpy(&a.e.g, &c.g, sizeof(Geom));
  a.e.parity = c.parity;
  a.e.sign = c.sign;
  a.e.kappa_dev = c.kappa_dev;
  a.e.skip = c.skip;
  a.e.partials = c.red.partials;
  a.e.ticket = c.red.ticket;
  a.e.result = c.red.result;
  a.u.p = reinterpret_cast<decltype(a.u.p)>(c.u.p);
  a.in = make_ref<SP>(c.in, c.g.V);
  a.out = make_ref<SP>(c.out, c.g.V);
  a.self = make_ref<SP>(c.self, c.g.V);
  a.b = make_ref<SP>(c.b, c.g.V);
  if (c.red.result) {
    auto k = dslash_eo_kernel<SP, C12, DAG, SELF, RESID, true>;
    k<<<stride_grid(k, c.g.V / 2, c.block), c.block, 0, st>>>(a);
  } else {
    auto k = dslash_eo_kernel<SP, C12, DAG, SELF, RESID, false>;
    k<<<stride_grid(k, c.g.V / 2, c.block), c.block, 0, st>>>(a);
  }
  return cudaGetLastError();
}

template <int SP, bool C12, bool DAG>
static cudaError_t eo_launch_d(const EoCall& c, cudaStream_t st) {
  if (c.use_self) {
    return c.resid ? eo_launch_t<SP, C12, DAG, true, true>(c, st) : eo_launch_t<SP, C12, DAG, true, false>(c, st);
  }
  return c.resid ? eo_launch_t<SP, C12, DAG, false, true>(c, st) : eo_launch_t<SP, C12, DAG, false, false>(c, st);
}

template <int SP, bool C12>
static cudaError_t eo_launch_p(const EoCall& c, cudaStream_t st) {
  return c.dagger ? eo_launch_d<SP, C12, true>(c, st) : eo_launch_d<SP, C12, false>(c, st);
}

cudaError_t launch_dslash_eo(const EoCall& c, cudaStream_t st) {
  if (c.block <= 0 || c.block > kDslashMaxThreads || c.block % 32 || !c.kappa_dev) return cudaErrorInvalidValue;
  if (c.in.prec == SPDF) {
    if (c.u.prec != SPDF) return cudaErrorInvalidValue;
    return eo_launch_p<PDF, false>(c, st);
  }
  if (c.in.prec == SP64) {
    if (c.u.prec != SP64) return cudaErrorInvalidValue;
    return eo_launch_p<P64, false>(c, st);
  }
  if (c.u.prec != SP32) return cudaErrorInvalidValue;
  if (c.in.prec == SP32) return c.u.c12 ? eo_launch_p<P32, true>(c, st) : eo_launch_p<P32, false>(c, st);
  if (c.in.prec == SP16) return c.u.c12 ? eo_launch_p<P16, true>(c, st) : eo_launch_p<P16, false>(c, st);
  return cudaErrorInvalidValue;
}

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
  a.y.bar = c.bar;
  a.y.err = c.err;
  auto k = cg_eo_loop_kernel<SP, C12>;
  int grid = resident_blocks(reinterpret_cast<const void*>(k), c.block);
  const int need = grid_for(c.g.V / 2, c.block);
  if (need < grid) grid = need;
  if (grid > c.max_grid) grid = c.max_grid;
  void* args[] = {&a};
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
