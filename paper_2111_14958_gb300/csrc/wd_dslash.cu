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
#include "wd_stencil.cuh"

namespace wdk {

template <int SP, bool C12, bool DAG, int EPI, bool NORM>
__global__ void __launch_bounds__(kDslashMaxThreads, DslashKernelMinBlocks<SP>::value)
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

// FP32 / FP16 under another load schedule (two blocks per SM, up to 128 registers):
//   MODE 2: thread t of the grid takes sites s0 and s0 + stride of each grid-stride step (every load
//           coalesced), hop by hop with both sites' loads issued first (dslash_sites);
//   MODE 3: one site per grid-stride step, both hops of each direction loaded before their
//           arithmetic (dslash_site_loaded).
template <int SP, bool C12, bool DAG, int EPI, bool NORM, int MODE>
__global__ void __launch_bounds__(kDslashMaxThreads, 2) dslash_sched_kernel(const DslashArgs<SP, C12> a) {
  if (a.skip != nullptr && *a.skip != 0) return;  // uniform over the grid
  const int V = a.g.V;
  const int stride = gridDim.x * blockDim.x;
  double n2 = 0.0;
  if constexpr (MODE == 2) {
    for (int s0 = blockIdx.x * blockDim.x + threadIdx.x; s0 < V; s0 += 2 * stride) {
      const int s1 = s0 + stride;
      const int sv[2] = {s0, s1 < V ? s1 : s0};  // a site past the end repeats s0 and is not stored
      const bool live[2] = {true, s1 < V};
      const double v = dslash_sites<SP, C12, DAG, EPI, 2>(a, sv, live);
      if (NORM) n2 += v;
    }
  } else {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += stride) {
      const double v = dslash_site_loaded<SP, C12, DAG, EPI>(a, s);
      if (NORM) n2 += v;
    }
  }
  if (NORM) {
    double v[1] = {n2}, tot[1];
    if (grid_reduce<OpSum, 1>(v, a.partials, a.ticket, tot) && threadIdx.x == 0) *a.result = tot[0];
  }
}

template <int SP, bool C12, bool DAG, int EPI, int MODE>
static cudaError_t launch_sched(const DslashCall& c, const DslashArgs<SP, C12>& a, cudaStream_t st) {
  const int units = MODE == 2 ? (c.g.V + 1) / 2 : c.g.V;
  if (c.red.result) {
    auto k = dslash_sched_kernel<SP, C12, DAG, EPI, true, MODE>;
    const int grid = stride_grid(k, units, c.block);
    if (!red_fits(c.red, grid)) return cudaErrorInvalidValue;
    k<<<grid, c.block, 0, st>>>(a);
  } else {
    auto k = dslash_sched_kernel<SP, C12, DAG, EPI, false, MODE>;
    k<<<stride_grid(k, units, c.block), c.block, 0, st>>>(a);
  }
  return cudaGetLastError();
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

template <int L, bool DAG, int EPI, bool NORM>
__global__ void __launch_bounds__(kDslashMaxThreads) dslash_lanes_kernel(const DslashArgs<P64, false> a) {
  if (a.skip != nullptr && *a.skip != 0) return;  // uniform over the grid
  const double n2 = lanes_sites<L, DAG, EPI>(a);
  if (NORM) {
    double v[1] = {n2}, tot[1];
    if (grid_reduce<OpSum, 1>(v, a.partials, a.ticket, tot) && threadIdx.x == 0) *a.result = tot[0];
  }
}

template <int L, bool DAG, int EPI>
static cudaError_t launch_lanes(const DslashArgs<P64, false>& a, const DslashCall& c, cudaStream_t st) {
  if (c.red.result) {
    auto k = dslash_lanes_kernel<L, DAG, EPI, true>;
    const int grid = stride_grid(k, L * c.g.V, c.block);
    if (!red_fits(c.red, grid)) return cudaErrorInvalidValue;
    k<<<grid, c.block, 0, st>>>(a);
  } else {
    auto k = dslash_lanes_kernel<L, DAG, EPI, false>;
    k<<<stride_grid(k, L * c.g.V, c.block), c.block, 0, st>>>(a);
  }
  return cudaSuccess;
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
    if (c.variant >= 2) {  // 4, 8 or 16 lanes per site
      cudaError_t e;
      if (c.variant == 2) e = launch_lanes<4, DAG, EPI>(a, c, st);
      else if (c.variant == 3) e = launch_lanes<8, DAG, EPI>(a, c, st);
      else e = launch_lanes<16, DAG, EPI>(a, c, st);
      if (e != cudaSuccess) return e;
      return cudaGetLastError();
    }
    if (c.variant == 1) {  // two lanes per site
      if (c.red.result) {
        auto k = dslash_pair_kernel<C12, DAG, EPI, true>;
        const int grid = stride_grid(k, 2 * c.g.V, c.block);
        if (!red_fits(c.red, grid)) return cudaErrorInvalidValue;
        k<<<grid, c.block, 0, st>>>(a);
      } else {
        auto k = dslash_pair_kernel<C12, DAG, EPI, false>;
        k<<<stride_grid(k, 2 * c.g.V, c.block), c.block, 0, st>>>(a);
      }
      return cudaGetLastError();
    }
  }
  if constexpr (SP == P32 || SP == P16) {
    if (c.schedule == 2) return launch_sched<SP, C12, DAG, EPI, 2>(c, a, st);
    if (c.schedule == 3) return launch_sched<SP, C12, DAG, EPI, 3>(c, a, st);
  }
  if (c.red.result) {
    auto k = dslash_kernel<SP, C12, DAG, EPI, true>;
    const int grid = stride_grid(k, c.g.V, c.block);
    if (!red_fits(c.red, grid)) return cudaErrorInvalidValue;
    k<<<grid, c.block, 0, st>>>(a);
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
  if (c.tma) {
    if (!c.err) return cudaErrorInvalidValue;
    return launch_dslash_tma(c, c.tma - 1, c.err, st);
  }
  if (c.block <= 0 || c.block > kDslashMaxThreads || c.block % 32) return cudaErrorInvalidValue;
  if (c.variant != 0 && (c.variant < 0 || c.variant > kMaxDslashVariant || c.in.prec != SP64))
    return cudaErrorInvalidValue;
  if (c.schedule < 0 || c.schedule > 3 || (c.schedule >= 2 && c.in.prec != SP32 && c.in.prec != SP16))
    return cudaErrorInvalidValue;
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

}  // namespace wdk
