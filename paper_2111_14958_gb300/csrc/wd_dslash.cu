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
    const R k = (wrap && a.g.bc[MU] < 0) ? -mk : mk;
    Cx<R> psi[12];
    load_spinor(a.in, nb, V, psi);
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
    const R k = (wrap && a.g.bc[MU] < 0) ? -mk : mk;
    Cx<R> psi[12];
    load_spinor(a.in, nb, V, psi);
    Cx<R> h[6];
    spin_project<MU, -S_FWD>(psi, h);
    Cx<R> u[9];
    load_link(a.u, MU, nb, V, u);
    Cx<R> chi[6];
    su3_dag_mul(u, h, chi);
    spin_reconstruct<MU, -S_FWD>(acc, chi, k);
  }
}

// Occupancy: the kernel is latency-bound at large volumes (memory-level parallelism comes from
// resident warps), so registers are capped for 3 blocks of 256 threads per SM in FP32/FP16
// (24 warps) and 2 in FP64 (whose FP64 pipe saturates with few warps).
constexpr int kDslashMaxThreads = 256;
template <int SP>
struct DslashMinBlocks {
  static constexpr int value = SP == P64 ? 2 : 3;
};

template <int SP, bool C12, bool DAG, int EPI, bool NORM>
__global__ void __launch_bounds__(kDslashMaxThreads, DslashMinBlocks<SP>::value)
    dslash_kernel(const DslashArgs<SP, C12> a) {
  typedef typename RealOf<SP>::type R;
  if (a.skip != nullptr && *a.skip != 0) return;  // uniform over the grid
  const int V = a.g.V;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double n2 = 0.0;
  if (s < V) {
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
    hop_pair<0, SF>(a, mk, s, c, acc);
    hop_pair<1, SF>(a, mk, s, c, acc);
    hop_pair<2, SF>(a, mk, s, c, acc);
    hop_pair<3, SF>(a, mk, s, c, acc);
    if (EPI == EPI_RESID) {
      Cx<R> bv[12];
      load_spinor(a.b, s, V, bv);
#pragma unroll
      for (int i = 0; i < 12; ++i) acc[i] = cx<R>(bv[i].re - acc[i].re, bv[i].im - acc[i].im);
    }
    store_spinor(a.out, s, V, acc);
    if (NORM) n2 = norm2_site(acc);
  }
  if (NORM) {
    double v[1] = {n2}, tot[1];
    if (grid_reduce<OpSum, 1>(v, a.partials, a.ticket, tot) && threadIdx.x == 0) *a.result = tot[0];
  }
}

template <int SP, bool C12, bool DAG, int EPI>
static cudaError_t launch_t(const DslashCall& c, cudaStream_t st) {
  DslashArgs<SP, C12> a;
  static_assert(sizeof(GeomH) == sizeof(Geom), "geometry mirror");
  memcpy(&a.g, &c.g, sizeof(Geom));
  a.u.p = reinterpret_cast<decltype(a.u.p)>(c.u.p);
  a.in.p = reinterpret_cast<decltype(a.in.p)>(c.in.p);
  a.out.p = reinterpret_cast<decltype(a.out.p)>(c.out.p);
  a.b.p = reinterpret_cast<decltype(a.b.p)>(c.b.p);
  if constexpr (SP == P16) {
    a.in.norm = c.in.norm;
    a.out.norm = c.out.norm;
    a.b.norm = c.b.norm;
  }
  a.mkappa = (typename RealOf<SP>::type)(-c.kappa);
  a.kappa_dev = c.kappa_dev;
  a.skip = c.skip;
  a.partials = c.red.partials;
  a.ticket = c.red.ticket;
  a.result = c.red.result;
  const int grid = grid_for(c.g.V, c.block);
  if (c.red.result)
    dslash_kernel<SP, C12, DAG, EPI, true><<<grid, c.block, 0, st>>>(a);
  else
    dslash_kernel<SP, C12, DAG, EPI, false><<<grid, c.block, 0, st>>>(a);
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
