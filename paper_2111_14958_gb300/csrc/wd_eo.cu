// The even-odd half-lattice hopping kernel and its launcher (see wd_stencil.cuh for the site
// body and the parity-ordered layout).
#include "wd_stencil.cuh"

namespace wdk {

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
    const int grid = stride_grid(k, c.g.V / 2, c.block);
    if (!red_fits(c.red, grid)) return cudaErrorInvalidValue;
    k<<<grid, c.block, 0, st>>>(a);
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

}  // namespace wdk
