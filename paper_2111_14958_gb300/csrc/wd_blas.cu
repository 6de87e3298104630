// Layout conversion, gauge loading and the fused BLAS-1 steps of CG (Sec. 2: dot products and
// vector additions), with deterministic FP64 grid reductions.
#include <cstring>

#include "wd_device.cuh"
#include "wd_internal.h"

namespace wdk {

// ---------------------------------------------------------------- packing

template <int SP>
struct Work {
  typedef float R;
};
template <>
struct Work<P64> {
  typedef double R;
};

// Canonical (lexicographic) site n -> storage site: n itself, or its parity-ordered index when the
// context stores fields even-odd (L = extents; all even).
struct SiteMap {
  int eo;
  int L[4];
  int V;
};

__device__ __forceinline__ int map_site(const SiteMap& m, int n) {
  if (!m.eo) return n;
  int r = n;
  const int x = r % m.L[0];
  r /= m.L[0];
  const int y = r % m.L[1];
  r /= m.L[1];
  const int z = r % m.L[2];
  const int t = r / m.L[2];
  const int par = (x + y + z + t) & 1;
  return par * (m.V >> 1) + (x >> 1) + (m.L[0] >> 1) * (y + m.L[1] * (z + m.L[2] * t));
}

template <int SP, bool NORM>
__global__ void pack_kernel(const double2* __restrict__ canon, SpinorRef<SP> out, int V, SiteMap m, double* partials,
                            unsigned* ticket, double* result) {
  typedef typename Work<SP>::R R;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double n2 = 0.0;
  if (s < V) {
    Cx<R> v[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const double2 d = canon[(size_t)s * 12 + c];
      n2 = fma(d.x, d.x, n2);
      n2 = fma(d.y, d.y, n2);
      v[c] = cx<R>((R)d.x, (R)d.y);
    }
    store_spinor(out, map_site(m, s), V, v);
  }
  if (NORM) {
    double a[1] = {n2}, tot[1];
    if (grid_reduce<OpSum, 1>(a, partials, ticket, tot) && threadIdx.x == 0) *result = tot[0];
  }
}

__global__ void pack_c64_kernel(const float2* __restrict__ canon, SpinorRef<P32> out, int V, SiteMap m) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  Cx<float> v[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const float2 d = canon[(size_t)s * 12 + c];
    v[c] = cx(d.x, d.y);
  }
  store_spinor(out, map_site(m, s), V, v);
}

template <int SP>
__global__ void unpack_kernel(SpinorRef<SP> in, double2* __restrict__ canon, int V, SiteMap m) {
  typedef typename Work<SP>::R R;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  Cx<R> v[12];
  load_spinor(in, map_site(m, s), V, v);
#pragma unroll
  for (int c = 0; c < 12; ++c) canon[(size_t)s * 12 + c] = make_double2((double)v[c].re, (double)v[c].im);
}

__global__ void unpack_c64_kernel(SpinorRef<P32> in, float2* __restrict__ canon, int V, SiteMap m) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  Cx<float> v[12];
  load_spinor(in, map_site(m, s), V, v);
#pragma unroll
  for (int c = 0; c < 12; ++c) canon[(size_t)s * 12 + c] = make_float2(v[c].re, v[c].im);
}

template <int SP>
static SpinorRef<SP> view(FieldPtr f);

template <>
SpinorRef<P64> view<P64>(FieldPtr f) {
  SpinorRef<P64> r;
  r.p = reinterpret_cast<double2*>(f.p);
  return r;
}
template <>
SpinorRef<P32> view<P32>(FieldPtr f) {
  SpinorRef<P32> r;
  r.p = reinterpret_cast<float4*>(f.p);
  return r;
}
template <>
SpinorRef<P16> view<P16>(FieldPtr f) {
  SpinorRef<P16> r;
  r.p = reinterpret_cast<uint4*>(f.p);
  r.norm = f.norm;
  return r;
}

// double-float fields need the stride V to find the lo half
static SpinorRef<PDF> view_df(FieldPtr f, int V) {
  SpinorRef<PDF> r;
  r.hi = reinterpret_cast<float4*>(f.p);
  r.lo = reinterpret_cast<float4*>(f.p) + (size_t)6 * V;
  return r;
}

static SiteMap site_map(const GeomH* eo) {
  SiteMap m;
  m.eo = eo != nullptr;
  for (int i = 0; i < 4; ++i) m.L[i] = eo ? eo->L[i] : 0;
  m.V = eo ? eo->V : 0;
  return m;
}

template <int SP>
static cudaError_t pack_t(const double* canon, FieldPtr out, int V, const GeomH* eo, Red red, int block,
                          cudaStream_t st) {
  const int grid = grid_for(V, block);
  if (!red_fits(red, grid)) return cudaErrorInvalidValue;
  const double2* c2 = reinterpret_cast<const double2*>(canon);
  const SiteMap m = site_map(eo);
  if (red.result)
    pack_kernel<SP, true><<<grid, block, 0, st>>>(c2, view<SP>(out), V, m, red.partials, red.ticket, red.result);
  else
    pack_kernel<SP, false><<<grid, block, 0, st>>>(c2, view<SP>(out), V, m, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_pack(const double* canon, FieldPtr out, int V, const GeomH* eo, Red red, int block,
                        cudaStream_t st) {
  switch (out.prec) {
    case SP64: return pack_t<P64>(canon, out, V, eo, red, block, st);
    case SP32: return pack_t<P32>(canon, out, V, eo, red, block, st);
    case SP16: return pack_t<P16>(canon, out, V, eo, red, block, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_pack_c64(const float* canon, FieldPtr out, int V, const GeomH* eo, int block, cudaStream_t st) {
  if (out.prec != SP32) return cudaErrorInvalidValue;
  pack_c64_kernel<<<grid_for(V, block), block, 0, st>>>(reinterpret_cast<const float2*>(canon), view<P32>(out), V,
                                                        site_map(eo));
  return cudaGetLastError();
}

cudaError_t launch_unpack(FieldPtr in, double* canon, int V, const GeomH* eo, int block, cudaStream_t st) {
  double2* c2 = reinterpret_cast<double2*>(canon);
  const int grid = grid_for(V, block);
  const SiteMap m = site_map(eo);
  switch (in.prec) {
    case SP64: unpack_kernel<P64><<<grid, block, 0, st>>>(view<P64>(in), c2, V, m); break;
    case SP32: unpack_kernel<P32><<<grid, block, 0, st>>>(view<P32>(in), c2, V, m); break;
    case SP16: unpack_kernel<P16><<<grid, block, 0, st>>>(view<P16>(in), c2, V, m); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_unpack_c64(FieldPtr in, float* canon, int V, const GeomH* eo, int block, cudaStream_t st) {
  if (in.prec != SP32) return cudaErrorInvalidValue;
  unpack_c64_kernel<<<grid_for(V, block), block, 0, st>>>(view<P32>(in), reinterpret_cast<float2*>(canon), V,
                                                          site_map(eo));
  return cudaGetLastError();
}

// ---------------------------------------------------------------- gauge load

// One thread per (site, mu). Stores the link in the device layout and measures its distance
// from SU(3): max(|U^dag U - 1|_max, |det U - 1|).
template <int GP, bool C12, bool CHECK>
__global__ void gauge_load_kernel(const double2* __restrict__ canon, void* out, int V, SiteMap m, double* partials,
                                  unsigned* ticket, double* result) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // i = 4 * n + mu, n canonical
  double dev = 0.0;
  if (i < 4 * V) {
    const int s = map_site(m, i >> 2), mu = i & 3;
    Cx<double> u[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double2 d = canon[(size_t)i * 9 + k];
      u[k] = cx(d.x, d.y);
    }
    if (CHECK) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          double re = 0, im = 0;  // (U^dag U)_ab = sum_c conj(U_ca) U_cb
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const Cx<double> x = u[3 * c + a], y = u[3 * c + b];
            re += x.re * y.re + x.im * y.im;
            im += x.re * y.im - x.im * y.re;
          }
          if (a == b) re -= 1.0;
          dev = fmax(dev, fmax(fabs(re), fabs(im)));
        }
      }
      // det by cofactors of row 0
      const Cx<double> m0 = cmul(u[4], u[8]), m1 = cmul(u[5], u[7]);
      const Cx<double> m2 = cmul(u[3], u[8]), m3 = cmul(u[5], u[6]);
      const Cx<double> m4 = cmul(u[3], u[7]), m5 = cmul(u[4], u[6]);
      const Cx<double> c0 = cx(m0.re - m1.re, m0.im - m1.im);
      const Cx<double> c1 = cx(m2.re - m3.re, m2.im - m3.im);
      const Cx<double> c2 = cx(m4.re - m5.re, m4.im - m5.im);
      const Cx<double> t0 = cmul(u[0], c0), t1 = cmul(u[1], c1), t2 = cmul(u[2], c2);
      const double dre = t0.re - t1.re + t2.re - 1.0, dim = t0.im - t1.im + t2.im;
      dev = fmax(dev, sqrt(dre * dre + dim * dim));
      if (!(dev == dev)) dev = 1e300;  // NaN links fail the check
    }
    if (GP == P64) {
      double2* o = reinterpret_cast<double2*>(out) + (size_t)mu * 9 * V + s;
#pragma unroll
      for (int k = 0; k < 9; ++k) o[(size_t)k * V] = make_double2(u[k].re, u[k].im);
    } else if (GP == PDF) {
      float2* hi = reinterpret_cast<float2*>(out) + (size_t)mu * 9 * V + s;
      float2* lo = hi + (size_t)36 * V;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float hr = __double2float_rn(u[k].re), hm = __double2float_rn(u[k].im);
        hi[(size_t)k * V] = make_float2(hr, hm);
        lo[(size_t)k * V] = make_float2(__double2float_rn(u[k].re - (double)hr), __double2float_rn(u[k].im - (double)hm));
      }
    } else if (!C12) {
      float2* o = reinterpret_cast<float2*>(out) + (size_t)mu * 9 * V + s;
#pragma unroll
      for (int k = 0; k < 9; ++k) o[(size_t)k * V] = make_float2((float)u[k].re, (float)u[k].im);
    } else {
      float4* o = reinterpret_cast<float4*>(out) + (size_t)mu * 3 * V + s;
#pragma unroll
      for (int j = 0; j < 3; ++j)
        o[(size_t)j * V] = make_float4((float)u[2 * j].re, (float)u[2 * j].im, (float)u[2 * j + 1].re,
                                       (float)u[2 * j + 1].im);
    }
  }
  if (CHECK) {
    double a[1] = {dev}, tot[1];
    if (grid_reduce<OpMax, 1>(a, partials, ticket, tot) && threadIdx.x == 0) *result = tot[0];
  }
}

cudaError_t launch_gauge_load(const double* canon, GaugePtr out, int V, const GeomH* eo, Red red, int block,
                              cudaStream_t st) {
  const int grid = grid_for(4 * V, block);
  if (!red_fits(red, grid)) return cudaErrorInvalidValue;
  const SiteMap m = site_map(eo);
  const double2* c2 = reinterpret_cast<const double2*>(canon);
  void* o = const_cast<void*>(out.p);
  const bool chk = red.result != nullptr;
#define WD_GL(GP, C12)                                                                                        \
  do {                                                                                                        \
    if (chk)                                                                                                  \
      gauge_load_kernel<GP, C12, true><<<grid, block, 0, st>>>(c2, o, V, m, red.partials, red.ticket, red.result); \
    else                                                                                                      \
      gauge_load_kernel<GP, C12, false><<<grid, block, 0, st>>>(c2, o, V, m, nullptr, nullptr, nullptr);         \
  } while (0)
  if (out.prec == SP64)
    WD_GL(P64, false);
  else if (out.prec == SPDF)
    WD_GL(PDF, false);
  else if (out.c12)
    WD_GL(P32, true);
  else
    WD_GL(P32, false);
#undef WD_GL
  return cudaGetLastError();
}

// ---------------------------------------------------------------- CG scalar steps

__global__ void cg_init_kernel(CgScalars* sc, int reset_iter) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc->status = ST_RUNNING;
    if (reset_iter) {
      sc->iter = 0;
      sc->updates = 0;
    }
    sc->need_update = 0;
    sc->no_update = 1;
  }
}

// After r = eta - D x and p = D^dag r (or p = r): decide whether the loop has work to do.
__global__ void cg_check_kernel(CgScalars* sc, int use_cond, cudaGraphConditionalHandle cond, int gamma_from_rr) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int st = ST_RUNNING;
    if (gamma_from_rr) sc->gamma = sc->rr;
    const double eta2 = sc->eta2, rr = sc->rr, g = sc->gamma;
    if (!isfinite(eta2) || !isfinite(rr) || !isfinite(g))
      st = ST_BREAKDOWN;
    else if (rr <= sc->tol2 * eta2)
      st = ST_CONVERGED;
    else if (sc->iter >= sc->maxit)
      st = ST_MAXIT;
    else if (!(g > 0.0))
      st = ST_BREAKDOWN;
    sc->status = st;
    sc->rr_ref = rr;
    if (use_cond) cudaGraphSetConditional(cond, st == ST_RUNNING ? 1u : 0u);
  }
}

// alpha = gamma / ||q||^2; r -= alpha q; ||r||^2. Converged or breakdown is decided here.
template <int SP>
__global__ void cg_update_r_kernel(SpinorRef<SP> r, SpinorRef<SP> q, int n, int V, CgScalars* sc, double* partials,
                                   int gamma_from_rr) {
  typedef typename Work<SP>::R R;
  if (sc->status != ST_RUNNING) return;  // uniform
  const double qq = sc->qq, gamma = sc->gamma;
  const bool ok = qq > 0.0 && isfinite(qq) && isfinite(gamma);
  const double alpha = ok ? gamma / qq : 0.0;
  const R a = (R)alpha;
  double n2 = 0.0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; ok && s < n; s += gridDim.x * blockDim.x) {
    Cx<R> rv[12], qv[12];
    load_spinor(r, s, V, rv);
    load_spinor(q, s, V, qv);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      rv[c].re = fma(-a, qv[c].re, rv[c].re);
      rv[c].im = fma(-a, qv[c].im, rv[c].im);
    }
    store_spinor(r, s, V, rv);
    n2 += norm2_site(rv);
  }
  double v[1] = {n2}, tot[1];
  if (grid_reduce<OpSum, 1>(v, partials, &sc->ticket[TK_UPD_R], tot) && threadIdx.x == 0) {
    sc->alpha = alpha;
    sc->rr = tot[0];
    record_residual(sc, sc->iter, tot[0]);
    if (gamma_from_rr) sc->gamma_new = tot[0];
    if (!ok || !isfinite(tot[0]))
      sc->status = ST_BREAKDOWN;
    else if (tot[0] <= sc->tol2 * sc->eta2)
      sc->status = ST_CONVERGED;
  }
}

// x += alpha d; p = s + beta p (beta = gamma_new / gamma; d is p itself in the CGLS arrangement).
// The last block advances the iteration, applies the iteration limit and sets the loop condition.
// Every block always takes a ticket, so the condition is set on every pass: the loop cannot run
// on without an update.
template <int SP>
__global__ void cg_update_xp_kernel(SpinorRef<SP> x, SpinorRef<SP> d, SpinorRef<SP> p, SpinorRef<SP> sv, int n, int V,
                                    CgScalars* sc, double* partials, int use_cond, cudaGraphConditionalHandle cond) {
  typedef typename Work<SP>::R R;
  const int st0 = sc->status;  // uniform: only this kernel's last block changes it below
  const double alpha = sc->alpha;
  const double gnew = sc->gamma_new, gold = sc->gamma;
  const bool do_x = (st0 == ST_RUNNING || st0 == ST_CONVERGED);
  const bool do_p = st0 == ST_RUNNING && isfinite(gnew) && gold > 0.0;
  const double beta = do_p ? gnew / gold : 0.0;
  const R a = (R)alpha, b = (R)beta;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; do_x && s < n; s += gridDim.x * blockDim.x) {
    Cx<R> xv[12], pv[12];
    load_spinor(x, s, V, xv);
    if (d.p != p.p) {  // uniform
      Cx<R> dv[12];
      load_spinor(d, s, V, dv);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        xv[c].re = fma(a, dv[c].re, xv[c].re);
        xv[c].im = fma(a, dv[c].im, xv[c].im);
      }
      if (do_p) load_spinor(p, s, V, pv);
    } else {
      load_spinor(p, s, V, pv);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        xv[c].re = fma(a, pv[c].re, xv[c].re);
        xv[c].im = fma(a, pv[c].im, xv[c].im);
      }
    }
    store_spinor(x, s, V, xv);
    if (do_p) {
      Cx<R> svv[12];
      load_spinor(sv, s, V, svv);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        pv[c].re = fma(b, pv[c].re, svv[c].re);
        pv[c].im = fma(b, pv[c].im, svv[c].im);
      }
      store_spinor(p, s, V, pv);
    }
  }
  double v[1] = {0.0}, tot[1];
  if (grid_reduce<OpSum, 1>(v, partials, &sc->ticket[TK_UPD_XP], tot) && threadIdx.x == 0) {
    int st = st0;
    if (do_x) sc->iter += 1;
    if (st == ST_RUNNING) {
      if (!do_p) {
        st = ST_BREAKDOWN;
      } else {
        sc->beta = beta;
        sc->gamma = gnew;
        if (sc->iter >= sc->maxit) st = ST_MAXIT;
      }
    }
    sc->status = st;
    if (use_cond) cudaGraphSetConditional(cond, st == ST_RUNNING ? 1u : 0u);
  }
}

cudaError_t launch_cg_init(CgScalars* sc, int reset_iter, cudaStream_t st) {
  cg_init_kernel<<<1, 32, 0, st>>>(sc, reset_iter);
  return cudaGetLastError();
}

cudaError_t launch_cg_check(CgScalars* sc, int use_cond, unsigned long long cond, cudaStream_t st,
                            int gamma_from_rr) {
  cg_check_kernel<<<1, 32, 0, st>>>(sc, use_cond, (cudaGraphConditionalHandle)cond, gamma_from_rr);
  return cudaGetLastError();
}

#define WD_STRIDE(K) K<<<stride_grid(K, n, block), block, 0, st>>>

cudaError_t launch_cg_update_r(int prec, FieldPtr r, FieldPtr q, int n, int V, CgScalars* sc, double* partials,
                               int block, cudaStream_t st, int gamma_from_rr) {
  const int g = gamma_from_rr;
  switch (prec) {
    case SP64: WD_STRIDE(cg_update_r_kernel<P64>)(view<P64>(r), view<P64>(q), n, V, sc, partials, g); break;
    case SP32: WD_STRIDE(cg_update_r_kernel<P32>)(view<P32>(r), view<P32>(q), n, V, sc, partials, g); break;
    case SP16: WD_STRIDE(cg_update_r_kernel<P16>)(view<P16>(r), view<P16>(q), n, V, sc, partials, g); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_cg_update_xp(int prec, FieldPtr x, FieldPtr d, FieldPtr p, FieldPtr s, int n, int V,
                                CgScalars* sc, double* partials, int use_cond, unsigned long long cond, int block,
                                cudaStream_t st) {
  const cudaGraphConditionalHandle h = (cudaGraphConditionalHandle)cond;
  switch (prec) {
    case SP64:
      WD_STRIDE(cg_update_xp_kernel<P64>)(view<P64>(x), view<P64>(d), view<P64>(p), view<P64>(s), n, V, sc, partials,
                                          use_cond, h);
      break;
    case SP32:
      WD_STRIDE(cg_update_xp_kernel<P32>)(view<P32>(x), view<P32>(d), view<P32>(p), view<P32>(s), n, V, sc, partials,
                                          use_cond, h);
      break;
    case SP16:
      WD_STRIDE(cg_update_xp_kernel<P16>)(view<P16>(x), view<P16>(d), view<P16>(p), view<P16>(s), n, V, sc, partials,
                                          use_cond, h);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- mixed precision (reliable updates)
//
// Inner CG in a low storage precision (W = FP32 or FP16 spinors) accumulates the solution
// increment x_lo (FP32) since the last reliable update. When the recursive ||r|| has dropped by
// the factor delta since that update, or reached the tolerance, the increment is folded into the
// FP64 solution and the residual is recomputed in FP64 from it.

// alpha = gamma / ||q||^2; r_lo -= alpha q; x_lo += alpha p; ||r_lo||^2; decide on an update.
template <int SPW>
__global__ void mp_update_rx_kernel(SpinorRef<SPW> r, SpinorRef<SPW> q, SpinorRef<SPW> p, SpinorRef<P32> xlo,
                                    int n, int V, CgScalars* sc, double* partials, int use_cond,
                                    cudaGraphConditionalHandle upd) {
  typedef float R;
  const int st0 = sc->status;
  const double qq = sc->qq, gamma = sc->gamma;
  const bool ok = st0 == ST_RUNNING && qq > 0.0 && isfinite(qq) && isfinite(gamma);
  const double alpha = ok ? gamma / qq : 0.0;
  const R a = (R)alpha;
  double n2 = 0.0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; ok && s < n; s += gridDim.x * blockDim.x) {
    Cx<R> rv[12], qv[12], pv[12], xv[12];
    load_spinor(r, s, V, rv);
    load_spinor(q, s, V, qv);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      rv[c].re = fma(-a, qv[c].re, rv[c].re);
      rv[c].im = fma(-a, qv[c].im, rv[c].im);
    }
    store_spinor(r, s, V, rv);
    n2 += norm2_site(rv);
    load_spinor(p, s, V, pv);
    load_spinor(xlo, s, V, xv);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      xv[c].re = fma(a, pv[c].re, xv[c].re);
      xv[c].im = fma(a, pv[c].im, xv[c].im);
    }
    store_spinor(xlo, s, V, xv);
  }
  double v[1] = {n2}, tot[1];
  if (grid_reduce<OpSum, 1>(v, partials, &sc->ticket[TK_UPD_R], tot) && threadIdx.x == 0) {
    int need = 0;
    if (st0 == ST_RUNNING) {
      if (!ok || !isfinite(tot[0])) {
        sc->status = ST_BREAKDOWN;
      } else {
        sc->alpha = alpha;
        sc->rr = tot[0];
        record_residual(sc, sc->iter, tot[0]);
        need = (tot[0] <= sc->delta2 * sc->rr_ref) || (tot[0] <= sc->tol2 * sc->eta2);
      }
    }
    sc->need_update = need;
    sc->no_update = !need;
    if (use_cond) cudaGraphSetConditional(upd, need ? 1u : 0u);
  }
}

// x_hi += x_lo; x_lo = 0
__global__ void mp_accumulate_kernel(SpinorRef<P64> xhi, SpinorRef<P32> xlo, int n, int V, const int* skip) {
  if (skip != nullptr && *skip == 0) return;  // runs only when an update is pending
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  Cx<double> xh[12];
  Cx<float> xl[12];
  load_spinor(xhi, s, V, xh);
  load_spinor(xlo, s, V, xl);
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    xh[c].re += (double)xl[c].re;
    xh[c].im += (double)xl[c].im;
    xl[c] = cx(0.f, 0.f);
  }
  store_spinor(xhi, s, V, xh);
  store_spinor(xlo, s, V, xl);
}

// r_lo = r_hi (FP64 -> W). The last block adopts ||r_hi||^2 as the new reference and decides
// convergence on this FP64 residual. count = 0 for the initial conversion.
template <int SPW>
__global__ void mp_convert_kernel(SpinorRef<P64> rhi, SpinorRef<SPW> rlo, int n, int V, CgScalars* sc, double* partials,
                                  int count, const int* skip) {
  if (skip != nullptr && *skip == 0) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) {
    Cx<double> h[12];
    Cx<float> l[12];
    load_spinor(rhi, s, V, h);
#pragma unroll
    for (int c = 0; c < 12; ++c) l[c] = cx((float)h[c].re, (float)h[c].im);
    store_spinor(rlo, s, V, l);
  }
  double v[1] = {0.0}, tot[1];
  if (grid_reduce<OpSum, 1>(v, partials, &sc->ticket[TK_UPD_REL], tot) && threadIdx.x == 0) {
    const double rr = sc->rr_true;
    sc->rr = rr;
    sc->rr_ref = rr;
    sc->need_update = 0;
    sc->no_update = 1;
    if (count) sc->updates += 1;
    if (!isfinite(rr))
      sc->status = ST_BREAKDOWN;
    else if (rr <= sc->tol2 * sc->eta2)
      sc->status = ST_CONVERGED;
  }
}

// p = s + beta p. The last block advances the iteration and sets the loop condition.
template <int SPW>
__global__ void mp_update_p_kernel(SpinorRef<SPW> p, SpinorRef<SPW> sv, int n, int V, CgScalars* sc, double* partials,
                                   int use_cond, cudaGraphConditionalHandle cond) {
  typedef float R;
  const int st0 = sc->status;
  const double gnew = sc->gamma_new, gold = sc->gamma;
  const bool do_p = st0 == ST_RUNNING && isfinite(gnew) && gold > 0.0;
  const double beta = do_p ? gnew / gold : 0.0;
  const R b = (R)beta;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; do_p && s < n; s += gridDim.x * blockDim.x) {
    Cx<R> pv[12], svv[12];
    load_spinor(p, s, V, pv);
    load_spinor(sv, s, V, svv);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      pv[c].re = fma(b, pv[c].re, svv[c].re);
      pv[c].im = fma(b, pv[c].im, svv[c].im);
    }
    store_spinor(p, s, V, pv);
  }
  double v[1] = {0.0}, tot[1];
  if (grid_reduce<OpSum, 1>(v, partials, &sc->ticket[TK_UPD_XP], tot) && threadIdx.x == 0) {
    int st = st0;
    // an iteration that ran its r update counts, including one that converged in its update
    if (st0 == ST_RUNNING || st0 == ST_CONVERGED) sc->iter += 1;
    if (st == ST_RUNNING) {
      if (!do_p) {
        st = ST_BREAKDOWN;
      } else {
        sc->beta = beta;
        sc->gamma = gnew;
        if (sc->iter >= sc->maxit) st = ST_MAXIT;
      }
    }
    sc->status = st;
    if (use_cond) cudaGraphSetConditional(cond, st == ST_RUNNING ? 1u : 0u);
  }
}

__global__ void zero_kernel(float4* p, size_t n4) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n4) p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

cudaError_t launch_mp_update_rx(int precw, FieldPtr r, FieldPtr q, FieldPtr p, FieldPtr xlo, int n, int V,
                                CgScalars* sc, double* partials, int use_cond, unsigned long long upd, int block,
                                cudaStream_t st) {
  const cudaGraphConditionalHandle h = (cudaGraphConditionalHandle)upd;
  if (xlo.prec != SP32) return cudaErrorInvalidValue;
  switch (precw) {
    case SP32:
      WD_STRIDE(mp_update_rx_kernel<P32>)(view<P32>(r), view<P32>(q), view<P32>(p), view<P32>(xlo), n, V, sc, partials,
                                          use_cond, h);
      break;
    case SP16:
      WD_STRIDE(mp_update_rx_kernel<P16>)(view<P16>(r), view<P16>(q), view<P16>(p), view<P32>(xlo), n, V, sc, partials,
                                          use_cond, h);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_mp_accumulate(FieldPtr xhi, FieldPtr xlo, int n, int V, const int* skip, int block,
                                 cudaStream_t st) {
  if (xhi.prec != SP64 || xlo.prec != SP32) return cudaErrorInvalidValue;
  mp_accumulate_kernel<<<grid_for(n, block), block, 0, st>>>(view<P64>(xhi), view<P32>(xlo), n, V, skip);
  return cudaGetLastError();
}

cudaError_t launch_mp_convert(FieldPtr rhi, FieldPtr rlo, int n, int V, CgScalars* sc, double* partials, int count,
                              const int* skip, int block, cudaStream_t st) {
  const int grid = grid_for(n, block);
  if (rhi.prec != SP64) return cudaErrorInvalidValue;
  switch (rlo.prec) {
    case SP32:
      mp_convert_kernel<P32><<<grid, block, 0, st>>>(view<P64>(rhi), view<P32>(rlo), n, V, sc, partials, count, skip);
      break;
    case SP16:
      mp_convert_kernel<P16><<<grid, block, 0, st>>>(view<P64>(rhi), view<P16>(rlo), n, V, sc, partials, count, skip);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_mp_update_p(int precw, FieldPtr p, FieldPtr s, int n, int V, CgScalars* sc, double* partials,
                               int use_cond, unsigned long long cond, int block, cudaStream_t st) {
  const cudaGraphConditionalHandle h = (cudaGraphConditionalHandle)cond;
  switch (precw) {
    case SP32:
      WD_STRIDE(mp_update_p_kernel<P32>)(view<P32>(p), view<P32>(s), n, V, sc, partials, use_cond, h);
      break;
    case SP16:
      WD_STRIDE(mp_update_p_kernel<P16>)(view<P16>(p), view<P16>(s), n, V, sc, partials, use_cond, h);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- double-float helpers

// FP64 -> double-float (hi = rn(x), lo = rn(x - hi)) and back (hi + lo in FP64)
__global__ void f64_to_df_kernel(SpinorRef<P64> in, SpinorRef<PDF> out, int n, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  Cx<double> v[12];
  load_spinor(in, s, V, v);
  Cx<dfloat> w[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) w[c] = cx(dfloat(v[c].re), dfloat(v[c].im));
  store_spinor(out, s, V, w);
}

__global__ void df_to_f64_kernel(SpinorRef<PDF> in, SpinorRef<P64> out, int n, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  Cx<dfloat> w[12];
  load_spinor(in, s, V, w);
  Cx<double> v[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) v[c] = cx((double)w[c].re, (double)w[c].im);
  store_spinor(out, s, V, v);
}

// x_hi += x_lo in double-float (TwoSum of the hi parts), x_lo = 0
__global__ void mp_accumulate_df_kernel(SpinorRef<PDF> xhi, SpinorRef<P32> xlo, int n, int V, const int* skip) {
  if (skip != nullptr && *skip == 0) return;  // runs only when an update is pending
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  Cx<dfloat> xh[12];
  Cx<float> xl[12];
  load_spinor(xhi, s, V, xh);
  load_spinor(xlo, s, V, xl);
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    xh[c].re = xh[c].re + dfloat(xl[c].re, 0.f);
    xh[c].im = xh[c].im + dfloat(xl[c].im, 0.f);
    xl[c] = cx(0.f, 0.f);
  }
  store_spinor(xhi, s, V, xh);
  store_spinor(xlo, s, V, xl);
}

// r_lo = r_hi from a double-float residual (its hi part), then the same bookkeeping as
// mp_convert_kernel
template <int SPW>
__global__ void mp_convert_df_kernel(SpinorRef<PDF> rhi, SpinorRef<SPW> rlo, int n, int V, CgScalars* sc,
                                     double* partials, int count, const int* skip) {
  if (skip != nullptr && *skip == 0) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) {
    Cx<dfloat> h[12];
    Cx<float> l[12];
    load_spinor(rhi, s, V, h);
#pragma unroll
    for (int c = 0; c < 12; ++c) l[c] = cx(h[c].re.hi, h[c].im.hi);
    store_spinor(rlo, s, V, l);
  }
  double v[1] = {0.0}, tot[1];
  if (grid_reduce<OpSum, 1>(v, partials, &sc->ticket[TK_UPD_REL], tot) && threadIdx.x == 0) {
    const double rr = sc->rr_true;
    sc->rr = rr;
    sc->rr_ref = rr;
    sc->need_update = 0;
    sc->no_update = 1;
    if (count) sc->updates += 1;
    if (!isfinite(rr))
      sc->status = ST_BREAKDOWN;
    else if (rr <= sc->tol2 * sc->eta2)
      sc->status = ST_CONVERGED;
  }
}

cudaError_t launch_convert_f64_df(FieldPtr in, FieldPtr out, int n, int V, int to_df, int block, cudaStream_t st) {
  const int grid = grid_for(n, block);
  if (to_df) {
    if (in.prec != SP64 || out.prec != SPDF) return cudaErrorInvalidValue;
    f64_to_df_kernel<<<grid, block, 0, st>>>(view<P64>(in), view_df(out, V), n, V);
  } else {
    if (in.prec != SPDF || out.prec != SP64) return cudaErrorInvalidValue;
    df_to_f64_kernel<<<grid, block, 0, st>>>(view_df(in, V), view<P64>(out), n, V);
  }
  return cudaGetLastError();
}

cudaError_t launch_mp_accumulate_df(FieldPtr xhi, FieldPtr xlo, int n, int V, const int* skip, int block,
                                    cudaStream_t st) {
  if (xhi.prec != SPDF || xlo.prec != SP32) return cudaErrorInvalidValue;
  mp_accumulate_df_kernel<<<grid_for(n, block), block, 0, st>>>(view_df(xhi, V), view<P32>(xlo), n, V, skip);
  return cudaGetLastError();
}

cudaError_t launch_mp_convert_df(FieldPtr rhi, FieldPtr rlo, int n, int V, CgScalars* sc, double* partials, int count,
                                 const int* skip, int block, cudaStream_t st) {
  const int grid = grid_for(n, block);
  if (rhi.prec != SPDF) return cudaErrorInvalidValue;
  switch (rlo.prec) {
    case SP32:
      mp_convert_df_kernel<P32><<<grid, block, 0, st>>>(view_df(rhi, V), view<P32>(rlo), n, V, sc, partials, count, skip);
      break;
    case SP16:
      mp_convert_df_kernel<P16><<<grid, block, 0, st>>>(view_df(rhi, V), view<P16>(rlo), n, V, sc, partials, count, skip);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st) {
  if (bytes % 16) return cudaErrorInvalidValue;
  const size_t n4 = bytes / 16;
  if (n4 == 0) return cudaSuccess;
  zero_kernel<<<(unsigned)((n4 + 255) / 256), 256, 0, st>>>(reinterpret_cast<float4*>(p), n4);
  return cudaGetLastError();
}

}  // namespace wdk
