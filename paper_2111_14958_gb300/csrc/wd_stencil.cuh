// Device-side building blocks of the Wilson-Dirac stencil (Eq. (1)), shared by the dslash,
// even-odd and persistent-loop translation units: precision views, the per-hop spin algebra and
// SU(3) multiply, one output site of D (or of a half-lattice hop), and the FP64 two-lanes-per-site
// pass. See wd_dslash.cu for the arithmetic and byte counts per site.
#pragma once

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

// Both hops of direction mu combined, for the FP64 kernels (bound by their FP64 instruction
// count). With t = U_mu(n) h_f and the backward product t_b = U_mu(n-mu)^dag h_b, the two hops
// add k_f t + k_b t_b to the upper spins and k_f S B^dag t - k_b S B^dag t_b to the lower ones.
// k_b = rho k_f, rho = -1 when exactly one of the two hops crosses an antiperiodic boundary, so
// the sums are k_f p and k_f S B^dag (2 t - p) with p = t + rho t_b: the backward product
// accumulates onto t (no separate multiply), and the pair needs 36 reconstruction operations
// instead of 48. rho is applied to h_b through the sign bits.
template <int MU, int S_FWD, typename In, typename Gauge, typename R>
__device__ __forceinline__ void hop_pair_combined(const In& in, const Gauge& gauge, int s, int nbf, int nbb, int V,
                                                  bool wf, bool wb, bool aper, R mk, Cx<R> (&acc)[12]) {
  Cx<R> t[6];
  {
    Cx<R> psi[12], h[6], u[9];
    load_spinor(in, nbf, V, psi);
    spin_project<MU, S_FWD>(psi, h);
    load_link(gauge, MU, s, V, u);
    su3_mul(u, h, t);
  }
  Cx<R> p[6];
  {
    Cx<R> psi[12], h[6], u[9];
    load_spinor(in, nbb, V, psi);
    spin_project<MU, -S_FWD>(psi, h);
    const unsigned long long m = (unsigned long long)(aper && wf != wb) << 63;
#pragma unroll
    for (int i = 0; i < 6; ++i) h[i] = cx<R>(flip_sign(h[i].re, m), flip_sign(h[i].im, m));
    load_link(gauge, MU, nbb, V, u);
    su3_dag_mul_add(u, h, t, p);
  }
  Cx<R> d[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) d[i] = cx<R>(madd((R)2, t[i].re, -p[i].re), madd((R)2, t[i].im, -p[i].im));
  spin_reconstruct2<MU, S_FWD>(acc, p, d, (aper && wf) ? -mk : mk);
}

template <int MU, int S_FWD, int SP, bool C12, typename R>
__device__ __forceinline__ void hop_pair(const DslashArgs<SP, C12>& a, R mk, int s, const int (&c)[4],
                                         Cx<R> (&acc)[12]) {
  const int V = a.g.V;
  if constexpr (SP == P64) {
    const bool wf = c[MU] == a.g.L[MU] - 1, wb = c[MU] == 0;
    const int nbf = wf ? s - (a.g.L[MU] - 1) * a.g.stride[MU] : s + a.g.stride[MU];
    const int nbb = wb ? s + (a.g.L[MU] - 1) * a.g.stride[MU] : s - a.g.stride[MU];
    hop_pair_combined<MU, S_FWD>(a.in, a.u, s, nbf, nbb, V, wf, wb, a.g.bc[MU] < 0, mk, acc);
    return;
  }
  // forward hop n -> n + mu with U_mu(n)
  {
    const bool wrap = c[MU] == a.g.L[MU] - 1;
    const int nb = wrap ? s - (a.g.L[MU] - 1) * a.g.stride[MU] : s + a.g.stride[MU];
    Cx<R> h[6];
    const R k = load_project_hop<MU, S_FWD>(a.in, nb, V, h, (wrap && a.g.bc[MU] < 0) ? -mk : mk);
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
    Cx<R> h[6];
    const R k = load_project_hop<MU, -S_FWD>(a.in, nb, V, h, (wrap && a.g.bc[MU] < 0) ? -mk : mk);
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

// ---------------------------------------------------------------- load schedules (FP32 / FP16)
//
// FP32 / FP16: the kernel is bound by the latency of its dependent neighbour loads, not by issue.
// Two other schedules keep more loads in flight per thread than hop_pair's one hop at a time: a
// thread that holds NS sites issues every site's loads of a hop before any site's arithmetic
// (dslash_sites), or one site's two hops of a direction are loaded together (hop_pair_loaded).
// The per-site arithmetic and its order are those of hop_pair, so the outputs are the same bits.

template <int SP>
struct HopRaw;
template <>
struct HopRaw<P32> {
  float4 d[6];
};
template <>
struct HopRaw<P16> {
  uint4 d[3];
  float nrm;
};

__device__ __forceinline__ void load_raw(const SpinorRef<P32>& f, int s, int V, HopRaw<P32>& r) {
#pragma unroll
  for (int j = 0; j < 6; ++j) r.d[j] = __ldg(f.p + (size_t)j * V + s);
}
__device__ __forceinline__ void load_raw(const SpinorRef<P16>& f, int s, int V, HopRaw<P16>& r) {
  r.nrm = __ldg(f.norm + s);
#pragma unroll
  for (int j = 0; j < 3; ++j) r.d[j] = __ldg(f.p + (size_t)j * V + s);
}

// spin_project<MU, S> of a loaded neighbour; returns the hop factor (FP16: times the site's norm)
template <int MU, int S>
__device__ __forceinline__ float project_raw(const HopRaw<P32>& r, Cx<float> (&h)[6], float k) {
  Cx<float> psi[12];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    psi[2 * j] = cx(r.d[j].x, r.d[j].y);
    psi[2 * j + 1] = cx(r.d[j].z, r.d[j].w);
  }
  spin_project<MU, S>(psi, h);
  return k;
}
template <int MU, int S>
__device__ __forceinline__ float project_raw(const HopRaw<P16>& r, Cx<float> (&h)[6], float k) {
  uint32_t w[12];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    w[4 * j] = r.d[j].x;
    w[4 * j + 1] = r.d[j].y;
    w[4 * j + 2] = r.d[j].z;
    w[4 * j + 3] = r.d[j].w;
  }
  spin_project_f16<MU, S>(w, h);
  return k * r.nrm;
}

template <bool C12>
struct LinkRaw;
template <>
struct LinkRaw<true> {
  float4 d[3];
};
template <>
struct LinkRaw<false> {
  float2 d[9];
};

__device__ __forceinline__ void load_link_raw(const GaugeRef<float, true>& g, int mu, int s, int V,
                                              LinkRaw<true>& l) {
  const float4* base = g.p + (size_t)mu * 3 * V + s;
#pragma unroll
  for (int j = 0; j < 3; ++j) l.d[j] = __ldg(base + (size_t)j * V);
}
__device__ __forceinline__ void load_link_raw(const GaugeRef<float, false>& g, int mu, int s, int V,
                                              LinkRaw<false>& l) {
  const float2* base = g.p + (size_t)mu * 9 * V + s;
#pragma unroll
  for (int k = 0; k < 9; ++k) l.d[k] = __ldg(base + (size_t)k * V);
}
__device__ __forceinline__ void unpack_link(const LinkRaw<true>& l, Cx<float> (&u)[9]) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    u[2 * j] = cx(l.d[j].x, l.d[j].y);
    u[2 * j + 1] = cx(l.d[j].z, l.d[j].w);
  }
  reconstruct_row2(u);
}
__device__ __forceinline__ void unpack_link(const LinkRaw<false>& l, Cx<float> (&u)[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = cx(l.d[k].x, l.d[k].y);
}

// One hop (DIR 0: forward with U_mu(n); 1: backward with U_mu(n - mu)^dagger) of NS sites.
template <int MU, int DIR, int S, int NS, int SP, bool C12>
__device__ __forceinline__ void hop_sites(const DslashArgs<SP, C12>& a, float mk, const int (&s)[NS],
                                          const int (&c)[NS][4], Cx<float> (&acc)[NS][12]) {
  const int V = a.g.V;
  HopRaw<SP> raw[NS];
  LinkRaw<C12> lk[NS];
  float k[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const bool wrap = DIR == 0 ? c[i][MU] == a.g.L[MU] - 1 : c[i][MU] == 0;
    const int nb = DIR == 0 ? (wrap ? s[i] - (a.g.L[MU] - 1) * a.g.stride[MU] : s[i] + a.g.stride[MU])
                            : (wrap ? s[i] + (a.g.L[MU] - 1) * a.g.stride[MU] : s[i] - a.g.stride[MU]);
    k[i] = (wrap && a.g.bc[MU] < 0) ? -mk : mk;
    load_raw(a.in, nb, V, raw[i]);
    load_link_raw(a.u, MU, DIR == 0 ? s[i] : nb, V, lk[i]);
  }
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    Cx<float> h[6], u[9], chi[6];
    const float kk = project_raw<MU, S>(raw[i], h, k[i]);
    unpack_link(lk[i], u);
    if (DIR == 0)
      su3_mul(u, h, chi);
    else
      su3_dag_mul(u, h, chi);
    spin_reconstruct<MU, S>(acc[i], chi, kk);
  }
}

// NS sites of out = D in (or b - D in); sites with live[i] false are computed but not stored.
// Returns the sum of |out(s)|^2 over the live sites.
template <int SP, bool C12, bool DAG, int EPI, int NS>
__device__ __forceinline__ double dslash_sites(const DslashArgs<SP, C12>& a, const int (&s)[NS],
                                               const bool (&live)[NS]) {
  const int V = a.g.V;
  int c[NS][4];
  Cx<float> acc[NS][12];
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    int r = s[i];
    c[i][0] = r % a.g.L[0];
    r /= a.g.L[0];
    c[i][1] = r % a.g.L[1];
    r /= a.g.L[1];
    c[i][2] = r % a.g.L[2];
    c[i][3] = r / a.g.L[2];
    load_spinor(a.in, s[i], V, acc[i]);
  }
  const float mk = a.kappa_dev ? (float)(-*a.kappa_dev) : a.mkappa;
  constexpr int SF = DAG ? +1 : -1;
  hop_sites<0, 0, SF, NS>(a, mk, s, c, acc);
  hop_sites<0, 1, -SF, NS>(a, mk, s, c, acc);
  hop_sites<1, 0, SF, NS>(a, mk, s, c, acc);
  hop_sites<1, 1, -SF, NS>(a, mk, s, c, acc);
  hop_sites<2, 0, SF, NS>(a, mk, s, c, acc);
  hop_sites<2, 1, -SF, NS>(a, mk, s, c, acc);
  hop_sites<3, 0, SF, NS>(a, mk, s, c, acc);
  hop_sites<3, 1, -SF, NS>(a, mk, s, c, acc);
  double n2 = 0.0;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    if (EPI == EPI_RESID) {
      Cx<float> bv[12];
      load_spinor(a.b, s[i], V, bv);
#pragma unroll
      for (int j = 0; j < 12; ++j) acc[i][j] = cx<float>(bv[j].re - acc[i][j].re, bv[j].im - acc[i][j].im);
    }
    if (live[i]) {
      store_spinor(a.out, s[i], V, acc[i]);
      n2 += norm2_site(acc[i]);
    }
  }
  return n2;
}

// Both hops of direction mu for one site, their loads (neighbour spinors and links) issued before
// either hop's arithmetic: two hops' loads in flight per thread (hop_pair issues them hop by hop).
template <int MU, int SF, int SP, bool C12>
__device__ __forceinline__ void hop_pair_loaded(const DslashArgs<SP, C12>& a, float mk, int s, const int (&c)[4],
                                                Cx<float> (&acc)[12]) {
  const int V = a.g.V;
  HopRaw<SP> rf, rb;
  LinkRaw<C12> lf, lb;
  const bool wf = c[MU] == a.g.L[MU] - 1, wb = c[MU] == 0;
  const int nbf = wf ? s - (a.g.L[MU] - 1) * a.g.stride[MU] : s + a.g.stride[MU];
  const int nbb = wb ? s + (a.g.L[MU] - 1) * a.g.stride[MU] : s - a.g.stride[MU];
  const float kf = (wf && a.g.bc[MU] < 0) ? -mk : mk, kb = (wb && a.g.bc[MU] < 0) ? -mk : mk;
  load_raw(a.in, nbf, V, rf);
  load_link_raw(a.u, MU, s, V, lf);
  load_raw(a.in, nbb, V, rb);
  load_link_raw(a.u, MU, nbb, V, lb);
  {
    Cx<float> h[6], u[9], chi[6];
    const float kk = project_raw<MU, SF>(rf, h, kf);
    unpack_link(lf, u);
    su3_mul(u, h, chi);
    spin_reconstruct<MU, SF>(acc, chi, kk);
  }
  {
    Cx<float> h[6], u[9], chi[6];
    const float kk = project_raw<MU, -SF>(rb, h, kb);
    unpack_link(lb, u);
    su3_dag_mul(u, h, chi);
    spin_reconstruct<MU, -SF>(acc, chi, kk);
  }
}

// One site of out = D in (or b - D in) with hop_pair_loaded; returns |out(s)|^2.
template <int SP, bool C12, bool DAG, int EPI>
__device__ __forceinline__ double dslash_site_loaded(const DslashArgs<SP, C12>& a, int s) {
  const int V = a.g.V;
  int c[4];
  int r = s;
  c[0] = r % a.g.L[0];
  r /= a.g.L[0];
  c[1] = r % a.g.L[1];
  r /= a.g.L[1];
  c[2] = r % a.g.L[2];
  c[3] = r / a.g.L[2];
  Cx<float> acc[12];
  load_spinor(a.in, s, V, acc);
  const float mk = a.kappa_dev ? (float)(-*a.kappa_dev) : a.mkappa;
  constexpr int SF = DAG ? +1 : -1;
  hop_pair_loaded<0, SF>(a, mk, s, c, acc);
  hop_pair_loaded<1, SF>(a, mk, s, c, acc);
  hop_pair_loaded<2, SF>(a, mk, s, c, acc);
  hop_pair_loaded<3, SF>(a, mk, s, c, acc);
  if (EPI == EPI_RESID) {
    Cx<float> bv[12];
    load_spinor(a.b, s, V, bv);
#pragma unroll
    for (int j = 0; j < 12; ++j) acc[j] = cx<float>(bv[j].re - acc[j].re, bv[j].im - acc[j].im);
  }
  store_spinor(a.out, s, V, acc);
  return norm2_site(acc);
}

// One site of out = D in (or b - D in); returns |out(s)|^2 and leaves the stored value in acc.
template <int SP, bool C12, bool DAG, int EPI>
__device__ __forceinline__ double dslash_site_out(const DslashArgs<SP, C12>& a, int s,
                                                  Cx<typename RealOf<SP>::type> (&acc)[12]) {
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

// One site of out = D in (or b - D in); returns |out(s)|^2.
template <int SP, bool C12, bool DAG, int EPI>
__device__ __forceinline__ double dslash_site(const DslashArgs<SP, C12>& a, int s) {
  Cx<typename RealOf<SP>::type> acc[12];
  return dslash_site_out<SP, C12, DAG, EPI>(a, s, acc);
}

// ---------------------------------------------------------------- FP64: time hops in the Dirac basis
//
// The FP64 dslash is bound by its FP64 instruction count. In the spin basis psi' = T psi with
// T = [[1, 1], [-1, 1]] acting on the (upper, lower) spin pairs, the spatial gammas of the chiral
// basis are unchanged (T gamma_k T^-1 = gamma_k, gamma_k = [[0, B], [-B, 0]] with B anti-Hermitian)
// and gamma_t becomes diag(1, 1, -1, -1), so (1 -/+ gamma_t) keeps two spins, doubled: a time hop
// needs no spin projection and its link product feeds only two output spins. The links act on
// colour and commute with T, so D' = T D T^-1 is Eq. (1) with these gammas and the same links and
// boundary phases. The time links enter pre-scaled (scale_time_link below), so a time direction
// costs 2 x 72 = 144 FP64 operations (the link products, accumulated onto the two output spins they
// feed) instead of the 204 of hop_pair_combined (24 projection adds, 144 link products, 36
// reconstruction operations).
// SF: -1 for D (forward hop (1 - gamma_t): lower spins), +1 for D^dagger (upper spins).

// The loop's time links, pre-scaled: tl(s) = 2 mk b(s) U_t(s), mk = -kappa, b(s) the time boundary
// phase when s is on the last time slice (the two hops that use U_t(s) across the lattice edge, the
// forward hop from s and the backward hop into s's neighbour, both start or end there), else 1;
// the 2 is the doubling of the spins (1 -/+ gamma_t) keeps in this basis. One rounding per real
// (the factor 2 is exact). Written by the loop's prologue, one site per call (tl: double2 [9][V]).
__device__ __forceinline__ void scale_time_link(const DslashArgs<P64, false>& a, double2* tl, int s) {
  const int V = a.g.V;
  const double mk = a.kappa_dev ? -*a.kappa_dev : a.mkappa;
  const bool last = s / a.g.stride[3] == a.g.L[3] - 1;
  const double k = 2.0 * ((last && a.g.bc[3] < 0) ? -mk : mk);
  Cx<double> u[9];
  load_link(a.u, 3, s, V, u);
#pragma unroll
  for (int j = 0; j < 9; ++j) tl[(size_t)j * V + s] = make_double2(k * u[j].re, k * u[j].im);
}

// Both time hops of site s in the basis above with the pre-scaled links: acc += tl(s) h_f on the
// spins the forward hop keeps and acc += tl(s - t)^dag h_b on the others. tl is written by the same
// launch, so it is read through the L2 (ld.global.cg), not the read-only path.
template <int SF>
__device__ __forceinline__ void hop_t_dirac(const DslashArgs<P64, false>& a, const double2* tl, int s,
                                            const int (&c)[4], Cx<double> (&acc)[12]) {
  constexpr int FO = SF < 0 ? 6 : 0;  // first component of the spins the forward hop keeps
  constexpr int BO = 6 - FO;          // ... and of those the backward hop keeps
  const int V = a.g.V, L = a.g.L[3], st = a.g.stride[3];
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    const int O = dir == 0 ? FO : BO;
    const int nb = dir == 0 ? (c[3] == L - 1 ? s - (L - 1) * st : s + st) : (c[3] == 0 ? s + (L - 1) * st : s - st);
    const int ls = dir == 0 ? s : nb;  // the link's site
    Cx<double> h[6], u[9], t[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const double2 d = __ldg(a.in.p + (size_t)(O + i) * V + nb);
      h[i] = cx(d.x, d.y);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double2 d = __ldcg(tl + (size_t)k * V + ls);
      u[k] = cx(d.x, d.y);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) t[i] = acc[O + i];
    if (dir == 0)
      su3_mul_add(u, h, t, t);
    else
      su3_dag_mul_add(u, h, t, t);
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[O + i] = t[i];
  }
}

// One site of out' = D' in' (the FP64 operator in the basis above, 18-real links, the time links
// pre-scaled in tl); returns |out'|^2 and leaves the stored value in acc.
template <bool DAG>
__device__ __forceinline__ double dslash_site_dirac_t(const DslashArgs<P64, false>& a, const double2* tl, int s,
                                                      Cx<double> (&acc)[12]) {
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
  const double mk = a.kappa_dev ? -*a.kappa_dev : a.mkappa;
  load_spinor(a.in, s, V, acc);
  constexpr int SF = DAG ? +1 : -1;
  hop_pair<0, SF>(a, mk, s, c, acc);
  hop_pair<1, SF>(a, mk, s, c, acc);
  hop_pair<2, SF>(a, mk, s, c, acc);
  hop_t_dirac<SF>(a, tl, s, c, acc);
  store_spinor(a.out, s, V, acc);
  return norm2_site(acc);
}

// psi' = T psi (upper' = upper + lower, lower' = lower - upper) and its inverse
// psi = T^-1 psi' (upper = (upper' - lower') / 2, lower = (upper' + lower') / 2), in place at site s.
template <bool INVERSE>
__device__ __forceinline__ void dirac_t_basis(const SpinorRef<P64>& f, int s, int V) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const double2 u = f.p[(size_t)i * V + s], l = f.p[(size_t)(6 + i) * V + s];
    double2 a, b;
    if (INVERSE) {
      a = make_double2(0.5 * (u.x - l.x), 0.5 * (u.y - l.y));
      b = make_double2(0.5 * (u.x + l.x), 0.5 * (u.y + l.y));
    } else {
      a = make_double2(u.x + l.x, u.y + l.y);
      b = make_double2(l.x - u.x, l.y - u.y);
    }
    f.p[(size_t)i * V + s] = a;
    f.p[(size_t)(6 + i) * V + s] = b;
  }
}

// Occupancy: the kernel is latency-bound at large volumes (memory-level parallelism comes from
// resident warps), so registers are capped for 3 blocks of 256 threads per SM in FP32/FP16
// (24 warps). The FP64 kernels take one block per SM and up to 255 registers: their FP64 pipe
// saturates with 8 warps, and the combined hops of a direction keep 24 more values live, which
// spill under the 128-register cap of two blocks (measured at 14^4: 62.5 us with one block of
// 255 registers, 63.0 us with two blocks and spills).
constexpr int kDslashMaxThreads = 256;
template <int SP>
struct DslashMinBlocks {
  static constexpr int value = SP == P64 ? 1 : (SP == PDF ? 1 : 3);
};
// The stand-alone FP16 dslash kernel: two blocks of 256 threads per SM (up to 128 registers) give
// it more loads in flight per warp than three blocks give it warps (32^4: 76.5 vs 78.0 us; 24^4
// with 128-thread blocks: 28.8 vs 31.3 us); FP32 stays at three (83.0 vs 86.4 us at 32^4).
template <int SP>
struct DslashKernelMinBlocks {
  static constexpr int value = SP == P16 ? 2 : DslashMinBlocks<SP>::value;
};


// ---------------------------------------------------------------- FP64: two threads per site
//
// The FP64 dslash is bound by the FP64 pipe. At small volumes (8^4, 12^4) one thread per site
// leaves many SMs idle or with one warp per scheduler, and a site's ~850 FP64 instructions set
// the time; splitting a site over two lanes halves that chain (measured at 8^4: 22.5 us against
// 36 us). From 14^4 up the one-thread-per-site kernel, with its combined directions, is faster
// (63 against 69 us), and the block-size tuner chooses between the two kernels per volume.
// Here lanes 2i and 2i+1 share a site: lane h projects only the half-spinor
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

// ---------------------------------------------------------------- FP64: L = 4, 8 or 16 lanes per site
//
// The FP64 pipe of GB300 retires about half a lane-operation per clock per SM sub-partition, so a
// warp's FP64 instruction stream advances one instruction every ~64 cycles and a site's ~850 FP64
// instructions on one thread take ~26 us. At the paper's small volumes (4^4: 256 sites, 8^4: 4,096)
// there are too few warps to occupy the 608 sub-partitions, and the time is that chain. Here L
// consecutive lanes share a site: with L = 4 a lane takes both hops of one direction mu; with L = 8
// one hop; with L = 16 one hop and one of the two rows of its half-spinor. Every lane runs the same
// instructions: the hop's direction, projector, dagger and boundary sign enter as runtime selects
// and sign-bit flips (integer operations), never as branches. Each lane accumulates the
// reconstructed spinor of its hops (24 reals, lower spins in a per-lane order made canonical by
// selects); the site's lanes then reduce-scatter the 24 reals with shuffles, so each lane ends with
// 24 / L of them (with L = 16 the two lanes of a row pair hold the same 3 and one stores), and only
// then apply out = in - kappa * sum (one FMA per real) and the norm. FP64 instructions per lane:
// L = 4: 2 x (12 + 72) + 18 + 6 + 6; L = 8: 84 + 21 + 3 + 3; L = 16: 42 + 24 + 3 + 3.

// bits of a double's high word
__device__ __forceinline__ double neg_if(double x, bool n) {
  return __hiloint2double(__double2hiint(x) ^ (n ? (int)0x80000000 : 0), __double2loint(x));
}

// z * i^e for a runtime e, by selects and sign flips only
__device__ __forceinline__ Cx<double> ipow_rt(Cx<double> z, int e) {
  const bool sw = e & 1;
  const double re = sw ? z.im : z.re, im = sw ? z.re : z.im;
  const int m = e & 3;
  return cx(neg_if(re, m == 1 || m == 2), neg_if(im, m == 2 || m == 3));
}

template <int L>
struct LaneShape {
  static_assert(L == 4 || L == 8 || L == 16, "lanes per site");
  static constexpr int kHops = L == 4 ? 2 : 1;       // hops per lane
  static constexpr int kRows = L == 16 ? 1 : 2;      // half-spinor rows per hop
  static constexpr int kLevels = L == 4 ? 2 : 3;     // reduce-scatter levels (24 -> 24 >> levels reals)
  static constexpr int kOwn = 24 >> kLevels;         // reals a lane owns after the reduce-scatter
};

// The spinor field a lane hop reads: a single field, or (HASB) w = A + c B formed on the fly at
// every neighbour (the fused CG iteration of the persistent loop reads p = s + beta p and
// r = r - alpha q this way). fma(c, B, A) is the exact arithmetic of the vector updates. NC selects
// the read-only (non-coherent) load path, valid only for fields no thread writes during the launch;
// the persistent loop, which rewrites its fields between grid barriers, uses plain loads.
template <bool HASB, bool NC>
struct LaneSrc {
  const double2* A;
  const double2* B;
  double c;
  __device__ __forceinline__ double2 ld(const double2* p) const { return NC ? __ldg(p) : *p; }
  __device__ __forceinline__ double2 get(size_t i) const {
    const double2 a = ld(A + i);
    if (!HASB) return a;
    const double2 b = ld(B + i);
    return make_double2(fma(c, b.x, a.x), fma(c, b.y, a.y));
  }
};

// One hop (mu, dir) of lane rows [r0, r0 + nrows) into the lane accumulator: up[r] (3 complex) for
// upper spin r, lo[r] (3 complex) for the lower spin paired with row r (spin 2 + bcol(mu, r)). The
// first hop of a lane assigns (ACC = false): adding to zero would cost an FP64 add per real.
template <int NROWS, int SF, bool ACC, typename Src>
__device__ __forceinline__ void lane_hop(const Geom& g, const GaugeRef<double, false>& gauge, const Src& in, int s,
                                         const int (&c)[4], int mu, int dir, int r0, Cx<double> (&up)[2][3],
                                         Cx<double> (&lo)[2][3]) {
  const int V = g.V;
  const int L = g.L[mu], st = g.stride[mu];
  const int cm = mu == 0 ? c[0] : (mu == 1 ? c[1] : (mu == 2 ? c[2] : c[3]));
  const bool wrap = dir == 0 ? cm == L - 1 : cm == 0;
  const int nb = dir == 0 ? (wrap ? s - (L - 1) * st : s + st) : (wrap ? s + (L - 1) * st : s - st);
  const bool flip = wrap && g.bc[mu] < 0;  // boundary phase -1, applied to the projected spinor
  const int S = dir == 0 ? SF : -SF;       // projector (1 + S gamma_mu)
  // link U_mu(s) (forward) or U_mu(nb)^dagger (backward)
  Cx<double> u[9];
  load_link(gauge, mu, dir == 0 ? s : nb, V, u);
  Cx<double> ue[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const Cx<double> t = u[3 * j + i];
      ue[3 * i + j] = dir == 0 ? u[3 * i + j] : cx(t.re, -t.im);
    }
#pragma unroll
  for (int k = 0; k < NROWS; ++k) {
    const int r = r0 + k;
    const int col = bcol(mu, r);
    const int e = bph(mu, r) + (S < 0 ? 2 : 0);  // h_r = psi_r + S B[r][col] psi_{2+col}
    Cx<double> h[3];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      const double2 pu = in.get((size_t)(3 * r + cc) * V + nb);
      const double2 pl = in.get((size_t)(3 * (2 + col) + cc) * V + nb);
      const Cx<double> l = ipow_rt(cx(pl.x, pl.y), e);
      h[cc] = cx(neg_if(pu.x + l.re, flip), neg_if(pu.y + l.im, flip));
    }
    // chi = ue h; upper spin r += chi; lower spin 2 + col += S conj(B[r][col]) chi
    const int el = (4 - bph(mu, r)) + (S < 0 ? 2 : 0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const Cx<double> u0 = ue[3 * i], u1 = ue[3 * i + 1], u2 = ue[3 * i + 2];
      double re = u0.re * h[0].re;
      re = fma(-u0.im, h[0].im, re);
      re = fma(u1.re, h[1].re, re);
      re = fma(-u1.im, h[1].im, re);
      re = fma(u2.re, h[2].re, re);
      re = fma(-u2.im, h[2].im, re);
      double im = u0.re * h[0].im;
      im = fma(u0.im, h[0].re, im);
      im = fma(u1.re, h[1].im, im);
      im = fma(u1.im, h[1].re, im);
      im = fma(u2.re, h[2].im, im);
      im = fma(u2.im, h[2].re, im);
      const Cx<double> t = ipow_rt(cx(re, im), el);
      if (ACC) {
        up[k][i] = cx(up[k][i].re + re, up[k][i].im + im);
        lo[k][i] = cx(lo[k][i].re + t.re, lo[k][i].im + t.im);
      } else {
        up[k][i] = cx(re, im);
        lo[k][i] = t;
      }
    }
  }
}

// The hopping sum of one site for this lane's share: on return v[0 .. kOwn) holds the lane's owned
// reals j = base + i of sum_hops (projector, link and boundary phase applied; -kappa not yet), with
// j = 2 (3 spin + colour) + (0 re, 1 im). All L lanes of the site must call it together.
template <int L, bool DAG, typename Src>
__device__ __forceinline__ void lanes_hopsum(const Geom& g, const GaugeRef<double, false>& gauge, const Src& in, int s,
                                             int lane, double (&v)[24], int& base) {
  typedef LaneShape<L> Sh;
  constexpr int SF = DAG ? +1 : -1;
  int c[4];
  {
    int r = s;
    c[0] = r % g.L[0];
    r /= g.L[0];
    c[1] = r % g.L[1];
    r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];
  }
  // the lane's hops all share one direction mu
  const int mu = L == 4 ? lane : (L == 8 ? lane >> 1 : lane >> 2);
  const int r0 = L == 16 ? (lane & 1) : 0;
  Cx<double> up[2][3], lo[2][3];
  if (L == 4) {  // both hops of direction mu
    lane_hop<Sh::kRows, SF, false>(g, gauge, in, s, c, mu, 0, r0, up, lo);
    lane_hop<Sh::kRows, SF, true>(g, gauge, in, s, c, mu, 1, r0, up, lo);
  } else {
    const int dir = L == 8 ? (lane & 1) : ((lane >> 1) & 1);
    lane_hop<Sh::kRows, SF, false>(g, gauge, in, s, c, mu, dir, r0, up, lo);
  }
  // canonical order. Row r's upper spin is r; its lower spin is 2 + bcol(mu, r) = 2 + (r ^ (mu < 2)).
  const bool swp = mu < 2;
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Cx<double> z;
      if (Sh::kRows == 2) {
        if (sp < 2) z = up[sp][i];
        else z = ((sp - 2) ^ (int)swp) ? lo[1][i] : lo[0][i];
      } else {  // one row r0: upper spin r0 and lower spin 2 + (r0 ^ swp); zero elsewhere
        const bool here = sp < 2 ? sp == r0 : (sp - 2) == (r0 ^ (int)swp);
        const Cx<double> src = sp < 2 ? up[0][i] : lo[0][i];
        z = here ? src : cx(0.0, 0.0);
      }
      v[2 * (3 * sp + i)] = z.re;
      v[2 * (3 * sp + i) + 1] = z.im;
    }
  // reduce-scatter over the site's lanes: at each level keep the half selected by one lane bit
  base = 0;
#pragma unroll
  for (int lev = 0; lev < Sh::kLevels; ++lev) {
    const int half = 12 >> lev;
    const int m = (L >> 1) >> lev;  // lane bit of this level (highest first)
    const bool hi = lane & m;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const double send = hi ? v[i] : v[i + half];
      const double keep = hi ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
    base += hi ? half : 0;
  }
  if (L == 16) {  // lanes 2i and 2i + 1 hold the same reals: sum them
#pragma unroll
    for (int i = 0; i < Sh::kOwn; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], 1);
  }
}

// flat double index of real j of site s in the [12][V] double2 layout
__device__ __forceinline__ size_t real_index(int j, int s, int V) { return ((size_t)(j >> 1) * V + s) * 2 + (j & 1); }

// All sites of out = D in (or b - D in) with L lanes per site over the whole grid (grid-stride on
// the warp's first site, so all 32 lanes take the same trips and meet at the shuffles); returns this
// thread's share of |out|^2.
template <int L, bool DAG, int EPI>
__device__ __forceinline__ double lanes_sites(const DslashArgs<P64, false>& a) {
  typedef LaneShape<L> Sh;
  const int V = a.g.V;
  const int lane = threadIdx.x & (L - 1);
  double n2 = 0.0;
  const int step = (gridDim.x * blockDim.x) / L;
  LaneSrc<false, true> src;
  src.A = a.in.p;
  src.B = nullptr;
  src.c = 0.0;
  for (int s0 = (blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / L; s0 < V; s0 += step) {
    const int sl = s0 + (threadIdx.x & 31) / L;
    const bool live = sl < V;
    const int s = live ? sl : s0;
    double v[24];
    int base;
    lanes_hopsum<L, DAG>(a.g, a.u, src, s, lane, v, base);
    if (!live || (L == 16 && (lane & 1))) continue;
    const double mk = a.kappa_dev ? -*a.kappa_dev : a.mkappa;
    const double* in = reinterpret_cast<const double*>(a.in.p);
    double* out = reinterpret_cast<double*>(a.out.p);
#pragma unroll
    for (int i = 0; i < Sh::kOwn; ++i) {
      const size_t idx = real_index(base + i, s, V);
      double o = fma(mk, v[i], __ldg(in + idx));
      if (EPI == EPI_RESID) o = __ldg(reinterpret_cast<const double*>(a.b.p) + idx) - o;
      out[idx] = o;
      n2 = fma(o, o, n2);
    }
  }
  return n2;
}

// One pass of the fused CG iteration with L lanes per site (persistent FP64 loop at small volumes):
// w = A + c B formed at every neighbour and at the site itself (w = A without B), out = D w (or
// D^dag w); the site's w is also stored to wout (if set) and x += ax * xs at the site (if x is set).
// Returns this thread's shares of |out|^2 and |w|^2.
struct FusedPass {
  const double2* A;
  const double2* B;
  double c;
  double2* wout;
  double2* out;
  double2* x;
  const double2* xs;
  double ax;
};

template <int L, bool DAG, bool HASB>
__device__ __forceinline__ void lanes_fused_sites(const Geom& g, const GaugeRef<double, false>& gauge, double mk,
                                                  const FusedPass& f, double& n_out, double& n_w) {
  typedef LaneShape<L> Sh;
  const int V = g.V;
  const int lane = threadIdx.x & (L - 1);
  const int step = (gridDim.x * blockDim.x) / L;
  LaneSrc<HASB, false> src;
  src.A = f.A;
  src.B = f.B;
  src.c = f.c;
  const double* A = reinterpret_cast<const double*>(f.A);
  const double* B = reinterpret_cast<const double*>(f.B);
  double* wout = reinterpret_cast<double*>(f.wout);
  double* out = reinterpret_cast<double*>(f.out);
  double* x = reinterpret_cast<double*>(f.x);
  const double* xs = reinterpret_cast<const double*>(f.xs);
  for (int s0 = (blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / L; s0 < V; s0 += step) {
    const int sl = s0 + (threadIdx.x & 31) / L;
    const bool live = sl < V;
    const int s = live ? sl : s0;
    double v[24];
    int base;
    lanes_hopsum<L, DAG>(g, gauge, src, s, lane, v, base);
    if (!live || (L == 16 && (lane & 1))) continue;
#pragma unroll
    for (int i = 0; i < Sh::kOwn; ++i) {
      const size_t idx = real_index(base + i, s, V);
      double w = A[idx];
      if (HASB) w = fma(f.c, B[idx], w);
      if (wout) wout[idx] = w;
      const double o = fma(mk, v[i], w);
      out[idx] = o;
      if (x) x[idx] = fma(f.ax, xs[idx], x[idx]);
      n_out = fma(o, o, n_out);
      n_w = fma(w, w, n_w);
    }
  }
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
  if constexpr (SP == P64) {
    const bool wf = c[MU] == a.e.g.L[MU] - 1, wb = c[MU] == 0;
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[MU] = wf ? 0 : c[MU] + 1;
    const int nbf = eo_index(a.e.g, n);
    n[MU] = wb ? a.e.g.L[MU] - 1 : c[MU] - 1;
    const int nbb = eo_index(a.e.g, n);
    hop_pair_combined<MU, SF>(a.in, a.u, s, nbf, nbb, V, wf, wb, a.e.g.bc[MU] < 0, k0, acc);
    return;
  }
  {
    int n[4] = {c[0], c[1], c[2], c[3]};
    const bool wrap = n[MU] == a.e.g.L[MU] - 1;
    n[MU] = wrap ? 0 : n[MU] + 1;
    const int nb = eo_index(a.e.g, n);
    Cx<R> h[6], u[9], chi[6];
    const R k = load_project_hop<MU, SF>(a.in, nb, V, h, (wrap && a.e.g.bc[MU] < 0) ? -k0 : k0);
    load_link(a.u, MU, s, V, u);
    su3_mul(u, h, chi);
    spin_reconstruct<MU, SF>(acc, chi, k);
  }
  {
    int n[4] = {c[0], c[1], c[2], c[3]};
    const bool wrap = n[MU] == 0;
    n[MU] = wrap ? a.e.g.L[MU] - 1 : n[MU] - 1;
    const int nb = eo_index(a.e.g, n);
    Cx<R> h[6], u[9], chi[6];
    const R k = load_project_hop<MU, -SF>(a.in, nb, V, h, (wrap && a.e.g.bc[MU] < 0) ? -k0 : k0);
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

}  // namespace wdk
