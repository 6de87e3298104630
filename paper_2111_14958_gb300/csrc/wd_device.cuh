// Device-side building blocks of the Wilson-Dirac library: field layouts, complex arithmetic,
// spin projection/reconstruction for the chiral basis, SU(3) products and deterministic grid
// reductions. Included by the kernel translation units only.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wdk {

// Storage precisions of spinor fields. PDF: double-float, two FP32 arrays (hi, lo) whose sum
// carries about 48 significant bits; arithmetic on the FP32 pipes (see dfloat below).
enum { P64 = 0, P32 = 1, P16 = 2, PDF = 3 };

// ---------------------------------------------------------------- double-float arithmetic
//
// A value is hi + lo with |lo| <= ulp(hi)/2, hi and lo FP32. Sums and products use the
// error-free transformations of Knuth (TwoSum), Dekker/FMA (TwoProduct) and the renormalisation
// FastTwoSum (Dekker 1971; see also Hida, Li, Bailey, "Library for double-double and quad-double
// arithmetic", 2000, for the "sloppy" double-double add used here). Every step uses the _rn
// intrinsics, which the compiler never fuses into FMAs, so each transformation stays exact.
// Relative error per operation ~2^-47; used where FP64 accuracy is needed but the FP64 pipe
// (1/58 of the FP32 rate on GB300) would be the bottleneck.
struct dfloat {
  float hi, lo;
  __device__ __forceinline__ dfloat() {}
  __device__ __forceinline__ dfloat(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit dfloat(double d) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
  }
  __device__ __forceinline__ dfloat(int i) : hi((float)i), lo(0.f) {}
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfloat(s, e);
}

__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
  dfloat s = df_two_sum(x.hi, y.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }
__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df_fast_two_sum(p, e);
}
// a * b + c. The templates below call madd for every precision (not fma, whose double overload a
// dfloat one would hide inside this namespace).
__device__ __forceinline__ double madd(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ dfloat madd(dfloat a, dfloat b, dfloat c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  dfloat s = df_two_sum(c.hi, p);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(c.lo, e)));
}

// Lattice geometry. Site index s = x + Lx*(y + Ly*(z + Lz*t)); stride[mu] = step of s along mu.
struct Geom {
  int L[4];
  int stride[4];
  int V;
  int bc[4];  // +1 periodic, -1 antiperiodic
};

template <typename R>
struct Cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> cx(R a, R b) {
  Cx<R> z;
  z.re = a;
  z.im = b;
  return z;
}

// ---------------------------------------------------------------- spinor field views
//
// Device layout: structure of arrays over sites, so that consecutive threads (sites) touch
// consecutive addresses for every component.
//   P64: double2 [12][V]           component c = 3*spin + colour
//   P32: float4  [6][V]            pair j holds components 2j and 2j+1
//   P16: uint4   [3][V] + float[V] each uint4 holds 4 components as half2 (re, im), scaled by
//                                   the per-site norm (max |re|, |im| over the site's 24 reals)

template <int P>
struct SpinorRef;

template <>
struct SpinorRef<P64> {
  double2* p;
  typedef double real;
};

template <>
struct SpinorRef<P32> {
  float4* p;
  typedef float real;
};

template <>
struct SpinorRef<P16> {
  uint4* p;
  float* norm;
  typedef float real;
};

// PDF: hi and lo arrays, each float4 [6][V] (the FP32 layout)
template <>
struct SpinorRef<PDF> {
  float4* hi;
  float4* lo;
  typedef dfloat real;
};

__device__ __forceinline__ void load_spinor(const SpinorRef<PDF>& f, int s, int V, Cx<dfloat> (&v)[12]) {
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float4 h = __ldg(f.hi + (size_t)j * V + s), l = __ldg(f.lo + (size_t)j * V + s);
    v[2 * j] = cx(dfloat(h.x, l.x), dfloat(h.y, l.y));
    v[2 * j + 1] = cx(dfloat(h.z, l.z), dfloat(h.w, l.w));
  }
}

__device__ __forceinline__ void store_spinor(const SpinorRef<PDF>& f, int s, int V, const Cx<dfloat> (&v)[12]) {
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    f.hi[(size_t)j * V + s] = make_float4(v[2 * j].re.hi, v[2 * j].im.hi, v[2 * j + 1].re.hi, v[2 * j + 1].im.hi);
    f.lo[(size_t)j * V + s] = make_float4(v[2 * j].re.lo, v[2 * j].im.lo, v[2 * j + 1].re.lo, v[2 * j + 1].im.lo);
  }
}

__device__ __forceinline__ void load_spinor(const SpinorRef<P64>& f, int s, int V, Cx<double> (&v)[12]) {
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const double2 d = __ldg(f.p + (size_t)c * V + s);
    v[c] = cx(d.x, d.y);
  }
}

__device__ __forceinline__ void load_spinor(const SpinorRef<P32>& f, int s, int V, Cx<float> (&v)[12]) {
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float4 d = __ldg(f.p + (size_t)j * V + s);
    v[2 * j] = cx(d.x, d.y);
    v[2 * j + 1] = cx(d.z, d.w);
  }
}

__device__ __forceinline__ void load_spinor(const SpinorRef<P16>& f, int s, int V, Cx<float> (&v)[12]) {
  const float nrm = __ldg(f.norm + s);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const uint4 d = __ldg(f.p + (size_t)j * V + s);
    const uint32_t w[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __half2 h = *reinterpret_cast<const __half2*>(&w[k]);
      const float2 fl = __half22float2(h);
      v[4 * j + k] = cx(fl.x * nrm, fl.y * nrm);
    }
  }
}

__device__ __forceinline__ void store_spinor(const SpinorRef<P64>& f, int s, int V, const Cx<double> (&v)[12]) {
#pragma unroll
  for (int c = 0; c < 12; ++c) f.p[(size_t)c * V + s] = make_double2(v[c].re, v[c].im);
}

__device__ __forceinline__ void store_spinor(const SpinorRef<P32>& f, int s, int V, const Cx<float> (&v)[12]) {
#pragma unroll
  for (int j = 0; j < 6; ++j)
    f.p[(size_t)j * V + s] = make_float4(v[2 * j].re, v[2 * j].im, v[2 * j + 1].re, v[2 * j + 1].im);
}

__device__ __forceinline__ void store_spinor(const SpinorRef<P16>& f, int s, int V, const Cx<float> (&v)[12]) {
  float m = 0.f;
#pragma unroll
  for (int c = 0; c < 12; ++c) m = fmaxf(m, fmaxf(fabsf(v[c].re), fabsf(v[c].im)));
  const float inv = m > 0.f ? 1.0f / m : 0.f;
  f.norm[s] = m;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __half2 h = __floats2half2_rn(v[4 * j + k].re * inv, v[4 * j + k].im * inv);
      w[k] = *reinterpret_cast<uint32_t*>(&h);
    }
    f.p[(size_t)j * V + s] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// ---------------------------------------------------------------- gauge field views
//
//   FP64, 18 reals: double2 [4][9][V]  (component k = 3*row + col)
//   FP32, 18 reals: float2  [4][9][V]
//   FP32, 12 reals: float4  [4][3][V]  (rows 0 and 1; pair j holds components 2j, 2j+1)

template <typename R, bool C12>
struct GaugeRef;

template <>
struct GaugeRef<double, false> {
  const double2* p;
};

template <>
struct GaugeRef<float, false> {
  const float2* p;
};

template <>
struct GaugeRef<float, true> {
  const float4* p;
};

// double-float links: hi and lo arrays, each float2 [4][9][V]
template <>
struct GaugeRef<dfloat, false> {
  const float2* p;  // hi; lo follows at p + 36 V
};

template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return cx<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}

template <typename R>
__device__ __forceinline__ Cx<R> conj_(Cx<R> a) {
  return cx<R>(a.re, -a.im);
}

// row 2 of an SU(3) matrix from rows 0 and 1: conj(row0 x row1)
template <typename R>
__device__ __forceinline__ void reconstruct_row2(Cx<R> (&u)[9]) {
  const Cx<R> a = cmul(u[1], u[5]), b = cmul(u[2], u[4]);
  const Cx<R> c = cmul(u[2], u[3]), d = cmul(u[0], u[5]);
  const Cx<R> e = cmul(u[0], u[4]), f = cmul(u[1], u[3]);
  u[6] = cx<R>(a.re - b.re, -(a.im - b.im));
  u[7] = cx<R>(c.re - d.re, -(c.im - d.im));
  u[8] = cx<R>(e.re - f.re, -(e.im - f.im));
}

__device__ __forceinline__ void load_link(const GaugeRef<double, false>& g, int mu, int s, int V,
                                          Cx<double> (&u)[9]) {
  const double2* base = g.p + (size_t)mu * 9 * V + s;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double2 d = __ldg(base + (size_t)k * V);
    u[k] = cx(d.x, d.y);
  }
}

__device__ __forceinline__ void load_link(const GaugeRef<float, false>& g, int mu, int s, int V,
                                          Cx<float> (&u)[9]) {
  const float2* base = g.p + (size_t)mu * 9 * V + s;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float2 d = __ldg(base + (size_t)k * V);
    u[k] = cx(d.x, d.y);
  }
}

__device__ __forceinline__ void load_link(const GaugeRef<dfloat, false>& g, int mu, int s, int V,
                                          Cx<dfloat> (&u)[9]) {
  const float2* hi = g.p + (size_t)mu * 9 * V + s;
  const float2* lo = hi + (size_t)36 * V;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float2 h = __ldg(hi + (size_t)k * V), l = __ldg(lo + (size_t)k * V);
    u[k] = cx(dfloat(h.x, l.x), dfloat(h.y, l.y));
  }
}

__device__ __forceinline__ void load_link(const GaugeRef<float, true>& g, int mu, int s, int V,
                                          Cx<float> (&u)[9]) {
  const float4* base = g.p + (size_t)mu * 3 * V + s;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float4 d = __ldg(base + (size_t)j * V);
    u[2 * j] = cx(d.x, d.y);
    u[2 * j + 1] = cx(d.z, d.w);
  }
  reconstruct_row2(u);
}

// ---------------------------------------------------------------- spin algebra (chiral basis)
//
// gamma_mu = [[0, B_mu], [B_mu^dag, 0]] in 2x2 spin blocks, with
//   B_x = -i sigma_1 = [[0,-i],[-i,0]],  B_y = -i sigma_2 = [[0,-1],[1,0]],
//   B_z = -i sigma_3 = diag(-i, i),      B_t = 1.
// For a hop with spin factor (1 + S gamma_mu), S = +1 or -1:
//   upper = psi_u + S B psi_l =: h,   lower = psi_l + S B^dag psi_u = S B^dag h,
// so only the two-spin half-spinor h is multiplied by the link (spin projection).

template <int S, typename R>
__device__ __forceinline__ R sg(R x) {
  return S > 0 ? x : -x;
}

template <int MU, int S, typename R>
__device__ __forceinline__ void spin_project(const Cx<R> (&psi)[12], Cx<R> (&h)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cx<R> p0 = psi[c], p1 = psi[3 + c], p2 = psi[6 + c], p3 = psi[9 + c];
    if (MU == 0) {  // B psi_l = (-i p3, -i p2); -i z = (z.im, -z.re)
      h[c] = cx<R>(p0.re + sg<S>(p3.im), p0.im - sg<S>(p3.re));
      h[3 + c] = cx<R>(p1.re + sg<S>(p2.im), p1.im - sg<S>(p2.re));
    } else if (MU == 1) {  // B psi_l = (-p3, p2)
      h[c] = cx<R>(p0.re - sg<S>(p3.re), p0.im - sg<S>(p3.im));
      h[3 + c] = cx<R>(p1.re + sg<S>(p2.re), p1.im + sg<S>(p2.im));
    } else if (MU == 2) {  // B psi_l = (-i p2, i p3); i z = (-z.im, z.re)
      h[c] = cx<R>(p0.re + sg<S>(p2.im), p0.im - sg<S>(p2.re));
      h[3 + c] = cx<R>(p1.re - sg<S>(p3.im), p1.im + sg<S>(p3.re));
    } else {  // B psi_l = (p2, p3)
      h[c] = cx<R>(p0.re + sg<S>(p2.re), p0.im + sg<S>(p2.im));
      h[3 + c] = cx<R>(p1.re + sg<S>(p3.re), p1.im + sg<S>(p3.im));
    }
  }
}

// ---------------------------------------------------------------- FP16 neighbour spinors
//
// The spin projection of a stored FP16 spinor without widening all 24 halves first: the upper
// two spins are converted to FP32, and each lower-spin half enters its sum through a mixed-precision
// FMA, c + (+-1) * a with a in FP16 and c in FP32 (the product by +-1 is exact, so this is the FP32
// sum of c and the widened a, rounded once: the same bits as converting then adding). 12
// conversions and 12 FMAs per hop instead of 24 conversions and 24 adds.

__device__ __forceinline__ void split_f16x2(uint32_t w, unsigned short& lo, unsigned short& hi) {
  asm("mov.b32 {%0, %1}, %2;" : "=h"(lo), "=h"(hi) : "r"(w));
}

__device__ __forceinline__ float f16_to_f32(unsigned short a) {
  float d;
  asm("cvt.f32.f16 %0, %1;" : "=f"(d) : "h"(a));
  return d;
}

// c + SGN * a
template <int SGN>
__device__ __forceinline__ float add_f16(unsigned short a, float c) {
  const unsigned short one = SGN > 0 ? (unsigned short)0x3C00 : (unsigned short)0xBC00;
  float d;
  asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(a), "h"(one), "f"(c));
  return d;
}

// spin_project on the 12 half2 words (re in the low half) of an FP16 spinor, component 4j + q in
// word 4j + q
template <int MU, int S>
__device__ __forceinline__ void spin_project_f16(const uint32_t (&w)[12], Cx<float> (&h)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    unsigned short r0, i0, r1, i1, r2, i2, r3, i3;
    split_f16x2(w[c], r0, i0);
    split_f16x2(w[3 + c], r1, i1);
    split_f16x2(w[6 + c], r2, i2);
    split_f16x2(w[9 + c], r3, i3);
    const float a0 = f16_to_f32(r0), b0 = f16_to_f32(i0), a1 = f16_to_f32(r1), b1 = f16_to_f32(i1);
    if (MU == 0) {  // (p0.re + S p3.im, p0.im - S p3.re), (p1.re + S p2.im, p1.im - S p2.re)
      h[c] = cx<float>(add_f16<S>(i3, a0), add_f16<-S>(r3, b0));
      h[3 + c] = cx<float>(add_f16<S>(i2, a1), add_f16<-S>(r2, b1));
    } else if (MU == 1) {  // (p0 - S p3), (p1 + S p2)
      h[c] = cx<float>(add_f16<-S>(r3, a0), add_f16<-S>(i3, b0));
      h[3 + c] = cx<float>(add_f16<S>(r2, a1), add_f16<S>(i2, b1));
    } else if (MU == 2) {  // (p0.re + S p2.im, p0.im - S p2.re), (p1.re - S p3.im, p1.im + S p3.re)
      h[c] = cx<float>(add_f16<S>(i2, a0), add_f16<-S>(r2, b0));
      h[3 + c] = cx<float>(add_f16<-S>(i3, a1), add_f16<S>(r3, b1));
    } else {  // (p0 + S p2), (p1 + S p3)
      h[c] = cx<float>(add_f16<S>(r2, a0), add_f16<S>(i2, b0));
      h[3 + c] = cx<float>(add_f16<S>(r3, a1), add_f16<S>(i3, b1));
    }
  }
}

// Neighbour spinor of a hop, projected: h = spin_project<MU, S>(psi(s)); returns the hop's
// reconstruction factor. The FP16 form leaves the per-site norm out of h and folds it into that
// factor instead (the hop is linear in the spinor): one multiply per hop instead of 24.
template <int MU, int S, typename Ref, typename R>
__device__ __forceinline__ R load_project_hop(const Ref& f, int s, int V, Cx<R> (&h)[6], R k) {
  Cx<R> psi[12];
  load_spinor(f, s, V, psi);
  spin_project<MU, S>(psi, h);
  return k;
}

template <int MU, int S>
__device__ __forceinline__ float load_project_hop(const SpinorRef<P16>& f, int s, int V, Cx<float> (&h)[6],
                                                  float k) {
  const float nrm = __ldg(f.norm + s);
  uint32_t w[12];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const uint4 d = __ldg(f.p + (size_t)j * V + s);
    w[4 * j] = d.x;
    w[4 * j + 1] = d.y;
    w[4 * j + 2] = d.z;
    w[4 * j + 3] = d.w;
  }
  spin_project_f16<MU, S>(w, h);
  return k * nrm;
}

// acc += k * [chi ; S B^dag chi]  (chi = link x h, two spins x three colours)
template <int MU, int S, typename R>
__device__ __forceinline__ void spin_reconstruct(Cx<R> (&acc)[12], const Cx<R> (&chi)[6], R k) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cx<R> c0 = chi[c], c1 = chi[3 + c];
    acc[c].re = madd(k, c0.re, acc[c].re);
    acc[c].im = madd(k, c0.im, acc[c].im);
    acc[3 + c].re = madd(k, c1.re, acc[3 + c].re);
    acc[3 + c].im = madd(k, c1.im, acc[3 + c].im);
    Cx<R> l0, l1;
    if (MU == 0) {  // B^dag chi = (i c1, i c0)
      l0 = cx<R>(-c1.im, c1.re);
      l1 = cx<R>(-c0.im, c0.re);
    } else if (MU == 1) {  // (c1, -c0)
      l0 = c1;
      l1 = cx<R>(-c0.re, -c0.im);
    } else if (MU == 2) {  // (i c0, -i c1)
      l0 = cx<R>(-c0.im, c0.re);
      l1 = cx<R>(c1.im, -c1.re);
    } else {  // (c0, c1)
      l0 = c0;
      l1 = c1;
    }
    acc[6 + c].re = madd(k, sg<S>(l0.re), acc[6 + c].re);
    acc[6 + c].im = madd(k, sg<S>(l0.im), acc[6 + c].im);
    acc[9 + c].re = madd(k, sg<S>(l1.re), acc[9 + c].re);
    acc[9 + c].im = madd(k, sg<S>(l1.im), acc[9 + c].im);
  }
}

// acc += k * [up ; S B^dag lo]: the reconstruction of spin_reconstruct with separate half-spinors
// for the upper and the lower spins (the two hops of one direction combined, see hop_pair)
template <int MU, int S, typename R>
__device__ __forceinline__ void spin_reconstruct2(Cx<R> (&acc)[12], const Cx<R> (&up)[6], const Cx<R> (&lo)[6],
                                                  R k) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c].re = madd(k, up[c].re, acc[c].re);
    acc[c].im = madd(k, up[c].im, acc[c].im);
    acc[3 + c].re = madd(k, up[3 + c].re, acc[3 + c].re);
    acc[3 + c].im = madd(k, up[3 + c].im, acc[3 + c].im);
    const Cx<R> c0 = lo[c], c1 = lo[3 + c];
    Cx<R> l0, l1;
    if (MU == 0) {
      l0 = cx<R>(-c1.im, c1.re);
      l1 = cx<R>(-c0.im, c0.re);
    } else if (MU == 1) {
      l0 = c1;
      l1 = cx<R>(-c0.re, -c0.im);
    } else if (MU == 2) {
      l0 = cx<R>(-c0.im, c0.re);
      l1 = cx<R>(c1.im, -c1.re);
    } else {
      l0 = c0;
      l1 = c1;
    }
    acc[6 + c].re = madd(k, sg<S>(l0.re), acc[6 + c].re);
    acc[6 + c].im = madd(k, sg<S>(l0.im), acc[6 + c].im);
    acc[9 + c].re = madd(k, sg<S>(l1.re), acc[9 + c].re);
    acc[9 + c].im = madd(k, sg<S>(l1.im), acc[9 + c].im);
  }
}

// Sign flip of a double through its sign bit (an integer operation, off the FP64 pipe).
__device__ __forceinline__ double flip_sign(double x, unsigned long long m) {
  return __longlong_as_double(__double_as_longlong(x) ^ m);
}

// ---------------------------------------------------------------- runtime hop (compact code)
//
// The same spin algebra as spin_project / spin_reconstruct, driven by small tables instead of
// template parameters, so one copy of the code serves all 8 hops. Used where the per-hop code is
// long (double-float): fully unrolled, such a kernel no longer fits the instruction cache.
// B_mu row r has its single non-zero at column bcol(mu, r) with phase i^bph(mu, r):
// B_x = [[0,-i],[-i,0]], B_y = [[0,-1],[1,0]], B_z = diag(-i, i), B_t = 1.
__device__ __forceinline__ int bcol(int mu, int r) { return mu < 2 ? 1 - r : r; }
__device__ __forceinline__ int bph(int mu, int r) {
  return mu == 0 ? 3 : (mu == 1 ? (r ? 0 : 2) : (mu == 2 ? (r ? 1 : 3) : 0));
}

template <typename R>
__device__ __forceinline__ Cx<R> mul_ipow(Cx<R> z, int k) {  // z * i^k
  switch (k & 3) {
    case 0: return z;
    case 1: return cx<R>(-z.im, z.re);
    case 2: return cx<R>(-z.re, -z.im);
    default: return cx<R>(z.im, -z.re);
  }
}

template <typename R>
__device__ __forceinline__ Cx<R> cadd(Cx<R> a, Cx<R> b) {
  return cx<R>(a.re + b.re, a.im + b.im);
}

// h = psi_u + S B_mu psi_l
template <typename R>
__device__ __forceinline__ void spin_project_rt(int mu, int S, const Cx<R> (&psi)[12], Cx<R> (&h)[6]) {
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int col = bcol(mu, r), ph = bph(mu, r) + (S < 0 ? 2 : 0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const Cx<R> l = col == 0 ? psi[6 + c] : psi[9 + c];  // selects: no dynamic register indexing
      h[3 * r + c] = cadd(psi[3 * r + c], mul_ipow(l, ph));
    }
  }
}

// acc_u += k chi;  acc_l += k S B_mu^dag chi  ((B^dag)[col][r] = conj(B[r][col]))
template <typename R>
__device__ __forceinline__ void spin_reconstruct_rt(int mu, int S, Cx<R> (&acc)[12], const Cx<R> (&chi)[6], R k) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    acc[i].re = madd(k, chi[i].re, acc[i].re);
    acc[i].im = madd(k, chi[i].im, acc[i].im);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int col = bcol(mu, r), ph = (4 - bph(mu, r)) + (S < 0 ? 2 : 0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const Cx<R> l = mul_ipow(chi[3 * r + c], ph);
      if (col == 0) {  // both branches index statically
        acc[6 + c].re = madd(k, l.re, acc[6 + c].re);
        acc[6 + c].im = madd(k, l.im, acc[6 + c].im);
      } else {
        acc[9 + c].re = madd(k, l.re, acc[9 + c].re);
        acc[9 + c].im = madd(k, l.im, acc[9 + c].im);
      }
    }
  }
}

// chi = U h (per spin), U row-major 3x3
template <typename R>
__device__ __forceinline__ void su3_mul(const Cx<R> (&u)[9], const Cx<R> (&h)[6], Cx<R> (&chi)[6]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const Cx<R> u0 = u[3 * a], u1 = u[3 * a + 1], u2 = u[3 * a + 2];
      const Cx<R> h0 = h[3 * sp], h1 = h[3 * sp + 1], h2 = h[3 * sp + 2];
      R re = u0.re * h0.re;
      re = madd(-u0.im, h0.im, re);
      re = madd(u1.re, h1.re, re);
      re = madd(-u1.im, h1.im, re);
      re = madd(u2.re, h2.re, re);
      re = madd(-u2.im, h2.im, re);
      R im = u0.re * h0.im;
      im = madd(u0.im, h0.re, im);
      im = madd(u1.re, h1.im, im);
      im = madd(u1.im, h1.re, im);
      im = madd(u2.re, h2.im, im);
      im = madd(u2.im, h2.re, im);
      chi[3 * sp + a] = cx<R>(re, im);
    }
  }
}

// p = t + U h (the product accumulated onto t: fused multiply-adds only). p may be t itself: each
// output entry reads only its own entry of t.
template <typename R>
__device__ __forceinline__ void su3_mul_add(const Cx<R> (&u)[9], const Cx<R> (&h)[6], const Cx<R> (&t)[6],
                                            Cx<R> (&p)[6]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const Cx<R> u0 = u[3 * a], u1 = u[3 * a + 1], u2 = u[3 * a + 2];
      const Cx<R> h0 = h[3 * sp], h1 = h[3 * sp + 1], h2 = h[3 * sp + 2];
      R re = madd(u0.re, h0.re, t[3 * sp + a].re);
      re = madd(-u0.im, h0.im, re);
      re = madd(u1.re, h1.re, re);
      re = madd(-u1.im, h1.im, re);
      re = madd(u2.re, h2.re, re);
      re = madd(-u2.im, h2.im, re);
      R im = madd(u0.re, h0.im, t[3 * sp + a].im);
      im = madd(u0.im, h0.re, im);
      im = madd(u1.re, h1.im, im);
      im = madd(u1.im, h1.re, im);
      im = madd(u2.re, h2.im, im);
      im = madd(u2.im, h2.re, im);
      p[3 * sp + a] = cx<R>(re, im);
    }
  }
}

// p = t + U^dag h (the product accumulated onto t: fused multiply-adds only; p may be t itself)
template <typename R>
__device__ __forceinline__ void su3_dag_mul_add(const Cx<R> (&u)[9], const Cx<R> (&h)[6], const Cx<R> (&t)[6],
                                                Cx<R> (&p)[6]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const Cx<R> u0 = u[a], u1 = u[3 + a], u2 = u[6 + a];
      const Cx<R> h0 = h[3 * sp], h1 = h[3 * sp + 1], h2 = h[3 * sp + 2];
      R re = madd(u0.re, h0.re, t[3 * sp + a].re);
      re = madd(u0.im, h0.im, re);
      re = madd(u1.re, h1.re, re);
      re = madd(u1.im, h1.im, re);
      re = madd(u2.re, h2.re, re);
      re = madd(u2.im, h2.im, re);
      R im = madd(u0.re, h0.im, t[3 * sp + a].im);
      im = madd(-u0.im, h0.re, im);
      im = madd(u1.re, h1.im, im);
      im = madd(-u1.im, h1.re, im);
      im = madd(u2.re, h2.im, im);
      im = madd(-u2.im, h2.re, im);
      p[3 * sp + a] = cx<R>(re, im);
    }
  }
}

// chi = U^dag h: chi_a = sum_b conj(U_ba) h_b
template <typename R>
__device__ __forceinline__ void su3_dag_mul(const Cx<R> (&u)[9], const Cx<R> (&h)[6], Cx<R> (&chi)[6]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const Cx<R> u0 = u[a], u1 = u[3 + a], u2 = u[6 + a];
      const Cx<R> h0 = h[3 * sp], h1 = h[3 * sp + 1], h2 = h[3 * sp + 2];
      R re = u0.re * h0.re;
      re = madd(u0.im, h0.im, re);
      re = madd(u1.re, h1.re, re);
      re = madd(u1.im, h1.im, re);
      re = madd(u2.re, h2.re, re);
      re = madd(u2.im, h2.im, re);
      R im = u0.re * h0.im;
      im = madd(-u0.im, h0.re, im);
      im = madd(u1.re, h1.im, im);
      im = madd(-u1.im, h1.re, im);
      im = madd(u2.re, h2.im, im);
      im = madd(-u2.im, h2.re, im);
      chi[3 * sp + a] = cx<R>(re, im);
    }
  }
}

// ---------------------------------------------------------------- packed FP32 SU(3) products
//
// For FP32 the two spins of a half-spinor share every link entry, so each colour row's real parts
// (spin 0, spin 1) and imaginary parts accumulate as packed pairs (fma.rn.f32x2, the link entry
// broadcast to both halves): 36 packed instructions per product instead of 72 scalar ones, on the
// same FP32 pipe. Each half performs the scalar form's operations in the scalar form's order, so
// the results are the same bits. Used where instruction issue limits the kernel (the multi-RHS
// dslash, su3_mul_m / su3_dag_mul_m below); the single-RHS kernels are bound by load latency and
// measured slower with it (pair registers lengthen their live ranges: FP32 18r at 32^4 103 -> 117
// us), so they keep the scalar form.

typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
  f32x2 d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void unpk2(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 bc2(float x) { return pk2(x, x); }
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// The spin pairs (h[b], h[3 + b]) of a half-spinor: real parts and imaginary parts.
__device__ __forceinline__ void spin_pairs(const Cx<float> (&h)[6], f32x2 (&hr)[3], f32x2 (&hi)[3]) {
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    hr[b] = pk2(h[b].re, h[3 + b].re);
    hi[b] = pk2(h[b].im, h[3 + b].im);
  }
}

__device__ __forceinline__ void su3_mul_x2(const Cx<float> (&u)[9], const Cx<float> (&h)[6], Cx<float> (&chi)[6]) {
  f32x2 hr[3], hi[3];
  spin_pairs(h, hr, hi);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const Cx<float> u0 = u[3 * a], u1 = u[3 * a + 1], u2 = u[3 * a + 2];
    f32x2 re = mul2(bc2(u0.re), hr[0]);
    re = fma2(bc2(-u0.im), hi[0], re);
    re = fma2(bc2(u1.re), hr[1], re);
    re = fma2(bc2(-u1.im), hi[1], re);
    re = fma2(bc2(u2.re), hr[2], re);
    re = fma2(bc2(-u2.im), hi[2], re);
    f32x2 im = mul2(bc2(u0.re), hi[0]);
    im = fma2(bc2(u0.im), hr[0], im);
    im = fma2(bc2(u1.re), hi[1], im);
    im = fma2(bc2(u1.im), hr[1], im);
    im = fma2(bc2(u2.re), hi[2], im);
    im = fma2(bc2(u2.im), hr[2], im);
    unpk2(re, chi[a].re, chi[3 + a].re);
    unpk2(im, chi[a].im, chi[3 + a].im);
  }
}

__device__ __forceinline__ void su3_dag_mul_x2(const Cx<float> (&u)[9], const Cx<float> (&h)[6],
                                               Cx<float> (&chi)[6]) {
  f32x2 hr[3], hi[3];
  spin_pairs(h, hr, hi);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const Cx<float> u0 = u[a], u1 = u[3 + a], u2 = u[6 + a];
    f32x2 re = mul2(bc2(u0.re), hr[0]);
    re = fma2(bc2(u0.im), hi[0], re);
    re = fma2(bc2(u1.re), hr[1], re);
    re = fma2(bc2(u1.im), hi[1], re);
    re = fma2(bc2(u2.re), hr[2], re);
    re = fma2(bc2(u2.im), hi[2], re);
    f32x2 im = mul2(bc2(u0.re), hi[0]);
    im = fma2(bc2(-u0.im), hr[0], im);
    im = fma2(bc2(u1.re), hi[1], im);
    im = fma2(bc2(-u1.im), hr[1], im);
    im = fma2(bc2(u2.re), hi[2], im);
    im = fma2(bc2(-u2.im), hr[2], im);
    unpk2(re, chi[a].re, chi[3 + a].re);
    unpk2(im, chi[a].im, chi[3 + a].im);
  }
}

// The issue-bound kernels' SU(3) products: packed pairs for FP32, the scalar form otherwise.
template <typename R>
__device__ __forceinline__ void su3_mul_m(const Cx<R> (&u)[9], const Cx<R> (&h)[6], Cx<R> (&chi)[6]) {
  su3_mul(u, h, chi);
}
__device__ __forceinline__ void su3_mul_m(const Cx<float> (&u)[9], const Cx<float> (&h)[6], Cx<float> (&chi)[6]) {
  su3_mul_x2(u, h, chi);
}
template <typename R>
__device__ __forceinline__ void su3_dag_mul_m(const Cx<R> (&u)[9], const Cx<R> (&h)[6], Cx<R> (&chi)[6]) {
  su3_dag_mul(u, h, chi);
}
__device__ __forceinline__ void su3_dag_mul_m(const Cx<float> (&u)[9], const Cx<float> (&h)[6],
                                              Cx<float> (&chi)[6]) {
  su3_dag_mul_x2(u, h, chi);
}

// ---------------------------------------------------------------- deterministic grid reductions
//
// Every block reduces its threads' values with a fixed shuffle tree, stores one partial per block,
// and takes a ticket. The block that draws the last ticket (ticket % gridDim == gridDim - 1) sums
// the partials in a fixed order and publishes the result: the same grid always gives the same
// bits, whatever order the blocks ran in. No block waits for another, so nothing can hang.

struct OpSum {
  static __device__ __forceinline__ double identity() { return 0.0; }
  static __device__ __forceinline__ double apply(double a, double b) { return a + b; }
};

struct OpMax {
  static __device__ __forceinline__ double identity() { return 0.0; }  // used for non-negative values
  static __device__ __forceinline__ double apply(double a, double b) { return fmax(a, b); }
};

template <typename Op, int N>
__device__ __forceinline__ void block_reduce(double (&v)[N], double* smem /* [N][32] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] = Op::apply(v[i], __shfl_down_sync(0xffffffffu, v[i], off));
  }
  __syncthreads();  // smem may still be read by a previous reduction in this kernel
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) smem[i * 32 + wid] = v[i];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double t = lane < nw ? smem[i * 32 + lane] : Op::identity();
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t = Op::apply(t, __shfl_down_sync(0xffffffffu, t, off));
      v[i] = t;  // valid in thread 0
    }
  }
}

// Reduce v over the whole grid. Must be reached by every thread of every block.
// Returns true in every thread of the single block that finished last; in that block's thread 0,
// total[] holds the grid-wide result. partials must hold N * gridDim.x doubles.
template <typename Op, int N>
__device__ __forceinline__ bool grid_reduce(double (&v)[N], double* partials, unsigned* ticket,
                                            double (&total)[N]) {
  __shared__ double smem[N * 32];
  __shared__ int is_last;
  block_reduce<Op, N>(v, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) partials[(size_t)i * gridDim.x + blockIdx.x] = v[i];
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    is_last = (t % gridDim.x) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  // The last block sums the partials in a fixed order: eight independent loads per step (so the
  // L2 latency is paid once per eight partials, not once per partial), combined as a fixed tree.
  double w[N];
  const int G = (int)gridDim.x, S = (int)blockDim.x;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const double* p = partials + (size_t)i * G;
    w[i] = Op::identity();
    int b = threadIdx.x;
    for (; b + 7 * S < G; b += 8 * S) {
      double x[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = __ldcg(p + b + k * S);
      const double lo = Op::apply(Op::apply(x[0], x[1]), Op::apply(x[2], x[3]));
      const double hi = Op::apply(Op::apply(x[4], x[5]), Op::apply(x[6], x[7]));
      w[i] = Op::apply(w[i], Op::apply(lo, hi));
    }
    for (; b < G; b += S) w[i] = Op::apply(w[i], __ldcg(p + b));
  }
  block_reduce<Op, N>(w, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) total[i] = w[i];
    atomicExch(ticket, 0u);
  }
  return true;
}

__device__ __forceinline__ double norm2_site(const Cx<dfloat> (&v)[12]) {
  float a = 0.f;  // the norm steers the solver only: the hi parts suffice
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    a = fmaf(v[c].re.hi, v[c].re.hi, a);
    a = fmaf(v[c].im.hi, v[c].im.hi, a);
  }
  return (double)a;
}

template <typename R>
__device__ __forceinline__ double norm2_site(const Cx<R> (&v)[12]) {
  R a = 0;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    a = madd(v[c].re, v[c].re, a);
    a = madd(v[c].im, v[c].im, a);
  }
  return (double)a;
}

}  // namespace wdk
