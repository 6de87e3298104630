// Seeded gauge-field and source generation on the device (counter-based, reproducible on a CPU).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
// 1, 2, 3", SC11), key = the 64-bit seed, counter = (object index low, object index high, stream,
// draw). Uniforms u = (x + 1/2) 2^-32, Gaussians by Box-Muller: r = sqrt(-2 ln u1),
// (r cos 2 pi u2, r sin 2 pi u2). A link takes 18 Gaussians (Re, Im of the 9 entries of M, in
// row-major order), i.e. 9 Box-Muller pairs from 5 Philox blocks; a site's source takes 24.
//
// Links: H = (M + M^dag)/2 - tr/3, U = exp(i eps H) by the Cayley-Hamilton closed form for a
// traceless Hermitian 3x3 matrix (Morningstar and Peardon, Phys. Rev. D 69 (2004) 054501, Eqs.
// (21)-(34)), then re-unitarised to SU(3) (Gram-Schmidt on rows 0, 1; row 2 = conj(row0 x row1)).
// The CPU generator in synthetic/ uses the same random stream but an eigen-decomposition for the
// exponential, so the two agree to rounding.
#include <cstring>

#include "wd_device.cuh"
#include "wd_internal.h"

namespace wdk {

struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
    const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
    U4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
  }
  return c;
}

__device__ __forceinline__ double u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

// n Gaussians (n even, <= 24) for object `idx` on `stream`
template <int NG>
__device__ __forceinline__ void gaussians(uint64_t seed, uint64_t idx, uint32_t stream, double (&g)[NG]) {
  constexpr int NU = NG;  // one uniform per Gaussian (pairs)
  uint32_t u[(NU + 3) / 4 * 4];
#pragma unroll
  for (int j = 0; j < (NU + 3) / 4; ++j) {
    U4 c;
    c.x = (uint32_t)idx;
    c.y = (uint32_t)(idx >> 32);
    c.z = stream;
    c.w = (uint32_t)j;
    const U4 o = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    u[4 * j] = o.x;
    u[4 * j + 1] = o.y;
    u[4 * j + 2] = o.z;
    u[4 * j + 3] = o.w;
  }
#pragma unroll
  for (int k = 0; k < NG / 2; ++k) {
    const double r = sqrt(-2.0 * log(u01(u[2 * k])));
    double sn, cs;
    sincospi(2.0 * u01(u[2 * k + 1]), &sn, &cs);
    g[2 * k] = r * cs;
    g[2 * k + 1] = r * sn;
  }
}

// exp(iQ) for traceless Hermitian Q (Cayley-Hamilton form): exp(iQ) = f0 + f1 Q + f2 Q^2
__device__ void expiq(const Cx<double> (&Q)[9], Cx<double> (&E)[9]) {
  Cx<double> Q2[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Cx<double> s = cx(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const Cx<double> t = cmul(Q[3 * a + k], Q[3 * k + b]);
        s.re += t.re;
        s.im += t.im;
      }
      Q2[3 * a + b] = s;
    }
  // c0 = det Q = tr(Q^3)/3 (real), c1 = tr(Q^2)/2 (>= 0)
  double c1 = 0.5 * (Q2[0].re + Q2[4].re + Q2[8].re);
  double c0 = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) c0 += cmul(Q[3 * a + k], Q2[3 * k + a]).re;
  c0 /= 3.0;
  Cx<double> f0, f1, f2;
  if (c1 < 1e-30) {  // Q = 0 (up to rounding): exp = 1 + iQ - Q^2/2
    f0 = cx(1.0, 0.0);
    f1 = cx(0.0, 1.0);
    f2 = cx(-0.5, 0.0);
  } else {
    const bool neg = c0 < 0.0;
    const double ac0 = fabs(c0);
    const double c0max = 2.0 * pow(c1 / 3.0, 1.5);
    double ratio = ac0 / c0max;
    ratio = ratio > 1.0 ? 1.0 : ratio;
    const double theta = acos(ratio);
    const double u = sqrt(c1 / 3.0) * cos(theta / 3.0);
    const double w = sqrt(c1) * sin(theta / 3.0);
    const double w2 = w * w;
    const double xi0 = fabs(w) < 0.05 ? 1.0 - w2 / 6.0 * (1.0 - w2 / 20.0 * (1.0 - w2 / 42.0)) : sin(w) / w;
    const double cw = cos(w);
    double s2u, c2u, su, cu;
    sincos(2.0 * u, &s2u, &c2u);
    sincos(u, &su, &cu);
    const Cx<double> e2iu = cx(c2u, s2u), emiu = cx(cu, -su);
    const double uu = u * u;
    // h0 = (u^2 - w^2) e^{2iu} + e^{-iu} (8 u^2 cos w + 2 i u (3 u^2 + w^2) xi0)
    Cx<double> h0 = cx((uu - w2) * e2iu.re, (uu - w2) * e2iu.im);
    Cx<double> t = cmul(emiu, cx(8.0 * uu * cw, 2.0 * u * (3.0 * uu + w2) * xi0));
    h0.re += t.re;
    h0.im += t.im;
    // h1 = 2u e^{2iu} - e^{-iu} (2u cos w - i (3u^2 - w^2) xi0)
    Cx<double> h1 = cx(2.0 * u * e2iu.re, 2.0 * u * e2iu.im);
    t = cmul(emiu, cx(2.0 * u * cw, -(3.0 * uu - w2) * xi0));
    h1.re -= t.re;
    h1.im -= t.im;
    // h2 = e^{2iu} - e^{-iu} (cos w + 3 i u xi0)
    Cx<double> h2 = e2iu;
    t = cmul(emiu, cx(cw, 3.0 * u * xi0));
    h2.re -= t.re;
    h2.im -= t.im;
    const double den = 9.0 * uu - w2;
    f0 = cx(h0.re / den, h0.im / den);
    f1 = cx(h1.re / den, h1.im / den);
    f2 = cx(h2.re / den, h2.im / den);
    if (neg) {  // f_j(-c0) = (-1)^j conj(f_j(c0))
      f0 = cx(f0.re, -f0.im);
      f1 = cx(-f1.re, f1.im);
      f2 = cx(f2.re, -f2.im);
    }
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const Cx<double> a = cmul(f1, Q[i]), b = cmul(f2, Q2[i]);
    E[i] = cx(a.re + b.re, a.im + b.im);
  }
  E[0].re += f0.re;
  E[0].im += f0.im;
  E[4].re += f0.re;
  E[4].im += f0.im;
  E[8].re += f0.re;
  E[8].im += f0.im;
}

__device__ void reunitarise(Cx<double> (&u)[9]) {
  double n0 = 0;
#pragma unroll
  for (int b = 0; b < 3; ++b) n0 += u[b].re * u[b].re + u[b].im * u[b].im;
  const double i0 = 1.0 / sqrt(n0);
#pragma unroll
  for (int b = 0; b < 3; ++b) u[b] = cx(u[b].re * i0, u[b].im * i0);
  // row1 -= <row0, row1> row0
  Cx<double> d = cx(0.0, 0.0);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    d.re += u[b].re * u[3 + b].re + u[b].im * u[3 + b].im;
    d.im += u[b].re * u[3 + b].im - u[b].im * u[3 + b].re;
  }
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const Cx<double> t = cmul(d, u[b]);
    u[3 + b] = cx(u[3 + b].re - t.re, u[3 + b].im - t.im);
  }
  double n1 = 0;
#pragma unroll
  for (int b = 0; b < 3; ++b) n1 += u[3 + b].re * u[3 + b].re + u[3 + b].im * u[3 + b].im;
  const double i1 = 1.0 / sqrt(n1);
#pragma unroll
  for (int b = 0; b < 3; ++b) u[3 + b] = cx(u[3 + b].re * i1, u[3 + b].im * i1);
  reconstruct_row2(u);
}

// One thread per link i = 4 s + mu: generate, write the device layouts (and the canonical copy).
__global__ void gen_gauge_kernel(int V, GeomH eo, int use_eo, double eps, uint64_t seed, double2* __restrict__ g64,
                                 float2* __restrict__ g32, float4* __restrict__ g32c, double2* __restrict__ canon,
                                 float2* __restrict__ gdf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * V) return;
  const int mu = i & 3;
  int s = i >> 2;  // canonical site; storage site below
  if (use_eo) {
    int r = s;
    const int x = r % eo.L[0];
    r /= eo.L[0];
    const int y = r % eo.L[1];
    r /= eo.L[1];
    const int z = r % eo.L[2];
    const int t = r / eo.L[2];
    s = ((x + y + z + t) & 1) * (V >> 1) + (x >> 1) + (eo.L[0] >> 1) * (y + eo.L[1] * (z + eo.L[2] * t));
  }
  double g[18];
  gaussians<18>(seed, (uint64_t)i, 0u, g);
  Cx<double> M[9], Q[9], U[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) M[k] = cx(g[k], g[9 + k]);
  // Q = eps ((M + M^dag)/2 - tr/3)
  const double tr = (M[0].re + M[4].re + M[8].re) / 3.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const Cx<double> x = M[3 * a + b], y = M[3 * b + a];
      double re = 0.5 * (x.re + y.re), im = 0.5 * (x.im - y.im);
      if (a == b) re -= tr;
      Q[3 * a + b] = cx(eps * re, eps * im);
    }
  expiq(Q, U);
  reunitarise(U);
  if (canon) {
#pragma unroll
    for (int k = 0; k < 9; ++k) canon[(size_t)i * 9 + k] = make_double2(U[k].re, U[k].im);
  }
  if (g64) {
#pragma unroll
    for (int k = 0; k < 9; ++k) g64[((size_t)mu * 9 + k) * V + s] = make_double2(U[k].re, U[k].im);
  }
  if (g32) {
#pragma unroll
    for (int k = 0; k < 9; ++k) g32[((size_t)mu * 9 + k) * V + s] = make_float2((float)U[k].re, (float)U[k].im);
  }
  if (gdf) {  // double-float copy: hi [4][9][V], lo [4][9][V]
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float hr = __double2float_rn(U[k].re), hm = __double2float_rn(U[k].im);
      gdf[((size_t)mu * 9 + k) * V + s] = make_float2(hr, hm);
      gdf[((size_t)36 + mu * 9 + k) * V + s] =
          make_float2(__double2float_rn(U[k].re - (double)hr), __double2float_rn(U[k].im - (double)hm));
    }
  }
  if (g32c) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
      g32c[((size_t)mu * 3 + j) * V + s] =
          make_float4((float)U[2 * j].re, (float)U[2 * j].im, (float)U[2 * j + 1].re, (float)U[2 * j + 1].im);
  }
}

// One thread per site: 24 Gaussians -> 12 complex components (Re of all 12 first, then Im).
__global__ void gen_source_kernel(int V, uint64_t seed, double2* __restrict__ canon) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  double g[24];
  gaussians<24>(seed, (uint64_t)s, 1u, g);
#pragma unroll
  for (int c = 0; c < 12; ++c) canon[(size_t)s * 12 + c] = make_double2(g[c], g[12 + c]);
}

cudaError_t launch_gen_gauge(int V, const GeomH* eo, double eps, unsigned long long seed, void* g64, void* g32,
                             int c12, double* canon, void* gdf, cudaStream_t st) {
  const int block = 128;
  const int grid = (4 * V + block - 1) / block;
  GeomH g;
  memset(&g, 0, sizeof(g));
  if (eo) g = *eo;
  gen_gauge_kernel<<<grid, block, 0, st>>>(V, g, eo != nullptr, eps, (uint64_t)seed, reinterpret_cast<double2*>(g64),
                                           c12 ? nullptr : reinterpret_cast<float2*>(g32),
                                           c12 ? reinterpret_cast<float4*>(g32) : nullptr,
                                           reinterpret_cast<double2*>(canon), reinterpret_cast<float2*>(gdf));
  return cudaGetLastError();
}

cudaError_t launch_gen_source(int V, unsigned long long seed, double* canon, cudaStream_t st) {
  const int block = 128;
  gen_source_kernel<<<(V + block - 1) / block, block, 0, st>>>(V, (uint64_t)seed, reinterpret_cast<double2*>(canon));
  return cudaGetLastError();
}

}  // namespace wdk
