// Multi right-hand-side dslash and CG kernels.
//
// N right-hand sides share one operator. Their fields are stored as [unit][V][N] (unit = the
// 16-byte word of the single-RHS layout), so the N values of one site and unit are contiguous.
// Threads are mapped to (site, rhs) with the K right-hand sides of a group in consecutive threads:
// those threads read the same link address in the same instruction, which the memory system
// serves with one transaction, so each link is fetched once per site and group of K (instead of
// once per right-hand side). The launch shape (K, sites per block) is chosen by the autotuner in
// wd_api.cu. All loops over sites are grid-stride with a fixed grid, and every per-RHS reduction
// is deterministic (fixed block and grid orders).
#include <cstring>

#include "wd_device.cuh"
#include "wd_internal.h"

namespace wdk {

template <int SP>
struct MSpinor;

template <>
struct MSpinor<P64> {
  double2* p;
  typedef double real;
};
template <>
struct MSpinor<P32> {
  float4* p;
  typedef float real;
};
template <>
struct MSpinor<P16> {
  uint4* p;
  float* norm;  // [V][N]
  typedef float real;
};

// double-float: hi float4 [6][V][N], then lo float4 [6][V][N]
template <>
struct MSpinor<PDF> {
  float4* hi;
  float4* lo;
  typedef dfloat real;
};

__device__ __forceinline__ void mload(const MSpinor<PDF>& f, int s, int r, int V, int N, Cx<dfloat> (&v)[12]) {
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const size_t i = ((size_t)j * V + s) * N + r;
    const float4 h = __ldg(f.hi + i), l = __ldg(f.lo + i);
    v[2 * j] = cx(dfloat(h.x, l.x), dfloat(h.y, l.y));
    v[2 * j + 1] = cx(dfloat(h.z, l.z), dfloat(h.w, l.w));
  }
}

__device__ __forceinline__ void mstore(const MSpinor<PDF>& f, int s, int r, int V, int N, const Cx<dfloat> (&v)[12]) {
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const size_t i = ((size_t)j * V + s) * N + r;
    f.hi[i] = make_float4(v[2 * j].re.hi, v[2 * j].im.hi, v[2 * j + 1].re.hi, v[2 * j + 1].im.hi);
    f.lo[i] = make_float4(v[2 * j].re.lo, v[2 * j].im.lo, v[2 * j + 1].re.lo, v[2 * j + 1].im.lo);
  }
}

__device__ __forceinline__ void mload(const MSpinor<P64>& f, int s, int r, int V, int N, Cx<double> (&v)[12]) {
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const double2 d = __ldg(f.p + ((size_t)c * V + s) * N + r);
    v[c] = cx(d.x, d.y);
  }
}
__device__ __forceinline__ void mload(const MSpinor<P32>& f, int s, int r, int V, int N, Cx<float> (&v)[12]) {
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float4 d = __ldg(f.p + ((size_t)j * V + s) * N + r);
    v[2 * j] = cx(d.x, d.y);
    v[2 * j + 1] = cx(d.z, d.w);
  }
}
__device__ __forceinline__ void mload(const MSpinor<P16>& f, int s, int r, int V, int N, Cx<float> (&v)[12]) {
  const float nrm = __ldg(f.norm + (size_t)s * N + r);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const uint4 d = __ldg(f.p + ((size_t)j * V + s) * N + r);
    const uint32_t w[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __half2 h = *reinterpret_cast<const __half2*>(&w[k]);
      const float2 fl = __half22float2(h);
      v[4 * j + k] = cx(fl.x * nrm, fl.y * nrm);
    }
  }
}

// Neighbour spinor of a hop, projected (spin_project<MU, S>), returning the hop's reconstruction
// factor (FP16: the per-site norm is folded into the factor instead of h, and the lower spins enter
// the projection through mixed-precision FMAs, as in the single right-hand-side kernel).
template <int MU, int S, typename Ref, typename R>
__device__ __forceinline__ R mload_project_hop(const Ref& f, int s, int r, int V, int N, Cx<R> (&h)[6], R k) {
  Cx<R> psi[12];
  mload(f, s, r, V, N, psi);
  spin_project<MU, S>(psi, h);
  return k;
}

template <int MU, int S>
__device__ __forceinline__ float mload_project_hop(const MSpinor<P16>& f, int s, int r, int V, int N,
                                                   Cx<float> (&h)[6], float k) {
  const float nrm = __ldg(f.norm + (size_t)s * N + r);
  uint32_t w[12];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const uint4 d = __ldg(f.p + ((size_t)j * V + s) * N + r);
    w[4 * j] = d.x;
    w[4 * j + 1] = d.y;
    w[4 * j + 2] = d.z;
    w[4 * j + 3] = d.w;
  }
  spin_project_f16<MU, S>(w, h);
  return k * nrm;
}

__device__ __forceinline__ void mstore(const MSpinor<P64>& f, int s, int r, int V, int N, const Cx<double> (&v)[12]) {
#pragma unroll
  for (int c = 0; c < 12; ++c) f.p[((size_t)c * V + s) * N + r] = make_double2(v[c].re, v[c].im);
}
__device__ __forceinline__ void mstore(const MSpinor<P32>& f, int s, int r, int V, int N, const Cx<float> (&v)[12]) {
#pragma unroll
  for (int j = 0; j < 6; ++j)
    f.p[((size_t)j * V + s) * N + r] = make_float4(v[2 * j].re, v[2 * j].im, v[2 * j + 1].re, v[2 * j + 1].im);
}
__device__ __forceinline__ void mstore(const MSpinor<P16>& f, int s, int r, int V, int N, const Cx<float> (&v)[12]) {
  float m = 0.f;
#pragma unroll
  for (int c = 0; c < 12; ++c) m = fmaxf(m, fmaxf(fabsf(v[c].re), fabsf(v[c].im)));
  const float inv = m > 0.f ? 1.0f / m : 0.f;
  f.norm[(size_t)s * N + r] = m;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __half2 h = __floats2half2_rn(v[4 * j + k].re * inv, v[4 * j + k].im * inv);
      w[k] = *reinterpret_cast<uint32_t*>(&h);
    }
    f.p[((size_t)j * V + s) * N + r] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <int SP>
static MSpinor<SP> mview(FieldPtr f);

// double-float multi-RHS fields need V and N to find the lo half
static MSpinor<PDF> mview_df(FieldPtr f, int V, int N) {
  MSpinor<PDF> r;
  r.hi = reinterpret_cast<float4*>(f.p);
  r.lo = reinterpret_cast<float4*>(f.p) + (size_t)6 * V * N;
  return r;
}
template <>
MSpinor<P64> mview<P64>(FieldPtr f) {
  MSpinor<P64> r;
  r.p = reinterpret_cast<double2*>(f.p);
  return r;
}
template <>
MSpinor<P32> mview<P32>(FieldPtr f) {
  MSpinor<P32> r;
  r.p = reinterpret_cast<float4*>(f.p);
  return r;
}
template <>
MSpinor<P16> mview<P16>(FieldPtr f) {
  MSpinor<P16> r;
  r.p = reinterpret_cast<uint4*>(f.p);
  r.norm = f.norm;
  return r;
}

template <int SP>
struct MReal {
  typedef float type;
};
template <>
struct MReal<P64> {
  typedef double type;
};
template <>
struct MReal<PDF> {
  typedef dfloat type;
};

// ---------------------------------------------------------------- per-RHS deterministic reduction
//
// Thread (sl, rl) of a block holds one value for right-hand side rl of its group (blockIdx.y).
// Two levels, each in a fixed order, so the result does not depend on block timing:
//  1. every block sums its values per rl into a block partial; the block that draws the last
//     ticket of its run of kRedGroup consecutive blocks sums that run's partials per rl;
//  2. the run that finishes last sums the run partials per rl, spread over the whole block.
// Either level loads its operands together, so the tail of the reduction costs two L2 round
// trips instead of one per block partial. Returns true in the finishing block; out[rl] (in shared
// memory) then holds the group's totals for rl < K, valid after the function returns (it ends
// with a barrier). Layout of `partials` (fixed offsets): block partials [r][gridDim.x], run
// partials [kMaxRhs][kMaxMultiRuns], run tickets [kMaxRhs][kMaxMultiRuns] (zero between launches).
//
// mreduce_sh takes the block's values already in sh[0 .. nv) (value i belongs to right-hand side
// i % K; nv = K * sites per block, which may exceed blockDim.x when a thread holds several
// right-hand sides); the block needs at least K threads.
__device__ bool mreduce_sh(int nv, int K, double* partials, unsigned* tickets, double* sh, double* out) {
  const int t = threadIdx.x, nt = blockDim.x, G = gridDim.x, y = blockIdx.y, b = blockIdx.x;
  double* p1 = partials;
  double* p2 = partials + (size_t)kMaxRhs * kMaxMultiGrid;
  unsigned* t1 = reinterpret_cast<unsigned*>(p2 + (size_t)kMaxRhs * kMaxMultiRuns);
  const int nruns = (G + kRedGroup - 1) / kRedGroup, run = b / kRedGroup;
  const int rsize = min(kRedGroup, G - run * kRedGroup);
  __shared__ int flag;
  if (t < K) {
    double a = 0.0;
    for (int i = t; i < nv; i += K) a += sh[i];
    p1[(size_t)(y * K + t) * G + b] = a;
    __threadfence();  // each writer publishes its partial before the ticket is taken
  }
  __syncthreads();
  if (t == 0) {
    __threadfence();
    flag = atomicAdd(&t1[y * kMaxMultiRuns + run], 1u) == (unsigned)(rsize - 1);
  }
  __syncthreads();
  if (!flag) return false;
  __threadfence();
  // level 1: the partials of this run, eight loads in flight per step, summed in order
  if (t < K) {
    const double* q = p1 + (size_t)(y * K + t) * G + run * kRedGroup;
    double a = 0.0;
    for (int i0 = 0; i0 < rsize; i0 += 8) {
      double x[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = i0 + k < rsize ? __ldcg(q + i0 + k) : 0.0;
      a += ((x[0] + x[1]) + (x[2] + x[3])) + ((x[4] + x[5]) + (x[6] + x[7]));
    }
    p2[(size_t)(y * K + t) * kMaxMultiRuns + run] = a;
    __threadfence();
  }
  __syncthreads();
  if (t == 0) {
    t1[y * kMaxMultiRuns + run] = 0u;  // every block of the run has taken its ticket
    __threadfence();
    flag = atomicAdd(&tickets[y], 1u) == (unsigned)(nruns - 1);
  }
  __syncthreads();
  if (!flag) return false;
  __threadfence();
  // level 2: thread (j, rl) sums runs j, j + J, ... of rl; then rl sums its J values in order
  const int J = nt / K, rl = t % K, j = t / K;
  double a = 0.0;
  if (j < J) {
    const double* q = p2 + (size_t)(y * K + rl) * kMaxMultiRuns;
#pragma unroll 4
    for (int r = j; r < nruns; r += J) a += __ldcg(q + r);
  }
  __syncthreads();
  sh[t] = a;
  __syncthreads();
  if (t < K) {
    double tot = 0.0;
    for (int jj = 0; jj < J; ++jj) tot += sh[jj * K + t];
    out[t] = tot;
  }
  if (t == 0) tickets[y] = 0u;
  __syncthreads();
  return true;
}

__device__ bool mreduce(double v, int K, double* partials, unsigned* tickets, double* sh /* >= blockDim + 2*kMaxRhs */,
                        double* out) {
  sh[threadIdx.x] = v;
  __syncthreads();
  return mreduce_sh(blockDim.x, K, partials, tickets, sh, out);
}

// ---------------------------------------------------------------- multi-RHS dslash

template <int SP, bool C12>
struct MArgs {
  Geom g;
  GaugeRef<typename MReal<SP>::type, C12> u;
  MSpinor<SP> in, out, b;
  typename MReal<SP>::type mkappa;
  const double* kappa_dev;
  int N, K;            // total RHS, RHS per group (blockDim.x = K * sites per block)
  const int* status;   // optional per-RHS status: only RUNNING right-hand sides are computed
  double* partials;
  unsigned* tickets;
  double* result;      // per-RHS ||out||^2 (written for computed right-hand sides only)
};

template <int MU, int SF, int SP, bool C12, typename R>
__device__ __forceinline__ void mhop(const MArgs<SP, C12>& a, R mk, int s, int r, const int (&c)[4], Cx<R> (&acc)[12]) {
  const int V = a.g.V, N = a.N;
  {
    const bool wrap = c[MU] == a.g.L[MU] - 1;
    const int nb = wrap ? s - (a.g.L[MU] - 1) * a.g.stride[MU] : s + a.g.stride[MU];
    Cx<R> h[6], u[9], chi[6];
    const R k = mload_project_hop<MU, SF>(a.in, nb, r, V, N, h, (wrap && a.g.bc[MU] < 0) ? -mk : mk);
    load_link(a.u, MU, s, V, u);
    su3_mul_m(u, h, chi);
    spin_reconstruct<MU, SF>(acc, chi, k);
  }
  {
    const bool wrap = c[MU] == 0;
    const int nb = wrap ? s + (a.g.L[MU] - 1) * a.g.stride[MU] : s - a.g.stride[MU];
    Cx<R> h[6], u[9], chi[6];
    const R k = mload_project_hop<MU, -SF>(a.in, nb, r, V, N, h, (wrap && a.g.bc[MU] < 0) ? -mk : mk);
    load_link(a.u, MU, nb, V, u);
    su3_dag_mul_m(u, h, chi);
    spin_reconstruct<MU, -SF>(acc, chi, k);
  }
}

// 8 hops in a runtime loop (compact code for double-float, see wd_dslash.cu)
template <int SF, int SP, bool C12, typename R>
__device__ __forceinline__ void mhops_rt(const MArgs<SP, C12>& a, R mk, int s, int r, const int (&c)[4],
                                         Cx<R> (&acc)[12]) {
  const int V = a.g.V, N = a.N;
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
    mload(a.in, nb, r, V, N, psi);
    spin_project_rt(mu, S, psi, h);
    load_link(a.u, mu, dir == 0 ? s : nb, V, u);
    if (dir == 0)
      su3_mul_m(u, h, chi);
    else
      su3_dag_mul_m(u, h, chi);
    spin_reconstruct_rt(mu, S, acc, chi, k);
  }
}

// Both hops of direction mu for KT right-hand sides r0 .. r0 + KT - 1 of one site: each link is
// loaded (and, with 12 reals, its third row rebuilt) once and applied to the KT half-spinors, so the
// link's instructions are shared and only the projection, SU(3) product and reconstruction are
// per right-hand side. The per-right-hand-side arithmetic is that of mhop, in the same order.
template <int MU, int SF, int KT, int SP, bool C12, typename R>
__device__ __forceinline__ void mhop_kt(const MArgs<SP, C12>& a, R mk, int s, int r0, const int (&c)[4],
                                        Cx<R> (&acc)[KT][12]) {
  const int V = a.g.V, N = a.N;
  {
    const bool wrap = c[MU] == a.g.L[MU] - 1;
    const int nb = wrap ? s - (a.g.L[MU] - 1) * a.g.stride[MU] : s + a.g.stride[MU];
    const R k0 = (wrap && a.g.bc[MU] < 0) ? -mk : mk;
    Cx<R> u[9];
    load_link(a.u, MU, s, V, u);
#pragma unroll
    for (int j = 0; j < KT; ++j) {
      Cx<R> h[6], chi[6];
      const R k = mload_project_hop<MU, SF>(a.in, nb, r0 + j, V, N, h, k0);
      su3_mul_m(u, h, chi);
      spin_reconstruct<MU, SF>(acc[j], chi, k);
    }
  }
  {
    const bool wrap = c[MU] == 0;
    const int nb = wrap ? s + (a.g.L[MU] - 1) * a.g.stride[MU] : s - a.g.stride[MU];
    const R k0 = (wrap && a.g.bc[MU] < 0) ? -mk : mk;
    Cx<R> u[9];
    load_link(a.u, MU, nb, V, u);
#pragma unroll
    for (int j = 0; j < KT; ++j) {
      Cx<R> h[6], chi[6];
      const R k = mload_project_hop<MU, -SF>(a.in, nb, r0 + j, V, N, h, k0);
      su3_dag_mul_m(u, h, chi);
      spin_reconstruct<MU, -SF>(acc[j], chi, k);
    }
  }
}

template <int SP>
struct MMinBlocks {
  static constexpr int value = SP == P64 ? 2 : (SP == PDF ? 1 : 3);
};

// A thread holding KT = 2 or 4 right-hand sides keeps KT accumulators live. Its blocks have at most
// 256 / KT threads (K * sites per block <= 256): bounds of 3 x 128 and 2 x 64 threads per SM leave up
// to 170 and 255 registers a thread.
template <int KT>
struct MKtBounds {
  static constexpr int threads = 256 / KT;
  static constexpr int blocks = KT == 2 ? 3 : 2;
};

// KT right-hand sides per thread (FP32 / FP16 working precision): thread (sl, tl) of a block takes
// site sl's right-hand sides blockIdx.y * K + tl * KT + j, j < KT; a block is K / KT threads per site
// times sites per block. The norms go through the same per-right-hand-side reduction as with one
// right-hand side per thread (values laid out as if each had its own thread).
template <int SP, bool C12, bool DAG, int EPI, bool NORM, int KT>
__global__ void __launch_bounds__(MKtBounds<KT>::threads, MKtBounds<KT>::blocks)
    dslash_multi_kt_kernel(const MArgs<SP, C12> a) {
  typedef typename MReal<SP>::type R;
  extern __shared__ double msh[];
  const int K = a.K, V = a.g.V, TK = K / KT;
  const int tl = threadIdx.x % TK, sl = threadIdx.x / TK;
  const int spb = blockDim.x / TK;
  const int r0 = blockIdx.y * K + tl * KT;
  bool live[KT];
  bool any = false;
#pragma unroll
  for (int j = 0; j < KT; ++j) {
    live[j] = sl < spb && (a.status == nullptr || a.status[r0 + j] == ST_RUNNING);
    any = any || live[j];
  }
  double n2[KT];
#pragma unroll
  for (int j = 0; j < KT; ++j) n2[j] = 0.0;
  const R mk = a.kappa_dev ? (R)(-*a.kappa_dev) : a.mkappa;
  if (any) {
    for (int s = blockIdx.x * spb + sl; s < V; s += gridDim.x * spb) {
      int c[4];
      int q = s;
      c[0] = q % a.g.L[0];
      q /= a.g.L[0];
      c[1] = q % a.g.L[1];
      q /= a.g.L[1];
      c[2] = q % a.g.L[2];
      c[3] = q / a.g.L[2];
      Cx<R> acc[KT][12];
#pragma unroll
      for (int j = 0; j < KT; ++j) mload(a.in, s, r0 + j, V, a.N, acc[j]);
      constexpr int SF = DAG ? +1 : -1;
      mhop_kt<0, SF, KT>(a, mk, s, r0, c, acc);
      mhop_kt<1, SF, KT>(a, mk, s, r0, c, acc);
      mhop_kt<2, SF, KT>(a, mk, s, r0, c, acc);
      mhop_kt<3, SF, KT>(a, mk, s, r0, c, acc);
#pragma unroll
      for (int j = 0; j < KT; ++j) {
        if (EPI == EPI_RESID) {
          Cx<R> bv[12];
          mload(a.b, s, r0 + j, V, a.N, bv);
#pragma unroll
          for (int i = 0; i < 12; ++i) acc[j][i] = cx<R>(bv[i].re - acc[j][i].re, bv[i].im - acc[j][i].im);
        }
        if (live[j]) {  // converged right-hand sides were computed alongside but are not stored
          mstore(a.out, s, r0 + j, V, a.N, acc[j]);
          if (NORM) n2[j] += norm2_site(acc[j]);
        }
      }
    }
  }
  if (NORM) {
    const int nv = spb * K;
    double* out = msh + nv;
#pragma unroll
    for (int j = 0; j < KT; ++j) msh[sl * K + tl * KT + j] = n2[j];
    __syncthreads();
    if (mreduce_sh(nv, K, a.partials, a.tickets, msh, out) && threadIdx.x < K) {
      const int rr = blockIdx.y * K + threadIdx.x;
      if (a.status == nullptr || a.status[rr] == ST_RUNNING) a.result[rr] = out[threadIdx.x];
    }
  }
}

template <int SP, bool C12, bool DAG, int EPI, bool NORM>
__global__ void __launch_bounds__(256, MMinBlocks<SP>::value) dslash_multi_kernel(const MArgs<SP, C12> a) {
  typedef typename MReal<SP>::type R;
  extern __shared__ double msh[];
  const int K = a.K, V = a.g.V;
  const int rl = threadIdx.x % K, sl = threadIdx.x / K;
  const int spb = blockDim.x / K;
  const int r = blockIdx.y * K + rl;
  const bool live = sl < spb && (a.status == nullptr || a.status[r] == ST_RUNNING);
  double n2 = 0.0;
  const R mk = a.kappa_dev ? (R)(-*a.kappa_dev) : a.mkappa;
  if (live) {
    for (int s = blockIdx.x * spb + sl; s < V; s += gridDim.x * spb) {
      int c[4];
      int q = s;
      c[0] = q % a.g.L[0];
      q /= a.g.L[0];
      c[1] = q % a.g.L[1];
      q /= a.g.L[1];
      c[2] = q % a.g.L[2];
      c[3] = q / a.g.L[2];
      Cx<R> acc[12];
      mload(a.in, s, r, V, a.N, acc);
      constexpr int SF = DAG ? +1 : -1;
      if constexpr (SP == PDF) {
        mhops_rt<SF>(a, mk, s, r, c, acc);
      } else {
        mhop<0, SF>(a, mk, s, r, c, acc);
        mhop<1, SF>(a, mk, s, r, c, acc);
        mhop<2, SF>(a, mk, s, r, c, acc);
        mhop<3, SF>(a, mk, s, r, c, acc);
      }
      if (EPI == EPI_RESID) {
        Cx<R> bv[12];
        mload(a.b, s, r, V, a.N, bv);
#pragma unroll
        for (int i = 0; i < 12; ++i) acc[i] = cx<R>(bv[i].re - acc[i].re, bv[i].im - acc[i].im);
      }
      mstore(a.out, s, r, V, a.N, acc);
      if (NORM) n2 += norm2_site(acc);
    }
  }
  if (NORM) {
    double* out = msh + blockDim.x;
    if (mreduce(n2, K, a.partials, a.tickets, msh, out) && threadIdx.x < K) {
      const int rr = blockIdx.y * K + threadIdx.x;
      if (a.status == nullptr || a.status[rr] == ST_RUNNING) a.result[rr] = out[threadIdx.x];
    }
  }
}

template <int SP, bool C12, bool DAG, int EPI>
static cudaError_t mlaunch_t(const MDslashCall& c, cudaStream_t st) {
  MArgs<SP, C12> a;
  memcpy(&a.g, &c.g, sizeof(Geom));
  a.u.p = reinterpret_cast<decltype(a.u.p)>(c.u.p);
  if constexpr (SP == PDF) {
    a.in = mview_df(c.in, c.g.V, c.nrhs);
    a.out = mview_df(c.out, c.g.V, c.nrhs);
    a.b = mview_df(c.b, c.g.V, c.nrhs);
  } else {
    a.in = mview<SP>(c.in);
    a.out = mview<SP>(c.out);
    a.b = mview<SP>(c.b);
  }
  a.mkappa = (typename MReal<SP>::type)(-c.kappa);
  a.kappa_dev = c.kappa_dev;
  a.N = c.nrhs;
  a.K = c.group;
  a.status = c.status;
  a.partials = c.partials;
  a.tickets = c.tickets;
  a.result = c.result;
  const int spb = c.sites_per_block;
  const int groups = c.nrhs / c.group;
  const int kt = c.rhs_per_thread;
  // One wave of resident blocks over all groups (grid-stride over sites): with more blocks than
  // fit at once, the later ones would start only after the first wave had walked all its sites,
  // and the neighbour spinors shared across the two would be read from DRAM twice.
  auto launch = [&](auto k, int block, size_t smem) -> cudaError_t {
    int gx = resident_blocks(reinterpret_cast<const void*>(k), block) / groups;
    if (gx < 1) gx = 1;
    if (gx > c.grid_x) gx = c.grid_x;
    k<<<dim3(gx, groups), block, smem, st>>>(a);
    return cudaGetLastError();
  };
  if constexpr (SP == P32 || SP == P16) {
    if (kt == 2 || kt == 4) {
      const int block = c.group / kt * spb;
      const size_t smem = sizeof(double) * (c.group * spb + 32);
      if (kt == 2)
        return c.result ? launch(dslash_multi_kt_kernel<SP, C12, DAG, EPI, true, 2>, block, smem)
                        : launch(dslash_multi_kt_kernel<SP, C12, DAG, EPI, false, 2>, block, smem);
      return c.result ? launch(dslash_multi_kt_kernel<SP, C12, DAG, EPI, true, 4>, block, smem)
                      : launch(dslash_multi_kt_kernel<SP, C12, DAG, EPI, false, 4>, block, smem);
    }
  }
  const int block = c.group * spb;
  const size_t smem = sizeof(double) * (block + 32);
  return c.result ? launch(dslash_multi_kernel<SP, C12, DAG, EPI, true>, block, smem)
                  : launch(dslash_multi_kernel<SP, C12, DAG, EPI, false>, block, smem);
}

template <int SP, bool C12>
static cudaError_t mlaunch_p(const MDslashCall& c, cudaStream_t st) {
  if (c.dagger)
    return c.epi == EPI_RESID ? mlaunch_t<SP, C12, true, EPI_RESID>(c, st) : mlaunch_t<SP, C12, true, EPI_PLAIN>(c, st);
  return c.epi == EPI_RESID ? mlaunch_t<SP, C12, false, EPI_RESID>(c, st) : mlaunch_t<SP, C12, false, EPI_PLAIN>(c, st);
}

cudaError_t launch_dslash_multi(const MDslashCall& c, cudaStream_t st) {
  if (c.grid_x < 1 || c.grid_x > kMaxMultiGrid) return cudaErrorInvalidValue;  // reduction workspace bound
  if (c.nrhs < 1 || c.nrhs > kMaxRhs || c.group < 1 || c.nrhs % c.group || c.sites_per_block < 1 ||
      c.group * c.sites_per_block > 256 || c.grid_x < 1)
    return cudaErrorInvalidValue;
  // KT right-hand sides per thread: KT divides K, the block keeps at least K threads (the reduction
  // needs them), and only the FP32 / FP16 working precisions have the blocked kernel
  const int kt = c.rhs_per_thread;
  if (kt != 0 && kt != 1) {
    if ((kt != 2 && kt != 4) || c.group % kt || c.sites_per_block < kt ||
        (c.in.prec != SP32 && c.in.prec != SP16))
      return cudaErrorInvalidValue;
  }
  if (c.in.prec == SPDF) {
    if (c.u.prec != SPDF) return cudaErrorInvalidValue;
    return mlaunch_p<PDF, false>(c, st);
  }
  if (c.in.prec == SP64) {
    if (c.u.prec != SP64) return cudaErrorInvalidValue;
    return mlaunch_p<P64, false>(c, st);
  }
  if (c.u.prec != SP32) return cudaErrorInvalidValue;
  if (c.in.prec == SP32) return c.u.c12 ? mlaunch_p<P32, true>(c, st) : mlaunch_p<P32, false>(c, st);
  if (c.in.prec == SP16) return c.u.c12 ? mlaunch_p<P16, true>(c, st) : mlaunch_p<P16, false>(c, st);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- packing of N fields

// canonical: N fields back to back, each complex128 [V][12]
template <int SP>
__global__ void mpack_kernel(const double2* __restrict__ canon, MSpinor<SP> out, int V, int N, double* partials,
                             unsigned* tickets, double* result) {
  typedef typename MReal<SP>::type R;
  extern __shared__ double msh[];
  const int K = N;
  const int rl = threadIdx.x % K, sl = threadIdx.x / K, spb = blockDim.x / K;
  double n2 = 0.0;
  if (sl < spb) {
    for (int s = blockIdx.x * spb + sl; s < V; s += gridDim.x * spb) {
      Cx<R> v[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        const double2 d = canon[((size_t)rl * V + s) * 12 + c];
        n2 = fma(d.x, d.x, n2);
        n2 = fma(d.y, d.y, n2);
        v[c] = cx<R>((R)d.x, (R)d.y);
      }
      mstore(out, s, rl, V, N, v);
    }
  }
  if (result) {
    double* o = msh + blockDim.x;
    if (mreduce(n2, K, partials, tickets, msh, o) && threadIdx.x < K) result[threadIdx.x] = o[threadIdx.x];
  }
}

template <int SP>
__global__ void munpack_kernel(MSpinor<SP> in, double2* __restrict__ canon, int V, int N) {
  typedef typename MReal<SP>::type R;
  const int K = N;
  const int rl = threadIdx.x % K, sl = threadIdx.x / K, spb = blockDim.x / K;
  if (sl >= spb) return;
  for (int s = blockIdx.x * spb + sl; s < V; s += gridDim.x * spb) {
    Cx<R> v[12];
    mload(in, s, rl, V, N, v);
#pragma unroll
    for (int c = 0; c < 12; ++c) canon[((size_t)rl * V + s) * 12 + c] = make_double2((double)v[c].re, (double)v[c].im);
  }
}

static int mblock(int N) { return N * (256 / N); }

cudaError_t launch_mpack(const double* canon, FieldPtr out, int V, int N, int grid_x, double* partials,
                         unsigned* tickets, double* result, cudaStream_t st) {
  if (grid_x < 1 || grid_x > kMaxMultiGrid) return cudaErrorInvalidValue;  // reduction workspace bound
  const int block = mblock(N);
  const size_t smem = sizeof(double) * (block + 32);
  const double2* c2 = reinterpret_cast<const double2*>(canon);
  switch (out.prec) {
    case SP64: mpack_kernel<P64><<<grid_x, block, smem, st>>>(c2, mview<P64>(out), V, N, partials, tickets, result); break;
    case SP32: mpack_kernel<P32><<<grid_x, block, smem, st>>>(c2, mview<P32>(out), V, N, partials, tickets, result); break;
    case SP16: mpack_kernel<P16><<<grid_x, block, smem, st>>>(c2, mview<P16>(out), V, N, partials, tickets, result); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_munpack(FieldPtr in, double* canon, int V, int N, int grid_x, cudaStream_t st) {
  const int block = mblock(N);
  double2* c2 = reinterpret_cast<double2*>(canon);
  switch (in.prec) {
    case SP64: munpack_kernel<P64><<<grid_x, block, 0, st>>>(mview<P64>(in), c2, V, N); break;
    case SP32: munpack_kernel<P32><<<grid_x, block, 0, st>>>(mview<P32>(in), c2, V, N); break;
    case SP16: munpack_kernel<P16><<<grid_x, block, 0, st>>>(mview<P16>(in), c2, V, N); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- multi-RHS CG steps
//
// Per right-hand side r: status[r] in ST_RUNNING, ST_CONVERGED, ST_MAXIT, ST_BREAKDOWN and
// ST_PENDING (converged in this iteration's r update; its x update is still due).

__global__ void mcg_init_kernel(MCgScalars* sc) {
  const int r = threadIdx.x;
  if (blockIdx.x == 0 && r < sc->nrhs) {
    sc->status[r] = ST_RUNNING;
    sc->need[r] = 0;
  }
  if (blockIdx.x == 0 && r == 0) {
    sc->need_update = 0;
    sc->no_update = 1;
  }
}

__global__ void mcg_check_kernel(MCgScalars* sc, int use_cond, cudaGraphConditionalHandle cond) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int running = 0;
  for (int r = 0; r < sc->nrhs; ++r) {
    int st = ST_RUNNING;
    const double eta2 = sc->eta2[r], rr = sc->rr[r], g = sc->gamma[r];
    if (!isfinite(eta2) || !isfinite(rr) || !isfinite(g))
      st = ST_BREAKDOWN;
    else if (rr <= sc->tol2 * eta2)
      st = ST_CONVERGED;
    else if (sc->iter >= sc->maxit)
      st = ST_MAXIT;
    else if (!(g > 0.0))
      st = ST_BREAKDOWN;
    sc->status[r] = st;
    sc->rr_ref[r] = rr;
    running += st == ST_RUNNING;
  }
  sc->any_running = running;
  if (use_cond) cudaGraphSetConditional(cond, running ? 1u : 0u);
}

// alpha_r = gamma_r / |q_r|^2; r_r -= alpha_r q_r; |r_r|^2 (+ mixed: x_lo += alpha p, update flag)
template <int SPW, int SPX, bool MIXED>
__global__ void mcg_update_r_kernel(MSpinor<SPW> r, MSpinor<SPW> q, MSpinor<SPW> p, MSpinor<SPX> xlo, int V,
                                    MCgScalars* sc, double* partials, int K, int use_cond,
                                    cudaGraphConditionalHandle upd) {
  typedef typename MReal<SPW>::type R;
  typedef typename MReal<SPX>::type RX;
  extern __shared__ double msh[];
  const int N = sc->nrhs;
  const int rl = threadIdx.x % K, sl = threadIdx.x / K, spb = blockDim.x / K;
  const int rh = blockIdx.y * K + rl;
  const bool running = sc->status[rh] == ST_RUNNING;
  const double qq = sc->qq[rh], gamma = sc->gamma[rh];
  const bool ok = running && qq > 0.0 && isfinite(qq) && isfinite(gamma);
  const double alpha = ok ? gamma / qq : 0.0;
  const R a = (R)alpha;
  double n2 = 0.0;
  if (ok && sl < spb) {
    for (int s = blockIdx.x * spb + sl; s < V; s += gridDim.x * spb) {
      Cx<R> rv[12], qv[12];
      mload(r, s, rh, V, N, rv);
      mload(q, s, rh, V, N, qv);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        rv[c].re = fma(-a, qv[c].re, rv[c].re);
        rv[c].im = fma(-a, qv[c].im, rv[c].im);
      }
      mstore(r, s, rh, V, N, rv);
      n2 += norm2_site(rv);
      if (MIXED) {
        Cx<R> pv[12];
        Cx<RX> xv[12];
        mload(p, s, rh, V, N, pv);
        mload(xlo, s, rh, V, N, xv);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          xv[c].re = fma((RX)a, (RX)pv[c].re, xv[c].re);
          xv[c].im = fma((RX)a, (RX)pv[c].im, xv[c].im);
        }
        mstore(xlo, s, rh, V, N, xv);
      }
    }
  }
  double* out = msh + blockDim.x;
  if (mreduce(n2, K, partials, &sc->ticket[TKM_UPD_R], msh, out)) {
    if (threadIdx.x < K) {
      const int rr = blockIdx.y * K + threadIdx.x;
      if (sc->status[rr] == ST_RUNNING) {
        const double q2 = sc->qq[rr], g = sc->gamma[rr];
        const bool good = q2 > 0.0 && isfinite(q2) && isfinite(g) && isfinite(out[threadIdx.x]);
        if (!good) {
          sc->status[rr] = ST_BREAKDOWN;
          sc->need[rr] = 0;
        } else {
          const double v = out[threadIdx.x];
          sc->alpha[rr] = g / q2;
          sc->rr[rr] = v;
          if (MIXED) {
            sc->need[rr] = (v <= sc->delta2 * sc->rr_ref[rr]) || (v <= sc->tol2 * sc->eta2[rr]);
          } else if (v <= sc->tol2 * sc->eta2[rr]) {
            sc->status[rr] = ST_PENDING;
          }
        }
      } else {
        sc->need[rr] = 0;
      }
      __threadfence();
    }
    __syncthreads();
    // the group that finishes last over all groups publishes the any-update flag
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned k = atomicAdd(&sc->ticket[TKM_GROUPS], 1u);
      if ((k % gridDim.y) == gridDim.y - 1) {
        __threadfence();
        int any = 0;
        for (int i = 0; i < N; ++i) any |= *((volatile int*)&sc->need[i]);
        sc->need_update = any;
        sc->no_update = !any;
        atomicExch(&sc->ticket[TKM_GROUPS], 0u);
        if (use_cond) cudaGraphSetConditional(upd, any ? 1u : 0u);
      }
    }
  }
}

// Plain: x += alpha p; p = s + beta p. Mixed: p = s + beta p only (x_lo was updated with r).
// The last group advances the iteration and sets the loop condition.
template <int SPW, bool MIXED>
__global__ void mcg_update_xp_kernel(MSpinor<SPW> x, MSpinor<SPW> p, MSpinor<SPW> sv, int V, MCgScalars* sc,
                                     double* partials, int K, int use_cond, cudaGraphConditionalHandle cond) {
  typedef typename MReal<SPW>::type R;
  extern __shared__ double msh[];
  const int N = sc->nrhs;
  const int rl = threadIdx.x % K, sl = threadIdx.x / K, spb = blockDim.x / K;
  const int rh = blockIdx.y * K + rl;
  const int st0 = sc->status[rh];
  const double gnew = sc->gamma_new[rh], gold = sc->gamma[rh];
  const bool do_x = !MIXED && (st0 == ST_RUNNING || st0 == ST_PENDING);
  const bool do_p = st0 == ST_RUNNING && isfinite(gnew) && gold > 0.0;
  const R a = (R)sc->alpha[rh], b = (R)(do_p ? gnew / gold : 0.0);
  if ((do_x || do_p) && sl < spb) {
    for (int s = blockIdx.x * spb + sl; s < V; s += gridDim.x * spb) {
      Cx<R> pv[12];
      mload(p, s, rh, V, N, pv);
      if (do_x) {
        Cx<R> xv[12];
        mload(x, s, rh, V, N, xv);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          xv[c].re = fma(a, pv[c].re, xv[c].re);
          xv[c].im = fma(a, pv[c].im, xv[c].im);
        }
        mstore(x, s, rh, V, N, xv);
      }
      if (do_p) {
        Cx<R> svv[12];
        mload(sv, s, rh, V, N, svv);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          pv[c].re = fma(b, pv[c].re, svv[c].re);
          pv[c].im = fma(b, pv[c].im, svv[c].im);
        }
        mstore(p, s, rh, V, N, pv);
      }
    }
  }
  double* out = msh + blockDim.x;
  if (mreduce(0.0, K, partials, &sc->ticket[TKM_UPD_XP], msh, out)) {
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned k = atomicAdd(&sc->ticket[TKM_GROUPS2], 1u);
      if ((k % gridDim.y) == gridDim.y - 1) {
        __threadfence();
        sc->iter += 1;
        int running = 0;
        for (int i = 0; i < N; ++i) {
          volatile int* sti = &sc->status[i];
          int st = *sti;
          if (st == ST_RUNNING || st == ST_PENDING) sc->iters[i] = sc->iter;
          if (st == ST_PENDING) st = ST_CONVERGED;
          if (st == ST_RUNNING) {
            const double gn = sc->gamma_new[i], go = sc->gamma[i];
            if (!(isfinite(gn) && go > 0.0)) {
              st = ST_BREAKDOWN;
            } else {
              sc->gamma[i] = gn;
              if (sc->iter >= sc->maxit) st = ST_MAXIT;
            }
          }
          *sti = st;
          running += st == ST_RUNNING;
        }
        sc->any_running = running;
        atomicExch(&sc->ticket[TKM_GROUPS2], 0u);
        if (use_cond) cudaGraphSetConditional(cond, running ? 1u : 0u);
      }
    }
  }
}

// Mixed precision: x_hi += x_lo; x_lo = 0 (all right-hand sides)
__global__ void macc_kernel(MSpinor<P64> xhi, MSpinor<P32> xlo, int V, int N) {
  const int rl = threadIdx.x % N, sl = threadIdx.x / N, spb = blockDim.x / N;
  if (sl >= spb) return;
  for (int s = blockIdx.x * spb + sl; s < V; s += gridDim.x * spb) {
    Cx<double> xh[12];
    Cx<float> xl[12];
    mload(xhi, s, rl, V, N, xh);
    mload(xlo, s, rl, V, N, xl);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      xh[c].re += (double)xl[c].re;
      xh[c].im += (double)xl[c].im;
      xl[c] = cx(0.f, 0.f);
    }
    mstore(xhi, s, rl, V, N, xh);
    mstore(xlo, s, rl, V, N, xl);
  }
}

// Mixed precision: r_lo = r_hi for every right-hand side still running; adopt the FP64 residual.
template <int SPW>
__global__ void mconv_kernel(MSpinor<P64> rhi, MSpinor<SPW> rlo, int V, MCgScalars* sc, int count) {
  const int N = sc->nrhs;
  const int rl = threadIdx.x % N, sl = threadIdx.x / N, spb = blockDim.x / N;
  if (sl < spb && sc->status[rl] == ST_RUNNING) {
    for (int s = blockIdx.x * spb + sl; s < V; s += gridDim.x * spb) {
      Cx<double> h[12];
      Cx<float> l[12];
      mload(rhi, s, rl, V, N, h);
#pragma unroll
      for (int c = 0; c < 12; ++c) l[c] = cx((float)h[c].re, (float)h[c].im);
      mstore(rlo, s, rl, V, N, l);
    }
  }
}

// After the conversion: one thread updates the per-RHS scalars (a separate launch, so it runs
// after every block of the conversion).
__global__ void mconv_finish_kernel(MCgScalars* sc, int count) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int i = 0; i < sc->nrhs; ++i) {
    if (sc->status[i] != ST_RUNNING) continue;
    const double rr = sc->rr_true[i];
    sc->rr[i] = rr;
    sc->rr_ref[i] = rr;
    sc->need[i] = 0;
    if (!isfinite(rr))
      sc->status[i] = ST_BREAKDOWN;
    else if (rr <= sc->tol2 * sc->eta2[i])
      sc->status[i] = ST_PENDING;
  }
  sc->need_update = 0;
  sc->no_update = 1;
  if (count) sc->updates += 1;
}

template <int SP>
static cudaError_t mupd_r(FieldPtr r, FieldPtr q, FieldPtr p, FieldPtr xlo, int V, MCgScalars* sc, double* partials,
                          int N, int K, int spb, int grid_x, int mixed, int use_cond, unsigned long long upd,
                          cudaStream_t st) {
  dim3 grid(grid_x, N / K);
  const int block = K * spb;
  const size_t smem = sizeof(double) * (block + 32);
  const cudaGraphConditionalHandle h = (cudaGraphConditionalHandle)upd;
  if (mixed)
    mcg_update_r_kernel<SP, P32, true><<<grid, block, smem, st>>>(mview<SP>(r), mview<SP>(q), mview<SP>(p),
                                                                  mview<P32>(xlo), V, sc, partials, K, use_cond, h);
  else
    mcg_update_r_kernel<SP, SP, false><<<grid, block, smem, st>>>(mview<SP>(r), mview<SP>(q), mview<SP>(p),
                                                                  mview<SP>(r), V, sc, partials, K, use_cond, h);
  return cudaGetLastError();
}

cudaError_t launch_mcg_update_r(int prec, FieldPtr r, FieldPtr q, FieldPtr p, FieldPtr xlo, int V, MCgScalars* sc,
                                double* partials, int N, int K, int spb, int grid_x, int mixed, int use_cond,
                                unsigned long long upd, cudaStream_t st) {
  if (grid_x < 1 || grid_x > kMaxMultiGrid) return cudaErrorInvalidValue;  // reduction workspace bound
  switch (prec) {
    case SP64: return mixed ? cudaErrorInvalidValue : mupd_r<P64>(r, q, p, xlo, V, sc, partials, N, K, spb, grid_x, 0, use_cond, upd, st);
    case SP32: return mupd_r<P32>(r, q, p, xlo, V, sc, partials, N, K, spb, grid_x, mixed, use_cond, upd, st);
    case SP16: return mixed ? mupd_r<P16>(r, q, p, xlo, V, sc, partials, N, K, spb, grid_x, 1, use_cond, upd, st)
                            : cudaErrorInvalidValue;
  }
  return cudaErrorInvalidValue;
}

template <int SP>
static cudaError_t mupd_xp(FieldPtr x, FieldPtr p, FieldPtr s, int V, MCgScalars* sc, double* partials, int N, int K,
                           int spb, int grid_x, int mixed, int use_cond, unsigned long long cond, cudaStream_t st) {
  dim3 grid(grid_x, N / K);
  const int block = K * spb;
  const size_t smem = sizeof(double) * (block + 32);
  const cudaGraphConditionalHandle h = (cudaGraphConditionalHandle)cond;
  if (mixed)
    mcg_update_xp_kernel<SP, true><<<grid, block, smem, st>>>(mview<SP>(p), mview<SP>(p), mview<SP>(s), V, sc,
                                                              partials, K, use_cond, h);
  else
    mcg_update_xp_kernel<SP, false><<<grid, block, smem, st>>>(mview<SP>(x), mview<SP>(p), mview<SP>(s), V, sc,
                                                               partials, K, use_cond, h);
  return cudaGetLastError();
}

cudaError_t launch_mcg_update_xp(int prec, FieldPtr x, FieldPtr p, FieldPtr s, int V, MCgScalars* sc, double* partials,
                                 int N, int K, int spb, int grid_x, int mixed, int use_cond, unsigned long long cond,
                                 cudaStream_t st) {
  if (grid_x < 1 || grid_x > kMaxMultiGrid) return cudaErrorInvalidValue;  // reduction workspace bound
  switch (prec) {
    case SP64: return mupd_xp<P64>(x, p, s, V, sc, partials, N, K, spb, grid_x, mixed, use_cond, cond, st);
    case SP32: return mupd_xp<P32>(x, p, s, V, sc, partials, N, K, spb, grid_x, mixed, use_cond, cond, st);
    case SP16: return mupd_xp<P16>(x, p, s, V, sc, partials, N, K, spb, grid_x, mixed, use_cond, cond, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_mcg_init(MCgScalars* sc, cudaStream_t st) {
  mcg_init_kernel<<<1, kMaxRhs, 0, st>>>(sc);
  return cudaGetLastError();
}

cudaError_t launch_mcg_check(MCgScalars* sc, int use_cond, unsigned long long cond, cudaStream_t st) {
  mcg_check_kernel<<<1, 32, 0, st>>>(sc, use_cond, (cudaGraphConditionalHandle)cond);
  return cudaGetLastError();
}

cudaError_t launch_macc(FieldPtr xhi, FieldPtr xlo, int V, int N, int grid_x, cudaStream_t st) {
  if (xhi.prec != SP64 || xlo.prec != SP32) return cudaErrorInvalidValue;
  macc_kernel<<<grid_x, mblock(N), 0, st>>>(mview<P64>(xhi), mview<P32>(xlo), V, N);
  return cudaGetLastError();
}

cudaError_t launch_mconv(FieldPtr rhi, FieldPtr rlo, int V, int N, int grid_x, MCgScalars* sc, int count,
                         cudaStream_t st) {
  if (rhi.prec != SP64) return cudaErrorInvalidValue;
  switch (rlo.prec) {
    case SP32: mconv_kernel<P32><<<grid_x, mblock(N), 0, st>>>(mview<P64>(rhi), mview<P32>(rlo), V, sc, count); break;
    case SP16: mconv_kernel<P16><<<grid_x, mblock(N), 0, st>>>(mview<P64>(rhi), mview<P16>(rlo), V, sc, count); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  mconv_finish_kernel<<<1, 32, 0, st>>>(sc, count);
  return cudaGetLastError();
}


// ---------------------------------------------------------------- multi-RHS double-float helpers

// FP64 multi field (double2 [12][V][N]) <-> double-float multi field (float4 hi/lo [6][V][N])
__global__ void mconvert_kernel(MSpinor<P64> a, MSpinor<PDF> b, int V, int N, int to_df) {
  const int rl = threadIdx.x % N, sl = threadIdx.x / N, spb = blockDim.x / N;
  if (sl >= spb) return;
  for (int s = blockIdx.x * spb + sl; s < V; s += gridDim.x * spb) {
    if (to_df) {
      Cx<double> v[12];
      Cx<dfloat> w[12];
      mload(a, s, rl, V, N, v);
#pragma unroll
      for (int c = 0; c < 12; ++c) w[c] = cx(dfloat(v[c].re), dfloat(v[c].im));
      mstore(b, s, rl, V, N, w);
    } else {
      Cx<double> v[12];
      Cx<dfloat> w[12];
      mload(b, s, rl, V, N, w);
#pragma unroll
      for (int c = 0; c < 12; ++c) v[c] = cx((double)w[c].re, (double)w[c].im);
      mstore(a, s, rl, V, N, v);
    }
  }
}

// x_hi += x_lo in double-float, x_lo = 0 (all right-hand sides)
__global__ void macc_df_kernel(MSpinor<PDF> xhi, MSpinor<P32> xlo, int V, int N) {
  const int rl = threadIdx.x % N, sl = threadIdx.x / N, spb = blockDim.x / N;
  if (sl >= spb) return;
  for (int s = blockIdx.x * spb + sl; s < V; s += gridDim.x * spb) {
    Cx<dfloat> xh[12];
    Cx<float> xl[12];
    mload(xhi, s, rl, V, N, xh);
    mload(xlo, s, rl, V, N, xl);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      xh[c].re = xh[c].re + dfloat(xl[c].re, 0.f);
      xh[c].im = xh[c].im + dfloat(xl[c].im, 0.f);
      xl[c] = cx(0.f, 0.f);
    }
    mstore(xhi, s, rl, V, N, xh);
    mstore(xlo, s, rl, V, N, xl);
  }
}

// r_lo = hi part of the double-float residual, for every right-hand side still running
template <int SPW>
__global__ void mconv_df_kernel(MSpinor<PDF> rhi, MSpinor<SPW> rlo, int V, MCgScalars* sc) {
  const int N = sc->nrhs;
  const int rl = threadIdx.x % N, sl = threadIdx.x / N, spb = blockDim.x / N;
  if (sl < spb && sc->status[rl] == ST_RUNNING) {
    for (int s = blockIdx.x * spb + sl; s < V; s += gridDim.x * spb) {
      Cx<dfloat> h[12];
      Cx<float> l[12];
      mload(rhi, s, rl, V, N, h);
#pragma unroll
      for (int c = 0; c < 12; ++c) l[c] = cx(h[c].re.hi, h[c].im.hi);
      mstore(rlo, s, rl, V, N, l);
    }
  }
}

cudaError_t launch_mconvert_df(FieldPtr f64, FieldPtr df, int V, int N, int grid_x, int to_df, cudaStream_t st) {
  if (f64.prec != SP64 || df.prec != SPDF) return cudaErrorInvalidValue;
  mconvert_kernel<<<grid_x, mblock(N), 0, st>>>(mview<P64>(f64), mview_df(df, V, N), V, N, to_df);
  return cudaGetLastError();
}

cudaError_t launch_macc_df(FieldPtr xhi, FieldPtr xlo, int V, int N, int grid_x, cudaStream_t st) {
  if (xhi.prec != SPDF || xlo.prec != SP32) return cudaErrorInvalidValue;
  macc_df_kernel<<<grid_x, mblock(N), 0, st>>>(mview_df(xhi, V, N), mview<P32>(xlo), V, N);
  return cudaGetLastError();
}

cudaError_t launch_mconv_df(FieldPtr rhi, FieldPtr rlo, int V, int N, int grid_x, MCgScalars* sc, int count,
                            cudaStream_t st) {
  if (rhi.prec != SPDF) return cudaErrorInvalidValue;
  switch (rlo.prec) {
    case SP32: mconv_df_kernel<P32><<<grid_x, mblock(N), 0, st>>>(mview_df(rhi, V, N), mview<P32>(rlo), V, sc); break;
    case SP16: mconv_df_kernel<P16><<<grid_x, mblock(N), 0, st>>>(mview_df(rhi, V, N), mview<P16>(rlo), V, sc); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  mconv_finish_kernel<<<1, 32, 0, st>>>(sc, count);
  return cudaGetLastError();
}

}  // namespace wdk
