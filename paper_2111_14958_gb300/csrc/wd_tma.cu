// The FP32 dslash with its neighbour spinors staged in shared memory by the tensor memory
// accelerator (TMA), as an alternative to the per-thread neighbour loads of dslash_kernel that go
// through the L1 cache.
//
// A CTA owns tiles of Lx x BY x BZ x BT sites (whole x rows, so the x hops wrap inside the tile).
// For each tile one thread issues seven cp.async.bulk.tensor loads of the FP32 spinor field
// (float4 [6][V], viewed as a 5-D tensor of floats (4 Lx, Ly, Lz, Lt, 6)): the tile itself and the
// six face slabs one site thick in y, z and t (taken from the other side of the lattice at its edge:
// TMA does not wrap, so the periodic neighbours are addressed by their own coordinates). Every box
// starts at x = 0, so the innermost coordinate is always 16-byte aligned. The loads complete on an
// mbarrier whose wait is bounded: past the limit the kernel records an error and returns. Each
// thread then computes one site from shared memory (links, read once per site and direction, come
// from global memory), writes it, and the CTA moves to its next tile.
//
// Shared memory per tile (float4 words): 6 Lx (BY BZ BT + 2 BZ BT + 2 BY BT + 2 BY BZ); for Lx = 32
// and a 2 x 2 x 2 tile that is 96 KiB (two CTAs per SM) and 4x the interior, against the ~2.3x
// re-fetch from L2 that the L1 path measured at 32^4 (profiles/dslash_f32c12_32x4.md).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "wd_stencil.cuh"

namespace wdk {

namespace {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3, int c4,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];" ::"r"(smem_u32(dst)),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

struct TmaArgs {
  Geom g;
  const float4* u;      // FP32 12-real links float4 [4][3][V]
  float4* out;          // float4 [6][V]
  const double* kappa_dev;
  float mkappa;
  int BY, BZ, BT;       // tile extents in y, z, t (x: the whole row)
  int ntiles;
  long long spin_limit;
  int* err;
  double* partials;
  unsigned* ticket;
  double* result;
};

// Region of shared memory holding a box of extents (Lx, by, bz, bt) x 6 planes.
struct Box {
  const float4* p;
  int by, bz, bt;
  __device__ __forceinline__ float4 at(int plane, int x, int y, int z, int t, int Lx) const {
    return p[((((size_t)plane * bt + t) * bz + z) * by + y) * Lx + x];
  }
};

template <int MU, int SF>
__device__ __forceinline__ void tma_hop(const TmaArgs& a, const Box (&bx)[7], int x, int y, int z, int t, int s,
                                        const int (&gc)[4], float mk, Cx<float> (&acc)[12], int dir) {
  const int Lx = a.g.L[0];
  int nx = x, ny = y, nz = z, nt = t;
  int r = 0;  // region: 0 interior, 1/2 y- / y+, 3/4 z-, z+, 5/6 t-, t+
  const int step = dir == 0 ? 1 : -1;
  if (MU == 0) {
    nx = (x + step + Lx) % Lx;
  } else if (MU == 1) {
    ny = y + step;
    if (ny < 0) { r = 1; ny = 0; }
    else if (ny >= a.BY) { r = 2; ny = 0; }
  } else if (MU == 2) {
    nz = z + step;
    if (nz < 0) { r = 3; nz = 0; }
    else if (nz >= a.BZ) { r = 4; nz = 0; }
  } else {
    nt = t + step;
    if (nt < 0) { r = 5; nt = 0; }
    else if (nt >= a.BT) { r = 6; nt = 0; }
  }
  const bool wrap = dir == 0 ? gc[MU] == a.g.L[MU] - 1 : gc[MU] == 0;
  const float k = (wrap && a.g.bc[MU] < 0) ? -mk : mk;
  // r is 0 or one of this direction's two faces: select among compile-time indices (no local memory)
  constexpr int FM = MU == 0 ? 0 : 2 * MU - 1, FP = MU == 0 ? 0 : 2 * MU;
  const Box b = r == 0 ? bx[0] : (r == FM ? bx[FM] : bx[FP]);
  Cx<float> psi[12];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float4 d = b.at(j, nx, ny, nz, nt, Lx);
    psi[2 * j] = cx(d.x, d.y);
    psi[2 * j + 1] = cx(d.z, d.w);
  }
  // the link: U_mu(s) forward, U_mu(s - mu) backward (global site index of that neighbour)
  int ls = s;
  if (dir == 1) {
    const int st = a.g.stride[MU];
    ls = gc[MU] == 0 ? s + (a.g.L[MU] - 1) * st : s - st;
  }
  Cx<float> u[9];
  GaugeRef<float, true> gr;
  gr.p = a.u;
  load_link(gr, MU, ls, a.g.V, u);
  Cx<float> h[6], chi[6];
  if (dir == 0) {
    spin_project<MU, SF>(psi, h);
    su3_mul(u, h, chi);
    spin_reconstruct<MU, SF>(acc, chi, k);
  } else {
    spin_project<MU, -SF>(psi, h);
    su3_dag_mul(u, h, chi);
    spin_reconstruct<MU, -SF>(acc, chi, k);
  }
}

template <bool DAG, bool NORM>
__global__ void __launch_bounds__(512, 1) dslash_tma_kernel(const __grid_constant__ CUtensorMap tm_in,
                                                            const __grid_constant__ CUtensorMap tm_fy,
                                                            const __grid_constant__ CUtensorMap tm_fz,
                                                            const __grid_constant__ CUtensorMap tm_ft,
                                                            const TmaArgs a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ __align__(8) unsigned long long bar;
  // the regions start on a 1024-byte boundary whatever alignment the dynamic shared memory has (the
  // launch allocates 1024 bytes more than the regions need)
  float4* sm = reinterpret_cast<float4*>(sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u));
  const int Lx = a.g.L[0], Ly = a.g.L[1], Lz = a.g.L[2], Lt = a.g.L[3];
  const int BY = a.BY, BZ = a.BZ, BT = a.BT;
  // regions (float4 words): each a multiple of 6 Lx words, 96 Lx bytes, a multiple of 128 (Lx % 4 == 0)
  const int nI = 6 * Lx * BY * BZ * BT, nY = 6 * Lx * BZ * BT, nZ = 6 * Lx * BY * BT, nT = 6 * Lx * BY * BZ;
  Box bx[7];
  const float4* base = sm;
  bx[0] = Box{base, BY, BZ, BT};
  base += nI;
  bx[1] = Box{base, 1, BZ, BT};
  base += nY;
  bx[2] = Box{base, 1, BZ, BT};
  base += nY;
  bx[3] = Box{base, BY, 1, BT};
  base += nZ;
  bx[4] = Box{base, BY, 1, BT};
  base += nZ;
  bx[5] = Box{base, BY, BZ, 1};
  base += nT;
  bx[6] = Box{base, BY, BZ, 1};
  const unsigned bytes = 16u * (unsigned)(nI + 2 * nY + 2 * nZ + 2 * nT);
  const int tid = threadIdx.x;
  const int x = tid % Lx, y = (tid / Lx) % BY, z = (tid / (Lx * BY)) % BZ, t = tid / (Lx * BY * BZ);
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const float mk = a.kappa_dev ? (float)(-*a.kappa_dev) : a.mkappa;
  constexpr int SF = DAG ? +1 : -1;
  const int ty = Ly / BY, tz = Lz / BZ;
  double n2 = 0.0;
  unsigned phase = 0;
  bool ok = true;
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int y0 = (tile % ty) * BY, z0 = ((tile / ty) % tz) * BZ, t0 = (tile / (ty * tz)) * BT;
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads before the new writes
      mbar_expect_tx(&bar, bytes);
      tma_load_5d((void*)bx[0].p, &tm_in, 0, y0, z0, t0, 0, &bar);
      tma_load_5d((void*)bx[1].p, &tm_fy, 0, (y0 - 1 + Ly) % Ly, z0, t0, 0, &bar);
      tma_load_5d((void*)bx[2].p, &tm_fy, 0, (y0 + BY) % Ly, z0, t0, 0, &bar);
      tma_load_5d((void*)bx[3].p, &tm_fz, 0, y0, (z0 - 1 + Lz) % Lz, t0, 0, &bar);
      tma_load_5d((void*)bx[4].p, &tm_fz, 0, y0, (z0 + BZ) % Lz, t0, 0, &bar);
      tma_load_5d((void*)bx[5].p, &tm_ft, 0, y0, z0, (t0 - 1 + Lt) % Lt, 0, &bar);
      tma_load_5d((void*)bx[6].p, &tm_ft, 0, y0, z0, (t0 + BT) % Lt, 0, &bar);
    }
    long long spins = 0;
    while (!mbar_try_wait(&bar, phase & 1u)) {
      if (++spins > a.spin_limit) {
        ok = false;
        break;
      }
    }
    if (!__syncthreads_and(ok)) break;
    phase += 1;
    const int gc[4] = {x, y0 + y, z0 + z, t0 + t};
    const int s = x + Lx * (gc[1] + Ly * (gc[2] + Lz * gc[3]));
    Cx<float> acc[12];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float4 d = bx[0].at(j, x, y, z, t, Lx);
      acc[2 * j] = cx(d.x, d.y);
      acc[2 * j + 1] = cx(d.z, d.w);
    }
    tma_hop<0, SF>(a, bx, x, y, z, t, s, gc, mk, acc, 0);
    tma_hop<0, SF>(a, bx, x, y, z, t, s, gc, mk, acc, 1);
    tma_hop<1, SF>(a, bx, x, y, z, t, s, gc, mk, acc, 0);
    tma_hop<1, SF>(a, bx, x, y, z, t, s, gc, mk, acc, 1);
    tma_hop<2, SF>(a, bx, x, y, z, t, s, gc, mk, acc, 0);
    tma_hop<2, SF>(a, bx, x, y, z, t, s, gc, mk, acc, 1);
    tma_hop<3, SF>(a, bx, x, y, z, t, s, gc, mk, acc, 0);
    tma_hop<3, SF>(a, bx, x, y, z, t, s, gc, mk, acc, 1);
#pragma unroll
    for (int j = 0; j < 6; ++j)
      a.out[(size_t)j * a.g.V + s] = make_float4(acc[2 * j].re, acc[2 * j].im, acc[2 * j + 1].re, acc[2 * j + 1].im);
    if (NORM) n2 += norm2_site(acc);
    __syncthreads();  // every thread done with this tile's shared memory
  }
  if (!ok) {
    // a copy did not complete within the limit: record it, give the copies in flight a bounded time
    // to land (the CTA's shared memory must not be released under them), and stop
    if (tid == 0) {
      atomicExch(a.err, 1);
      long long spins = 0;
      while (!mbar_try_wait(&bar, phase & 1u) && ++spins < a.spin_limit) {
      }
    }
    return;
  }
  if (NORM) {
    double v[1] = {n2}, tot[1];
    if (grid_reduce<OpSum, 1>(v, a.partials, a.ticket, tot) && threadIdx.x == 0) *a.result = tot[0];
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

// The spinor field as floats (4 Lx, Ly, Lz, Lt, 6) with a box of (4 Lx, by, bz, bt, 6).
bool encode(CUtensorMap* tm, const void* field, const GeomH& g, int by, int bz, int bt) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], Lt = g.L[3];
  const cuuint64_t dims[5] = {4 * Lx, Ly, Lz, Lt, 6};
  const cuuint64_t strides[4] = {16 * Lx, 16 * Lx * Ly, 16 * Lx * Ly * Lz, 16 * Lx * Ly * Lz * Lt};
  const cuuint32_t box[5] = {(cuuint32_t)(4 * Lx), (cuuint32_t)by, (cuuint32_t)bz, (cuuint32_t)bt, 6};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(field), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Tile shapes: (2, 2, 2) with two CTAs per SM, or (4, 2, 2) with one.
bool tma_dslash_supported(const GeomH& g, int tile) {
  const int by = tile == 1 ? 4 : 2, bz = 2, bt = 2;
  // Lx a multiple of 4: every shared-memory region is then a multiple of 128 bytes (96 Lx bytes per
  // site row), so every box lands 128-byte aligned; 4 Lx <= 256 floats per box row
  return g.L[0] >= 4 && g.L[0] <= 64 && g.L[0] % 4 == 0 && g.L[1] % by == 0 && g.L[2] % bz == 0 &&
         g.L[3] % bt == 0 && g.L[0] * by * bz * bt <= 512 && encode_fn() != nullptr;
}

cudaError_t launch_dslash_tma(const DslashCall& c, int tile, int* err, cudaStream_t st) {
  if (c.in.prec != SP32 || c.u.prec != SP32 || !c.u.c12 || c.epi != EPI_PLAIN || !tma_dslash_supported(c.g, tile))
    return cudaErrorInvalidValue;
  const int by = tile == 1 ? 4 : 2, bz = 2, bt = 2;
  CUtensorMap tm_in, tm_fy, tm_fz, tm_ft;
  if (!encode(&tm_in, c.in.p, c.g, by, bz, bt) || !encode(&tm_fy, c.in.p, c.g, 1, bz, bt) ||
      !encode(&tm_fz, c.in.p, c.g, by, 1, bt) || !encode(&tm_ft, c.in.p, c.g, by, bz, 1))
    return cudaErrorInvalidValue;
  TmaArgs a;
  memcpy(&a.g, &c.g, sizeof(Geom));
  a.u = reinterpret_cast<const float4*>(c.u.p);
  a.out = reinterpret_cast<float4*>(c.out.p);
  a.kappa_dev = c.kappa_dev;
  a.mkappa = (float)(-c.kappa);
  a.BY = by;
  a.BZ = bz;
  a.BT = bt;
  a.ntiles = (c.g.L[1] / by) * (c.g.L[2] / bz) * (c.g.L[3] / bt);
  a.spin_limit = 1LL << 22;
  a.err = err;
  a.partials = c.red.partials;
  a.ticket = c.red.ticket;
  a.result = c.red.result;
  const int Lx = c.g.L[0];
  const int threads = Lx * by * bz * bt;
  const size_t smem = 16 * (size_t)6 * Lx * (by * bz * bt + 2 * bz * bt + 2 * by * bt + 2 * by * bz) + 1024;
  auto launch = [&](auto k) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = per_sm * sms;
    if (grid > a.ntiles) grid = a.ntiles;
    if (c.red.result && grid > kLoopMaxGrid) grid = kLoopMaxGrid;
    if (!red_fits(c.red, grid)) return cudaErrorInvalidValue;
    k<<<grid, threads, smem, st>>>(tm_in, tm_fy, tm_fz, tm_ft, a);
    return cudaGetLastError();
  };
  if (c.dagger) return c.red.result ? launch(dslash_tma_kernel<true, true>) : launch(dslash_tma_kernel<true, false>);
  return c.red.result ? launch(dslash_tma_kernel<false, true>) : launch(dslash_tma_kernel<false, false>);
}

}  // namespace wdk
