// wd_dslash_noalloc: the dslash with its fused ||out||^2, for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code running under a framework that owns every device
// allocation (a custom or pooled allocator that must account for all memory), plug-ins that are
// handed fixed buffers, or code paths where an allocation could block or fail late. They cannot
// create a wd_ctx (wd_create allocates its workspace), so this entry point takes every input and
// output from the caller, reads the fields in their canonical layout directly, and keeps the one
// piece of scratch the fused norm needs (one partial sum per thread block plus a ticket counter)
// in a fixed array in this file's device memory.
//
// The array below lives in the library's module on every GPU that loads the library and stays
// there until the process exits. Its size caps the volume this entry point accepts.
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/wd.h"
#include "wd_device.cuh"

namespace wdk {
void set_last_error(const std::string& msg);
}

namespace {

using namespace wdk;

constexpr int kBlock = 128;                       // threads per block (one site each)
constexpr int kMaxBlocks = 8192;                  // => at most 8192 * 128 = 2^20 sites
constexpr int kMaxSites = kBlock * kMaxBlocks;
constexpr size_t kPartialBytes = sizeof(double) * kMaxBlocks;
constexpr size_t kScratchBytes = kPartialBytes + 256;  // partials, then the ticket counter

// Shared by every call on a device; holds the last call's partial sums.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// canonical spinor: complex128 [V][4][3]; canonical links: complex128 [V][4][3][3]
__device__ __forceinline__ void load_canon_spinor(const double2* __restrict__ p, int s, Cx<double> (&v)[12]) {
  const double2* q = p + (size_t)s * 12;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const double2 d = __ldg(q + c);
    v[c] = cx(d.x, d.y);
  }
}

__device__ __forceinline__ void load_canon_link(const double2* __restrict__ p, int mu, int s, Cx<double> (&u)[9]) {
  const double2* q = p + ((size_t)s * 4 + mu) * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double2 d = __ldg(q + k);
    u[k] = cx(d.x, d.y);
  }
}

template <int MU, int SF>
__device__ __forceinline__ void canon_hops(const Geom& g, const double2* U, const double2* in, double mk, int s,
                                           const int (&c)[4], Cx<double> (&acc)[12]) {
  {
    const bool wrap = c[MU] == g.L[MU] - 1;
    const int nb = wrap ? s - (g.L[MU] - 1) * g.stride[MU] : s + g.stride[MU];
    const double k = (wrap && g.bc[MU] < 0) ? -mk : mk;
    Cx<double> psi[12], h[6], u[9], chi[6];
    load_canon_spinor(in, nb, psi);
    spin_project<MU, SF>(psi, h);
    load_canon_link(U, MU, s, u);
    su3_mul(u, h, chi);
    spin_reconstruct<MU, SF>(acc, chi, k);
  }
  {
    const bool wrap = c[MU] == 0;
    const int nb = wrap ? s + (g.L[MU] - 1) * g.stride[MU] : s - g.stride[MU];
    const double k = (wrap && g.bc[MU] < 0) ? -mk : mk;
    Cx<double> psi[12], h[6], u[9], chi[6];
    load_canon_spinor(in, nb, psi);
    spin_project<MU, -SF>(psi, h);
    load_canon_link(U, MU, nb, u);
    su3_dag_mul(u, h, chi);
    spin_reconstruct<MU, -SF>(acc, chi, k);
  }
}

template <bool DAG, bool NORM>
__global__ void __launch_bounds__(kBlock) dslash_canon_kernel(Geom g, const double2* __restrict__ U,
                                                              const double2* __restrict__ in, double2* __restrict__ out,
                                                              double mkappa, double* partials, unsigned* ticket,
                                                              double* result) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double n2 = 0.0;
  if (s < g.V) {
    int c[4];
    int r = s;
    c[0] = r % g.L[0];
    r /= g.L[0];
    c[1] = r % g.L[1];
    r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];
    Cx<double> acc[12];
    load_canon_spinor(in, s, acc);
    constexpr int SF = DAG ? +1 : -1;
    canon_hops<0, SF>(g, U, in, mkappa, s, c, acc);
    canon_hops<1, SF>(g, U, in, mkappa, s, c, acc);
    canon_hops<2, SF>(g, U, in, mkappa, s, c, acc);
    canon_hops<3, SF>(g, U, in, mkappa, s, c, acc);
    double2* o = out + (size_t)s * 12;
#pragma unroll
    for (int i = 0; i < 12; ++i) o[i] = make_double2(acc[i].re, acc[i].im);
    if (NORM) n2 = norm2_site(acc);
  }
  if (NORM) {
    double v[1] = {n2}, tot[1];
    if (grid_reduce<OpSum, 1>(v, partials, ticket, tot) && threadIdx.x == 0) *result = tot[0];
  }
}

std::mutex g_addr_mu;
void* g_addr[256];  // device address of g_noalloc_scratch, per device ordinal

// Host code cannot use &g_noalloc_scratch as a device address: ask the runtime, once per device.
// The address stays valid for the life of the device's primary context; a cudaDeviceReset after
// the first call would unload the module and leave the cached address stale, so such a reset is
// not supported in a process that uses this entry point.
wd_status scratch_address(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    wdk::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return WD_ECUDA;
  }
  if (dev < 0 || dev >= 256) {
    wdk::set_last_error("device ordinal out of range");
    return WD_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      wdk::set_last_error(std::string("cudaGetSymbolAddress of the no-allocation scratch: ") + cudaGetErrorString(e));
      return WD_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return WD_OK;
}

}  // namespace

extern "C" wd_status wd_dslash_noalloc(const int dims[4], double kappa, const int boundary[4], const double* U,
                                       const double* in, double* out, int dagger, double* norm2_out,
                                       void* cuda_stream) {
  wdk::set_last_error("");
  if (!dims || !U || !in || !out) {
    wdk::set_last_error("null argument");
    return WD_EINVAL;
  }
  if (in == out) {
    wdk::set_last_error("in and out must differ");
    return WD_EINVAL;
  }
  // the running product is checked at every step, so four large extents cannot overflow it
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 2) {
      wdk::set_last_error("every lattice extent must be >= 2");
      return WD_EINVAL;
    }
    V *= dims[i];
    if (V > kMaxSites) {
      wdk::set_last_error("volume exceeds the fixed scratch of wd_dslash_noalloc (at most 2^20 sites)");
      return WD_EINVAL;
    }
  }
  // in and out are V * 12 complex128 each; any overlap would let a site read a neighbour the
  // kernel has already overwritten
  {
    const unsigned long long n = (unsigned long long)V * 12 * sizeof(double2);
    const unsigned long long a = (unsigned long long)(uintptr_t)in, b = (unsigned long long)(uintptr_t)out;
    if (a < b + n && b < a + n) {
      wdk::set_last_error("in and out overlap");
      return WD_EINVAL;
    }
  }
  if (!std::isfinite(kappa) || std::fabs(kappa) >= 1.0) {
    wdk::set_last_error("kappa must be finite with |kappa| < 1");
    return WD_EINVAL;
  }
  wdk::Geom g;
  for (int i = 0; i < 4; ++i) {
    g.L[i] = dims[i];
    const int b = boundary ? boundary[i] : (i == 3 ? -1 : 1);
    if (b != 1 && b != -1) {
      wdk::set_last_error("boundary entries must be +1 or -1");
      return WD_EINVAL;
    }
    g.bc[i] = b;
  }
  g.stride[0] = 1;
  g.stride[1] = dims[0];
  g.stride[2] = dims[0] * dims[1];
  g.stride[3] = dims[0] * dims[1] * dims[2];
  g.V = (int)V;
  unsigned char* base = nullptr;
  wd_status st = scratch_address(&base);
  if (st != WD_OK) return st;
  double* partials = reinterpret_cast<double*>(base);
  unsigned* ticket = reinterpret_cast<unsigned*>(base + kPartialBytes);
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const int grid = (int)((V + kBlock - 1) / kBlock);
  const double2* U2 = reinterpret_cast<const double2*>(U);
  const double2* in2 = reinterpret_cast<const double2*>(in);
  double2* out2 = reinterpret_cast<double2*>(out);
  cudaError_t e = cudaSuccess;
  if (norm2_out) {
    // the ticket counter must start at zero; the partial sums are overwritten by every block
    e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), stream);
    if (e == cudaSuccess) {
      if (dagger)
        dslash_canon_kernel<true, true><<<grid, kBlock, 0, stream>>>(g, U2, in2, out2, -kappa, partials, ticket, norm2_out);
      else
        dslash_canon_kernel<false, true><<<grid, kBlock, 0, stream>>>(g, U2, in2, out2, -kappa, partials, ticket, norm2_out);
      e = cudaGetLastError();
    }
  } else {
    if (dagger)
      dslash_canon_kernel<true, false><<<grid, kBlock, 0, stream>>>(g, U2, in2, out2, -kappa, nullptr, nullptr, nullptr);
    else
      dslash_canon_kernel<false, false><<<grid, kBlock, 0, stream>>>(g, U2, in2, out2, -kappa, nullptr, nullptr, nullptr);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    wdk::set_last_error(std::string("wd_dslash_noalloc launch: ") + cudaGetErrorString(e));
    return WD_ECUDA;
  }
  return WD_OK;
}
