// FP64 fused multiply-add throughput of the current GPU, measured on independent chains of dependent
// FMAs: a cross-check of the compute ceiling pi of the roofline P = min(pi, beta I) (Eq. (2),
// Sec. 3.1) for the FP64 dslash, which on GB300 is bound by the FP64 pipe rather than by HBM. On
// GB300 it reads about 84 % of the unit count (2 DFMA per clock per SM), while the dslash's own mix
// of FMAs, adds and multiplies retires FP64 instructions at up to 95 % of it, so the unit count is
// the ceiling and this rate is reported beside it.
#include <cuda_runtime.h>

#include <string>

#include "../../include/wd.h"

namespace wdk {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int kChains = 8;       // independent FMA chains per thread (enough to cover the pipe latency)
constexpr int kProbeBlock = 256;
constexpr int kBlocksPerSm = 4;  // 32 resident warps per SM

// Receives the chains' sums in the (impossible) case below; keeps the compiler from dropping them.
static __device__ double g_probe_sink[kProbeBlock];

// Every thread runs kChains dependent chains a <- a * m + c for `iters` steps. The values stay
// finite and above 1 (m is within 1e-7 of 1, c > 0), and the final sum is stored only if it equals
// `never`, which the host sets negative so that it cannot happen.
__global__ void __launch_bounds__(kProbeBlock) dfma_probe_kernel(int iters, double m, double c, double never) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == never) g_probe_sink[threadIdx.x] = s;
}

}  // namespace

extern "C" wd_status wd_measure_fp64_peak(void* cuda_stream, int repeats, double* tflops) {
  if (!tflops || repeats < 1 || repeats > 1000) {
    wdk::set_last_error("tflops must be non-null and repeats in [1, 1000]");
    return WD_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const int iters = 4096;
  const int grid = sms * kBlocksPerSm;
  float best = 1e30f;
  for (int r = 0; e == cudaSuccess && r <= repeats; ++r) {  // r = 0 warms up
    e = cudaEventRecord(a, st);
    if (e == cudaSuccess) {
      dfma_probe_kernel<<<grid, kProbeBlock, 0, st>>>(iters, 1.0000001, 1e-9, -1.0);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && r > 0 && ms < best) best = ms;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) {
    wdk::set_last_error(std::string("wd_measure_fp64_peak: ") + cudaGetErrorString(e));
    return WD_ECUDA;
  }
  const double flops = 2.0 * kChains * (double)iters * (double)grid * kProbeBlock;
  *tflops = flops / ((double)best * 1e-3) / 1e12;
  return WD_OK;
}
