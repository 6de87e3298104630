// Host-visible interface between the C ABI (wd_api.cu) and the kernel translation units.
// Plain structs and launcher declarations only; no device code.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

namespace wdk {

// NVTX range over a scope (shows the library's phases in Nsight timelines; free without a tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct Geom;  // defined in wd_device.cuh; mirrored by GeomH below

// Same memory layout as wdk::Geom.
struct GeomH {
  int L[4];
  int stride[4];
  int V;
  int bc[4];
};

enum { SP64 = 0, SP32 = 1, SP16 = 2, SPDF = 3 };  // spinor storage precisions (match wd_device.cuh)
// SPDF fields: float4 hi [6][V] followed by float4 lo [6][V] in one allocation; SPDF links: float2 hi
// [4][9][V] followed by float2 lo [4][9][V].

// A spinor field in the device layout.
struct FieldPtr {
  void* p;
  float* norm;  // P16 only
  int prec;
};

// A gauge field in the device layout.
struct GaugePtr {
  const void* p;
  int prec;  // SP64 (18 reals), SP32, or SPDF (18 reals, double-float)
  int c12;   // SP32 only: 1 = 12 reals
};

// Device-resident solver scalars (one per context). Layout shared with the kernels.
struct CgScalars;
// Record the recursive residual of iteration `it` if the solve keeps a history (device side).
__device__ __forceinline__ void record_residual(CgScalars* sc, int it, double rr);

struct CgScalars {
  double eta2;       // ||eta||^2
  double rr;         // recursive ||r||^2
  double qq;         // ||D p||^2
  double gamma;      // ||D^dag r||^2 of the current direction
  double gamma_new;  // ||D^dag r||^2 after the r update
  double alpha;
  double beta;
  double tol2;       // tol^2 (relative, squared) of the current launch
  double rr_true;    // ||eta - D x||^2 recomputed
  double max_dev;    // gauge unitarity check
  double rr_ref;     // mixed precision: ||r||^2 at the last reliable update
  double delta2;     // mixed precision: reliable-update trigger factor, squared
  double kappa;      // hopping parameter read by every dslash of the context (settable between solves)
  double scratch[4];
  double* hist;      // optional: recursive ||r||^2 of each iteration (index = iteration)
  int hist_len;      // entries hist holds (0: no history)
  int iter;          // cumulative iterations
  int maxit;
  int status;        // ST_* below
  int updates;       // reliable updates done
  int need_update;   // mixed precision: set when ||r|| dropped by delta since the last update
  int no_update;     // = !need_update (skip flag of the FP64 dslash in the update)
  unsigned ticket[16];
};

__device__ __forceinline__ void record_residual(CgScalars* sc, int it, double rr) {
  if (sc->hist != nullptr && it >= 0 && it < sc->hist_len) sc->hist[it] = rr;
}

enum { ST_RUNNING = 0, ST_CONVERGED = 1, ST_MAXIT = 2, ST_BREAKDOWN = 3, ST_PENDING = 4 };

// ticket slots (each kernel role uses its own counter)
enum { TK_DSLASH_A = 0, TK_DSLASH_B = 1, TK_UPD_R = 2, TK_UPD_XP = 3, TK_PACK = 4, TK_GAUGE = 5,
       TK_DSLASH_C = 6, TK_MISC = 7, TK_UPD_REL = 8 };

enum { EPI_PLAIN = 0, EPI_RESID = 1 };

// A reduction target: result == nullptr means no reduction. A launcher whose grid would need more
// block partials than cap refuses the launch (cudaErrorInvalidValue) instead of writing past them.
struct Red {
  double* partials;  // >= N * gridDim doubles
  unsigned* ticket;
  double* result;
  long long cap;     // doubles available at partials
};
inline bool red_fits(const Red& r, long long grid, int n = 1) { return !r.result || grid * n <= r.cap; }

struct DslashCall {
  GeomH g;
  GaugePtr u;
  FieldPtr in, out, b;  // b: EPI_RESID only (out = b - D in)
  double kappa;
  int dagger;
  int epi;
  const int* skip;  // optional: if *skip != 0 the launch does nothing
  Red red;          // optional |out|^2
  int block;
  const double* kappa_dev;  // optional: kappa read from device memory (overrides `kappa`)
  int variant;              // FP64 only: lanes per site 1, 2, 4, 8, 16 for variant 0..4
  int tma;                  // FP32 12-real, plain epilogue: 0 per-thread loads; 1 / 2 neighbour spinors staged
                            // by TMA in tiles of Lx x 2 x 2 x 2 / Lx x 4 x 2 x 2 sites (wd_tma.cu)
  int* err;                 // tma: set to 1 if a staging wait gave up
  int schedule;             // FP32 / FP16 load schedule: 0 or 1 hop by hop; 2 two sites per thread;
                            // 3 both hops of each direction loaded together (dslash_sched_kernel)
};
bool tma_dslash_supported(const GeomH& g, int tile);
cudaError_t launch_dslash_tma(const DslashCall& c, int tile, int* err, cudaStream_t st);
constexpr int kMaxDslashVariant = 4;
inline int lanes_of_variant(int v) { return v <= 0 ? 1 : (1 << v); }

// Launchers. Each returns cudaGetLastError() after the launch.
cudaError_t launch_dslash(const DslashCall& c, cudaStream_t st);

// The whole plain CG loop (CGLS, lexicographic layout, FP64 or FP32) as one cooperative launch,
// from the state the prologue leaves in sc; it writes status, iterations and scalars back.
struct CgLoopCall {
  GeomH g;
  GaugePtr u;
  FieldPtr x, r, p, q, s;
  double kappa;
  const double* kappa_dev;
  CgScalars* sc;
  double* partials;  // >= 3 * max_grid
  unsigned* bar;     // 64-bit barrier counter (8-byte aligned); each launcher zeroes it first
  int* err;          // zero; set to 1 if a barrier wait gave up
  int block;
  int max_grid;
  int variant;  // FP64: 1 = the dslash phases use two lanes per site
  int time_basis;  // FP64, one thread per site: 1 = the loop runs in the basis where gamma_t is diagonal
  int cg_form;     // 1: the paper's CG on D D^dag (one thread per site; variant must be 0)
  int start_b;  // mixed loop: resume at the D^dag half of an iteration (after a reliable update)
  FieldPtr t;   // even-odd loop: the odd-site temporary
  FieldPtr p2, r2;  // FP64 loop with 4, 8 or 16 lanes per site: second buffers of p and r
  FieldPtr tl;      // FP64 loop in the time-diagonal basis: pre-scaled time links (double2 [9][V])
  long long wait_limit;  // grid-barrier polls (64 ns sleep each) before a wait gives up
};
constexpr long long kLoopWaitLimit = 1LL << 26;  // about 4 s
cudaError_t launch_cg_loop(const CgLoopCall& c, cudaStream_t st);
// Up to kMaxBatch loops of the same shape (lattice, precision, launch shape) in one cooperative
// launch, each problem on its own blocks (blockIdx.y) with the grid it has alone; returns
// cudaErrorCooperativeLaunchTooLarge when the batch's blocks cannot all be resident.
constexpr int kMaxBatch = 8;
cudaError_t launch_cg_loop_n(const CgLoopCall* cs, int n, cudaStream_t st);
// The inner loop of the mixed-precision solver (x = x_lo in FP32; r, p, q, s in the working
// precision) as one cooperative launch that returns when a reliable update is due or the loop ends.
cudaError_t launch_cg_mixed_loop(const CgLoopCall& c, cudaStream_t st);
cudaError_t launch_cg_mixed_loop_n(const CgLoopCall* cs, int n, cudaStream_t st);
// The plain CGLS loop on the even-site Schur complement of a parity-ordered context.
cudaError_t launch_cg_eo_loop(const CgLoopCall& c, cudaStream_t st);
constexpr int kLoopMaxGrid = 8192;

// eo: null for lexicographic storage, else the geometry of a parity-ordered context.
// canonical complex128 [V][12] -> field; optional |src|^2 into red
cudaError_t launch_pack(const double* canon, FieldPtr out, int V, const GeomH* eo, Red red, int block,
                        cudaStream_t st);
// canonical complex64 [V][12] -> P32 field
cudaError_t launch_pack_c64(const float* canon, FieldPtr out, int V, const GeomH* eo, int block, cudaStream_t st);
// field -> canonical complex128
cudaError_t launch_unpack(FieldPtr in, double* canon, int V, const GeomH* eo, int block, cudaStream_t st);
// P32 field -> canonical complex64
cudaError_t launch_unpack_c64(FieldPtr in, float* canon, int V, const GeomH* eo, int block, cudaStream_t st);
// canonical complex128 links [V][4][9] -> gauge field; optional max deviation from SU(3) into red
cudaError_t launch_gauge_load(const double* canon, GaugePtr out, int V, const GeomH* eo, Red red, int block,
                              cudaStream_t st);

// CG pieces (prec = storage precision of all vectors involved); n = sites updated, V = stride of the
// fields (n = V, or n = V/2 for the even half of a parity-ordered field)
cudaError_t launch_cg_init(CgScalars* sc, int reset_iter, cudaStream_t st);
// gamma_from_rr: the search direction starts as r itself (the paper's form), so gamma = |r|^2
cudaError_t launch_cg_check(CgScalars* sc, int use_cond, unsigned long long cond, cudaStream_t st,
                            int gamma_from_rr = 0);
// grid-stride launches sized to one wave of resident blocks
// gamma_from_rr: |r|^2 after the update is also the next gamma (the paper's form)
cudaError_t launch_cg_update_r(int prec, FieldPtr r, FieldPtr q, int n, int V, CgScalars* sc, double* partials,
                               int block, cudaStream_t st, int gamma_from_rr = 0);
// x += alpha d; p = s + beta p (d = p in the CGLS arrangement, d = D^dag p in the paper's form)
cudaError_t launch_cg_update_xp(int prec, FieldPtr x, FieldPtr d, FieldPtr p, FieldPtr s, int n, int V,
                                CgScalars* sc, double* partials, int use_cond, unsigned long long cond, int block,
                                cudaStream_t st);
// Mixed precision (inner W = SP32 or SP16 spinors, x_lo in SP32, outer FP64)
cudaError_t launch_mp_update_rx(int precw, FieldPtr r, FieldPtr q, FieldPtr p, FieldPtr xlo, int n, int V,
                                CgScalars* sc, double* partials, int use_cond, unsigned long long upd, int block,
                                cudaStream_t st);
// skip: pointer to CgScalars::need_update; the kernel runs only when it is non-zero (nullptr = always)
cudaError_t launch_mp_accumulate(FieldPtr xhi, FieldPtr xlo, int n, int V, const int* skip, int block,
                                 cudaStream_t st);
cudaError_t launch_mp_convert(FieldPtr rhi, FieldPtr rlo, int n, int V, CgScalars* sc, double* partials, int count,
                              const int* skip, int block, cudaStream_t st);
cudaError_t launch_mp_update_p(int precw, FieldPtr p, FieldPtr s, int n, int V, CgScalars* sc, double* partials,
                               int use_cond, unsigned long long cond, int block, cudaStream_t st);
// zero `bytes` (multiple of 16) of device memory with a kernel
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st);

// ---------------------------------------------------------------- multiple right-hand sides

constexpr int kMaxRhs = 16;

// Per-RHS solver scalars for the multi-RHS CG (one per context).
// Multi-RHS reductions: at most kMaxMultiGrid blocks per right-hand-side group, summed in runs of
// kRedGroup blocks (see mreduce); the partials buffer holds kMultiPartials doubles.
constexpr int kMaxMultiGrid = 4096;
constexpr int kRedGroup = 32;
constexpr int kMaxMultiRuns = kMaxMultiGrid / kRedGroup;
constexpr size_t kMultiPartials =
    (size_t)kMaxRhs * kMaxMultiGrid + (size_t)kMaxRhs * kMaxMultiRuns + (size_t)kMaxRhs * kMaxMultiRuns / 2;

struct MCgScalars {
  double eta2[kMaxRhs], rr[kMaxRhs], qq[kMaxRhs], gamma[kMaxRhs], gamma_new[kMaxRhs];
  double alpha[kMaxRhs], rr_true[kMaxRhs], rr_ref[kMaxRhs];
  double tol2, delta2;
  int status[kMaxRhs];  // ST_* per right-hand side
  int iters[kMaxRhs];   // iterations in which the right-hand side was updated
  int need[kMaxRhs];    // mixed precision: reliable update requested
  int nrhs, iter, maxit, any_running, need_update, no_update, updates, pad;
  unsigned ticket[128];
};

// ticket slots: the per-group slots take kMaxRhs entries each
enum { TKM_DSLASH_A = 0, TKM_DSLASH_B = 16, TKM_DSLASH_C = 32, TKM_UPD_R = 48, TKM_UPD_XP = 64, TKM_PACK = 80,
       TKM_GROUPS = 96, TKM_GROUPS2 = 97, TKM_MISC = 112 };

struct MDslashCall {
  GeomH g;
  GaugePtr u;
  FieldPtr in, out, b;  // layout [unit][V][nrhs]
  double kappa;
  int dagger, epi;
  int nrhs;             // right-hand sides in the fields
  int group;            // K: right-hand sides per thread group (divides nrhs)
  int sites_per_block;  // group * sites_per_block <= 256
  int rhs_per_thread;   // KT: 0 or 1, or (FP32 / FP16) 2 or 4 right-hand sides per thread, sharing
                        // each link load; block = group / KT * sites_per_block
  int grid_x;           // blocks per group (grid-stride over sites)
  const int* status;    // optional per-RHS status mask (only ST_RUNNING computed)
  double* partials;     // >= nrhs * grid_x
  unsigned* tickets;    // >= nrhs / group counters
  double* result;       // optional per-RHS |out|^2
  const double* kappa_dev;  // optional: kappa read from device memory (overrides `kappa`)
};

cudaError_t launch_dslash_multi(const MDslashCall& c, cudaStream_t st);
// canonical N fields back to back (complex128 [N][V][12]) <-> [unit][V][N]; block = N * (256 / N)
cudaError_t launch_mpack(const double* canon, FieldPtr out, int V, int N, int grid_x, double* partials,
                         unsigned* tickets, double* result, cudaStream_t st);
cudaError_t launch_munpack(FieldPtr in, double* canon, int V, int N, int grid_x, cudaStream_t st);
cudaError_t launch_mcg_init(MCgScalars* sc, cudaStream_t st);
cudaError_t launch_mcg_check(MCgScalars* sc, int use_cond, unsigned long long cond, cudaStream_t st);
cudaError_t launch_mcg_update_r(int prec, FieldPtr r, FieldPtr q, FieldPtr p, FieldPtr xlo, int V, MCgScalars* sc,
                                double* partials, int N, int K, int spb, int grid_x, int mixed, int use_cond,
                                unsigned long long upd, cudaStream_t st);
cudaError_t launch_mcg_update_xp(int prec, FieldPtr x, FieldPtr p, FieldPtr s, int V, MCgScalars* sc, double* partials,
                                 int N, int K, int spb, int grid_x, int mixed, int use_cond, unsigned long long cond,
                                 cudaStream_t st);
cudaError_t launch_macc(FieldPtr xhi, FieldPtr xlo, int V, int N, int grid_x, cudaStream_t st);
cudaError_t launch_mconv(FieldPtr rhi, FieldPtr rlo, int V, int N, int grid_x, MCgScalars* sc, int count,
                         cudaStream_t st);

// Seeded generation (Philox4x32-10): links into the device layouts (any pointer may be null) and
// optionally the canonical complex128 copy; Gaussian source in the canonical layout.
cudaError_t launch_gen_gauge(int V, const GeomH* eo, double eps, unsigned long long seed, void* g64, void* g32,
                             int c12, double* canon, void* gdf, cudaStream_t st);
cudaError_t launch_gen_source(int V, unsigned long long seed, double* canon, cudaStream_t st);

// Even-odd half hopping: out = [b -] ([self] + sign * kappa * H in) on the sites of `parity`
// (fields in parity order, see wd_dslash.cu).
struct EoCall {
  GeomH g;
  GaugePtr u;
  FieldPtr in, out, self, b;
  int parity;
  double sign;
  int dagger;
  int use_self;
  int resid;
  const double* kappa_dev;
  const int* skip;
  Red red;
  int block;
};
cudaError_t launch_dslash_eo(const EoCall& c, cudaStream_t st);

// The paper's COO representation of D (49 non-zeros per row) and its atomic SpMV (wd_coo.cu).
cudaError_t launch_coo_build(const GeomH& g, const double* U, double kappa, int* row, int* col, double* val,
                             cudaStream_t st);
cudaError_t launch_coo_spmv(long long nnz, const int* row, const int* col, const double* val, const double* in,
                            double* out, long long nrows, cudaStream_t st);

// Double-float support: FP64 <-> double-float fields (to_df = 1: FP64 -> df), x_hi += x_lo with a
// double-float x_hi, and r_lo = hi part of a double-float residual (+ reliable-update bookkeeping).
cudaError_t launch_convert_f64_df(FieldPtr in, FieldPtr out, int n, int V, int to_df, int block, cudaStream_t st);
cudaError_t launch_mp_accumulate_df(FieldPtr xhi, FieldPtr xlo, int n, int V, const int* skip, int block,
                                    cudaStream_t st);
cudaError_t launch_mp_convert_df(FieldPtr rhi, FieldPtr rlo, int n, int V, CgScalars* sc, double* partials, int count,
                                 const int* skip, int block, cudaStream_t st);

// multi-RHS double-float: FP64 <-> df conversion (to_df = 1: FP64 -> df), x_hi += x_lo, r_lo = hi(r_hi)
cudaError_t launch_mconvert_df(FieldPtr f64, FieldPtr df, int V, int N, int grid_x, int to_df, cudaStream_t st);
cudaError_t launch_macc_df(FieldPtr xhi, FieldPtr xlo, int V, int N, int grid_x, cudaStream_t st);
cudaError_t launch_mconv_df(FieldPtr rhi, FieldPtr rlo, int V, int N, int grid_x, MCgScalars* sc, int count,
                            cudaStream_t st);

// grid size used by a launcher for V sites at a block size
inline int grid_for(int V, int block) { return (V + block - 1) / block; }

// Blocks of `block` threads of kernel `fn` resident on the current device at once (occupancy of
// the instantiation times the SM count; cached per device, kernel and block size).
inline int resident_blocks(const void* fn, int block) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  std::lock_guard<std::mutex> g(mu);
  const auto key = std::make_tuple(dev, fn, block);
  auto it = cache.find(key);
  if (it == cache.end()) {
    int nb = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, 0) != cudaSuccess || nb < 1) nb = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    cudaGetLastError();
    it = cache.emplace(key, nb * sms).first;
  }
  return it->second;
}

// Grid of a grid-stride launch over `sites`: one wave of resident blocks, or fewer when the
// sites do not fill it.
template <typename K>
inline int stride_grid(K kernel, int sites, int block) {
  const int need = grid_for(sites, block);
  const int res = resident_blocks(reinterpret_cast<const void*>(kernel), block);
  return need < res ? need : res;
}

}  // namespace wdk
