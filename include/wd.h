/*
 * wd.h -- C ABI of the GB300 Wilson-Dirac conjugate-gradient library.
 *
 * The library solves D psi = eta for the Wilson-Dirac operator D of Eq. (1) of arXiv 2111.14958
 * ("Implementation of the conjugate gradient algorithm for heterogeneous systems", Sec. 1), using
 * conjugate gradient on the normal equations (Sec. 2: the gamma_5-hermiticity gamma_5 D gamma_5 =
 * D^dagger turns the problem into a Hermitian one). The operator, in the hopping form with Wilson
 * parameter r = 1, is
 *
 *   (D psi)(n) = psi(n) - kappa sum_mu [ (1 - gamma_mu) U_mu(n) b psi(n + mu)
 *                                       + (1 + gamma_mu) U_mu(n - mu)^dagger b psi(n - mu) ]
 *
 * with mu = 0,1,2,3 = x,y,z,t, the chiral gamma basis (gamma_k = [[0,-i sigma_k],[i sigma_k,0]],
 * gamma_t = [[0,1],[1,0]]), and b = boundary[mu] for a hop that wraps around the lattice in
 * direction mu (else 1). D^dagger swaps the two projectors.
 *
 * Canonical (caller-visible) layouts, site index n = x + Lx*(y + Ly*(z + Lz*t)):
 *   spinor field : complex [Lt][Lz][Ly][Lx][4 spin][3 colour], interleaved (re, im)
 *                  -- complex128 (double pairs) unless a function says otherwise;
 *   gauge field  : complex128 [Lt][Lz][Ly][Lx][4 mu][3][3], U[n][mu] = U_mu(n), the link
 *                  n -> n + mu, row-major (row = first colour index).
 * Internally every field is converted to a site-blocked structure-of-arrays layout; callers never
 * see it.
 *
 * Conventions for every call:
 *   - Pointers to fields are DEVICE pointers (memory of the context's device) unless a parameter
 *     says otherwise. The library borrows them for the duration of the call and never frees them.
 *   - All work is enqueued on the stream given to wd_create; calls return after the work they
 *     enqueued has finished unless stated otherwise.
 *   - Every call returns a wd_status. On failure, wd_last_error() returns a message (per thread).
 *   - A context is not thread-safe: one thread at a time per context.
 */
#ifndef WD_H
#define WD_H

#include <stddef.h> /* size_t */

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wd_ctx wd_ctx; /* opaque: device gauge copies, Krylov workspace, CUDA graphs */

typedef enum {
  WD_OK = 0,
  WD_NOT_CONVERGED = 1,  /* maxit reached; outputs are filled with the last iterate       */
  WD_EINVAL = -1,        /* bad argument (null pointer, bad dims, bad precision, ...)    */
  WD_ENOMEM = -2,        /* device allocation failed                                      */
  WD_ECUDA = -3,         /* a CUDA runtime call failed                                    */
  WD_ENOTUNITARY = -4,   /* loaded links deviate from SU(3) beyond the stated bound       */
  WD_BREAKDOWN = -5,     /* non-finite or non-positive CG scalar (e.g. NaN in the source) */
  WD_ENOGAUGE = -6       /* an operator call before wd_load_gauge                          */
} wd_status;

/* Precision of the dslash and Krylov vectors (the `precision` argument of wd_create). */
enum {
  WD_PREC_F64 = 64,        /* plain FP64 CG: FP64 spinors, FP64 links, FP64 arithmetic             */
  WD_PREC_F32 = 32,        /* plain FP32 CG: FP32 spinors and links, FP64 reductions               */
  WD_PREC_MIXED_F32 = 6432,/* FP32 inner CG with FP64 reliable updates (FP64 solution, residual)   */
  WD_PREC_MIXED_F16 = 6416, /* FP16 spinors with per-site FP32 norm inside, FP64 reliable updates  */
  /* Flag ORed into any of the above: even-odd (Schur) preconditioning. Every extent must be even.
   * Fields are stored in parity order and cg_solve runs on M = 1 - kappa^2 H_eo H_oe over the even
   * sites (b_e = eta_e + kappa H_eo eta_o; x_o = eta_o + kappa H_oe x_e afterwards), with the same
   * tolerance on the full-system residual ||eta - D x|| / ||eta||. Multi-RHS calls are not
   * available on such a context. */
  WD_EVEN_ODD = 0x10000
};

/* Options for wd_set_option. */
enum {
  WD_OPT_RELIABLE_DELTA = 1, /* mixed precision: reliable update when |r| drops by this factor
                                (default 0.1), in (0, 1). Measured on 24^3x48 and 32^3x64 to
                                1e-10: 0.01 takes the iterations of 0.1 with half the updates
                                (10-12 % faster); FP16 inner solves need more iterations below
                                about 0.003                                                      */
  WD_OPT_USE_GRAPH = 2,      /* how cg_solve runs the CG loop: 0 plain stream launches with a
                                host poll; 1 a CUDA graph with a device-side while node; 2 a
                                persistent cooperative kernel for the loop (CGLS, or the paper's
                                CG form on the lexicographic layout with one thread per site;
                                mixed precision returns to the host for each reliable update;
                                mixed even-odd contexts and the even-odd paper form use the
                                graph); 3
                                (default) automatic: the persistent kernel for plain FP32 on
                                the lexicographic layout at every volume, for plain FP64 on it up
                                to 65,536 sites (its launch shape, 1 to 16 threads per site,
                                timed on the loop itself on first use), and for the other cases
                                it serves up to 48,000 sites, where it measured faster on GB300;
                                the graph otherwise                                              */
  WD_OPT_BLOCK_DSLASH = 3,   /* threads per block of the dslash kernel, 32..256 (0 = 256)       */
  WD_OPT_BLOCK_BLAS = 4,     /* threads per block of the BLAS-1 kernels (0 = default)            */
  WD_OPT_MAX_RESTARTS = 5,   /* max restarts from the true residual (default 5)                  */
  WD_OPT_MULTI_GROUP = 6,    /* multi-RHS: right-hand sides sharing one link load (K, divides
                                nrhs); 0 (default) = chosen by the autotuner                     */
  WD_OPT_MULTI_SITES = 7,    /* multi-RHS: sites per thread block (K * sites <= 256); 0 = tuned   */
  WD_OPT_DF_UPDATES = 8,     /* mixed precision: 1 (default) computes the reliable-update residual
                                and accumulates the solution in double-float arithmetic (pairs of
                                FP32, ~48 bits, on the FP32 pipes, ~2^-47 relative error per
                                operation); 0 uses native FP64. The final true residual is always
                                recomputed in native FP64. Changing it needs a gauge reload.     */
  WD_OPT_APPLY_DF = 9,       /* mixed precision: 1 makes wd_apply use the double-float operator
                                (complex128 in and out), to check it; 0 (default) native FP64     */
  WD_OPT_CG_FORM = 10,       /* plain FP64 / FP32 contexts, single right-hand side: 0 (default)
                                CG on D^dag D x = D^dag eta (CGLS arrangement); 1 the paper's
                                form (Sec. 2): CG on D D^dag y = eta with x = D^dag y, carried in
                                x directly (x += alpha D^dag p), so x on input is the initial
                                guess in both forms. Same two operator applications, stopping
                                rule and true residual; mixed-precision contexts reject 1. The
                                paper's form needs three grid barriers per iteration in the
                                persistent loop, CGLS four.                                      */
  WD_OPT_DSLASH_VARIANT = 11,/* FP64 single-RHS dslash (FP64 contexts, and the reliable updates
                                of mixed ones), also inside the persistent CG loop: 0 (default)
                                chosen with the block size on first use (the wider splits are
                                tried up to 65,536 sites); 1 one thread per site; 2 two threads
                                per site (each owns one half-spinor row); 3, 4, 5: 4, 8 or 16
                                threads per site (one direction, one hop, or one hop and one
                                half-spinor row each, summed by shuffles). Lexicographic layout
                                only: even-odd contexts ignore it.                               */
  WD_OPT_LOOP_WAIT_LIMIT = 12,/* persistent loop: polls of 64 ns before a grid-barrier wait gives
                                up and cg_solve returns WD_ECUDA ("a grid barrier wait gave
                                up"), leaving the context usable; 0 or 2^26 (default, about
                                4 s). Small values exercise that failure path.                  */
  WD_OPT_RESIDUAL_HISTORY = 13,/* cg_solve records the recursive residual of its first N
                                iterations (N = value, 0 = off, the default) for
                                wd_get_residual_history                                          */
  WD_OPT_APPLY_INNER = 14,   /* mixed precision: 1 makes wd_apply and wd_apply_multi run the inner
                                solver's operator (complex128 in and out): the input is rounded
                                into the working precision (FP32, or FP16 with a per-site FP32
                                norm), D is applied with the FP32 links (12-real if loaded so)
                                and the working-precision result is widened to complex128; 0
                                (default) the FP64 operator                                      */
  WD_OPT_MULTI_RHS_PER_THREAD = 15, /* multi-RHS, FP32 / FP16 working precision: right-hand sides
                                held by one thread of the dslash, which loads and rebuilds each link
                                once for all of them (1, 2 or 4; must divide the group K and not
                                exceed the sites per block); 0 (default) = chosen by the autotuner */
  WD_OPT_DSLASH_TMA = 16,    /* FP32 working precision, lexicographic layout: 1 or 2 makes the
                                stand-alone operator (wd_apply, wd_time_dslash) stage the neighbour
                                spinors in shared memory by TMA bulk tensor copies, in tiles of
                                Lx x 2 x 2 x 2 (1) or Lx x 4 x 2 x 2 (2) sites, when the FP32 links
                                are 12-real (per-thread loads otherwise); needs Lx a multiple of 4
                                up to 64 and the other extents divisible by the tile. A copy that
                                does not land within its wait limit makes the call return
                                WD_ECUDA. 0 (default): per-thread neighbour loads. Solves ignore it */
  WD_OPT_DSLASH_SCHEDULE = 17,/* FP32 / FP16 working precision, lexicographic layout, the stand-alone
                                dslash launches (wd_apply, the graph and host-loop solvers): the
                                order of its loads. 1: hop by hop; 2: two sites per thread, each
                                hop's loads for both issued before either's arithmetic; 3: both
                                hops of each direction loaded before their arithmetic (1 and 3
                                at three and two blocks per SM). The same bits in every schedule.
                                0 (default): 1 or 3, timed with the block size on first use
                                (2 is never chosen: slower wherever measured on GB300)          */
  WD_OPT_LOOP_TIME_BASIS = 18 /* plain FP64 contexts, lexicographic layout, the persistent CG loop
                                with one thread per site: 1 (default) runs the loop in the spin
                                basis psi' = T psi, T = [[1, 1], [-1, 1]] on (upper, lower) spins,
                                where gamma_t of the chiral basis is diagonal and the spatial
                                gammas are unchanged (the operator is T D T^-1 of Eq. (1)), so a
                                time hop needs no spin projection, and with the time links
                                pre-scaled by the loop (2 x -kappa x the boundary phase, in a
                                buffer of the context) no separate scaling either: 789 instead of
                                849 FP64 operations per site and dslash. x, r, p, s enter the
                                basis in the loop kernel and leave it when the loop ends; cg_solve's inputs,
                                outputs, true residual and stopping rule are unchanged, and the
                                iterates equal the chiral ones up to rounding. 0: the chiral
                                basis throughout                                                 */
};

/* Per-solve statistics, filled by wd_get_stats after cg_solve. */
typedef struct {
  int iterations;          /* CG iterations (each = 2 dslash applications)                    */
  int restarts;            /* relaunches from the recomputed true residual                     */
  int reliable_updates;    /* mixed precision: FP64 residual recomputations                    */
  int dslash_calls;        /* dslash applications, all precisions                              */
  int dslash_calls_f64;    /* of which in FP64                                                  */
  int status;              /* wd_status of the solve                                            */
  int loop_mode;           /* how the CG loop ran: 0 host loop, 1 CUDA graph, 2 persistent kernel */
  int loop_lanes;          /* persistent FP64 loop: threads per lattice site (1, 2, 4, 8 or 16)   */
  double true_rel_residual;/* ||eta - D x|| / ||eta||, recomputed in the outer precision         */
  double solve_ms;         /* host wall time of cg_solve                                          */
  double loop_ms;          /* persistent kernel (loop_mode 2): its device time (CUDA events), all
                              passes; 0 for the other modes                                     */
} wd_stats;

/* Statistics of the last cg_solve_multi / wd_apply_multi, filled by wd_get_multi_stats. */
typedef struct {
  int nrhs;
  int iterations;          /* loop iterations until every right-hand side stopped               */
  int restarts;
  int reliable_updates;    /* mixed precision: FP64 residual recomputations (all RHS at once)   */
  int group;               /* K: right-hand sides per thread group sharing one link load         */
  int sites_per_block;
  int status;
  int rhs_per_thread;      /* KT: right-hand sides per thread of the working-precision dslash     */
  double solve_ms;         /* host wall time of the solve                                       */
  double dslash_ms;        /* one multi-RHS dslash launch at the tuned shape (working precision) */
} wd_multi_stats;

/*
 * Create a context for a lattice.
 *   dims[4]     : Lx, Ly, Lz, Lt; each >= 2 (for L = 2 the two hops land on the same site and
 *                 both terms of Eq. (1) are added), V = Lx*Ly*Lz*Lt <= 2^27.
 *   kappa       : hopping parameter (finite, |kappa| < 1).
 *   boundary[4] : +1 periodic or -1 antiperiodic per direction; NULL means (1, 1, 1, -1).
 *   precision   : one of WD_PREC_*.
 *   cuda_stream : cudaStream_t to enqueue on (NULL = the legacy default stream).
 *   out         : receives the context. Allocates the device workspace (about 8 spinor fields
 *                 of the working precision plus the gauge copies).
 * Errors: WD_EINVAL, WD_ENOMEM, WD_ECUDA.
 */
wd_status wd_create(const int dims[4], double kappa, const int boundary[4], int precision,
                    void* cuda_stream, wd_ctx** out);

/* Change the hopping parameter of an existing context (|kappa| < 1). Every later operator
 * application and solve uses it; links, workspace and graphs are kept. */
wd_status wd_set_kappa(wd_ctx* ctx, double kappa);

/* Free every device resource of the context. Null is ignored. */
void wd_destroy(wd_ctx* ctx);

/*
 * Load the gauge field U (links of Eq. (1); canonical complex128 layout above).
 *   U          : host pointer if on_device == 0, else device pointer; V*4*9 complex128.
 *   compress12 : 1 stores FP32 links of the inner solver (or of a WD_PREC_F32 context) as
 *                12 reals (rows 0 and 1; row 2 = conj(row0 x row1) rebuilt in the kernel);
 *                FP64 links are always stored as 18 reals.
 *   max_unitarity_dev : optional out (host pointer): max over links of max(|U^dag U - 1|_max,
 *                 |det U - 1|). Returns WD_ENOTUNITARY (data still loaded) if it exceeds 1e-6
 *                 and compress12 == 1, since the 12-real reconstruction assumes SU(3).
 */
wd_status wd_load_gauge(wd_ctx* ctx, const double* U, int on_device, int compress12,
                        double* max_unitarity_dev);

/*
 * out = D in (dagger == 0) or D^dagger in (dagger != 0), Eq. (1).
 *   in, out : device spinor fields in the canonical layout; complex128 for WD_PREC_F64 and the
 *             mixed modes (FP64 operator, or the inner one under WD_OPT_APPLY_INNER), complex64
 *             for WD_PREC_F32. in != out.
 * Errors: WD_EINVAL, WD_ENOGAUGE, WD_ECUDA.
 */
wd_status wd_apply(wd_ctx* ctx, const void* in, void* out, int dagger);

/*
 * Solve D x = src by CG on D^dagger D x = D^dagger src (CGLS arrangement: two dslash per
 * iteration, Sec. 2), stopping when the recursive ||r|| / ||src|| <= tol, then recomputing the
 * true residual ||src - D x|| / ||src|| and restarting from it while it exceeds tol (up to
 * WD_OPT_MAX_RESTARTS times, within maxit total iterations).
 *   src       : device, complex128 canonical.
 *   x         : device, complex128 canonical; initial guess on input, solution on output.
 *   tol       : > 0 relative tolerance; maxit: >= 0, <= 10^7.
 *   iters, true_rel_res : optional host outs.
 * Returns WD_OK, WD_NOT_CONVERGED (x holds the last iterate), WD_BREAKDOWN (non-finite source or
 * scalar; x holds the last finite iterate), WD_EINVAL, WD_ENOGAUGE, WD_ECUDA.
 */
wd_status cg_solve(wd_ctx* ctx, const void* src, void* x, double tol, int maxit, int* iters,
                   double* true_rel_res);

/*
 * cg_solve_batch -- n independent solves (one per context) as cg_solve would run each alone.
 *
 * No counterpart in the paper, which runs one solve at a time: this is the batching of the serving
 * runtime below, open to callers with several problems of one shape. When every context has the
 * same lattice, boundary, precision (mixed, plain FP32, or plain FP64 on the lexicographic layout)
 * and launch shape, and its CG loop is the persistent kernel (WD_OPT_USE_GRAPH), each pass runs the
 * contexts' prologues, ONE cooperative launch of the loop for all of them (problem i on its own
 * blocks, with its own fields, links, kappa, tolerance, scalars and grid barrier, and the grid its
 * solve alone uses) and their epilogues, all on ctxs[0]'s stream; reliable updates and restarts are
 * per problem. Every result (x, iterations, residual) is therefore bitwise the result of cg_solve
 * on that context alone. Otherwise the problems are solved one after another with cg_solve's path.
 *   ctxs[n], srcs[n], xs[n] : n distinct contexts (1 <= n <= 64) and their device fields as in
 *                             cg_solve (x: initial guess in, solution out);
 *   tols[n]                 : per-problem tolerance; maxit: shared iteration limit;
 *   iters, true_rel_res, statuses : optional host arrays of n (statuses: each problem's wd_status).
 * Returns WD_OK if every problem converged, WD_BREAKDOWN if any broke down, else WD_NOT_CONVERGED if
 * any reached maxit; WD_EINVAL, WD_ENOGAUGE, WD_ECUDA as cg_solve. Each context is used by this call
 * alone while it runs.
 */
wd_status cg_solve_batch(wd_ctx* const* ctxs, int n, const void* const* srcs, void* const* xs, const double* tols,
                         int maxit, int* iters, double* true_rel_res, int* statuses);

/*
 * Checkpoint and resume of a CG solve. The paper's CG (Sec. 2, the iteration carries x, r, p and
 * gamma from one step to the next) has no checkpoint; this lets a caller stop a long solve after
 * maxit iterations, keep its state in host memory (to give the GPU to other work, or to free the
 * context), and continue it later from exactly that iteration. Plain FP64 and FP32 contexts
 * (lexicographic or even-odd, either CG form); mixed-precision contexts return WD_EINVAL.
 *
 * wd_cg_state_size -- *bytes = size of a saved state for this context (a header, then x, r and p
 *   in the context's device layout: 3 x 192 B per site in FP64, 3 x 96 B in FP32).
 *
 * wd_cg_save_state -- copies the state into `host` (caller-owned host memory of >= that size;
 *   pageable or pinned). Valid only right after a cg_solve or cg_resume on this context that
 *   returned WD_NOT_CONVERGED because its CG loop reached maxit, and before any call that changes
 *   the context's fields or operator (wd_apply, wd_apply_multi, cg_solve_multi, wd_time_dslash,
 *   wd_load_gauge, wd_generate_gauge, wd_set_kappa, a new solve); otherwise WD_EINVAL. The state
 *   is opaque and tied to this library build.
 *
 * cg_resume -- continues the saved state on `ctx` (the same context or a new one with the same
 *   lattice, boundary, precision and kappa, with the same gauge field loaded; WD_EINVAL if the
 *   header does not match): no new starting residual is formed; the iteration goes on from the
 *   saved x, r, p, gamma and iteration count until the recursive residual meets tol, then the true
 *   residual is checked and restarts follow as in cg_solve.
 *   state, bytes : the saved state (host) and its size (>= wd_cg_state_size).
 *   src          : device, complex128 canonical: the source of the saved solve.
 *   x            : device, complex128 canonical; output only (the saved iterate is the start).
 *   tol, maxit   : as in cg_solve; maxit counts the iterations done before the save as well.
 *   iters, true_rel_res : optional host outs (iters: total, including those before the save;
 *                         so are the iteration and dslash counts of wd_get_stats afterwards).
 * On the same context and launch shape, a resumed solve computes bitwise what the uninterrupted
 * solve computes, except in the FP64 persistent loop's time-diagonal basis (WD_OPT_LOOP_TIME_BASIS),
 * whose state leaves and re-enters that basis at the stop (equal to rounding). Returns as cg_solve.
 */
wd_status wd_cg_state_size(const wd_ctx* ctx, size_t* bytes);
wd_status wd_cg_save_state(wd_ctx* ctx, void* host, size_t bytes);
wd_status cg_resume(wd_ctx* ctx, const void* state, size_t bytes, const void* src, void* x, double tol, int maxit,
                    int* iters, double* true_rel_res);

/*
 * Multiple right-hand sides sharing the operator (a propagator's 12 spin-colour sources, say).
 * Fields are nrhs canonical complex128 spinor fields back to back ([nrhs][Lt][Lz][Ly][Lx][4][3]),
 * 1 <= nrhs <= 16. The multi-RHS dslash maps the K right-hand sides of a group to consecutive
 * threads that read each link once; K and the block shape are autotuned on first use for a given
 * nrhs (timed with CUDA events on the context stream) unless fixed with WD_OPT_MULTI_*.
 *
 * wd_apply_multi: out_r = D in_r (or D^dagger), in the context's operator precision (FP64 for
 *   WD_PREC_F64 and the mixed modes, FP32 arithmetic on rounded inputs for WD_PREC_F32; the inner
 *   FP32 / FP16 operator of a mixed context under WD_OPT_APPLY_INNER).
 * cg_solve_multi: solves D x_r = src_r for every r with the context's solver (plain FP64, plain
 *   FP32, or mixed precision with FP64 reliable updates applied to all right-hand sides at once
 *   whenever one of them has dropped by delta), each right-hand side stopping on its own
 *   tolerance; iters[r] and true_rel_res[r] (optional host arrays of nrhs) receive the iterations
 *   each took and its true residual ||src_r - D x_r|| / ||src_r||.
 * Returns WD_OK when every right-hand side converged, WD_NOT_CONVERGED if any reached maxit,
 * WD_BREAKDOWN if any broke down (the others are still solved), WD_EINVAL, WD_ENOGAUGE,
 * WD_ENOMEM (workspace: about 8 fields of nrhs right-hand sides), WD_ECUDA.
 */
wd_status wd_apply_multi(wd_ctx* ctx, const double* in, double* out, int nrhs, int dagger);
wd_status cg_solve_multi(wd_ctx* ctx, const double* src, double* x, int nrhs, double tol, int maxit, int* iters,
                         double* true_rel_res);
wd_status wd_get_multi_stats(const wd_ctx* ctx, wd_multi_stats* out);

/*
 * Seeded synthetic inputs generated on the device (the paper's lattices come with no gauge
 * ensembles). Random numbers: Philox4x32-10 (Salmon et al., SC11) keyed by `seed`, Box-Muller
 * Gaussians. wd_generate_gauge draws every link as U = exp(i eps H), H the traceless Hermitian part
 * of a matrix with N(0,1) real and imaginary entries, re-unitarised to SU(3), straight into the
 * context's device layouts (as wd_load_gauge would store them; compress12 as there), and also
 * writes the canonical complex128 field to U_out if it is not NULL (device pointer).
 * wd_generate_source writes a complex Gaussian spinor field (Re, Im ~ N(0,1)) to `out` (device,
 * canonical complex128). The same streams are reproducible on a CPU (synthetic/ in this
 * repository). Errors: WD_EINVAL, WD_ENOMEM, WD_ECUDA.
 */
wd_status wd_generate_gauge(wd_ctx* ctx, double eps, unsigned long long seed, int compress12, double* U_out);
wd_status wd_generate_source(wd_ctx* ctx, unsigned long long seed, double* out);

/*
 * Serving: a persistent request loop with continuous admission and batching (no counterpart in the
 * paper, which runs one solve at a time). Each request is one single-RHS solve with its own
 * lattice, kappa, tolerance, seeded gauge field (wd_generate_gauge with eps, gauge_seed) and source
 * (seeded Gaussian, or src_host). A scheduler admits queued requests into `slots` execution slots
 * as slots free up and as device memory allows (an estimate of each request's footprint is charged
 * against budget_bytes): the oldest waiting request first, together with up to max_batch - 1 later
 * requests of the same operator (lattice, precision, boundary, maxit) whose CG loop is the
 * persistent kernel (plain FP32; plain FP64 up to 65,536 sites; mixed precision up to 48,000 sites
 * on the lexicographic layout), which the slot solves with cg_solve_batch. Every slot has its own
 * CUDA stream and host thread, so admitted work overlaps on the device; a slot keeps the contexts it
 * created resident (least recently used ones are evicted when new ones do not fit), and requests
 * whose operator matches an idle slot's resident contexts go there first (no allocation or graph
 * rebuild). Every result is bitwise the result of the same solve alone (same fields, same solver,
 * same launch shapes), batched or not.
 *
 * wd_server_submit queues a request (returns its id at once); wd_server_wait blocks until it is
 * done; wd_server_poll returns immediately (*done = 0/1). A finished result is returned once and
 * then forgotten. wd_server_set_max_batch sets the batch limit (1..16; 1 = no batching; default 8).
 * wd_server_set_policy chooses the request admitted next: 0 (default) the oldest; 1 the one with
 * the least estimated work (sites times a per-precision factor) unless the oldest has waited more
 * than max_wait_ms, which then goes first (no request waits unboundedly behind smaller ones).
 * wd_server_destroy finishes running solves, drops queued ones and frees all.
 * Errors: WD_EINVAL (bad request), WD_ENOMEM (a request larger than the whole budget), WD_ECUDA.
 */
typedef struct wd_server wd_server;

typedef struct {
  int dims[4];
  double kappa;
  double eps;                      /* link spread of the generated gauge field                 */
  unsigned long long gauge_seed;
  unsigned long long source_seed;  /* ignored when src_host is set                             */
  double tol;
  int maxit;
  int precision;                   /* WD_PREC_*                                                */
  int boundary_set;                /* 0: boundary (1, 1, 1, -1); 1: use boundary[]             */
  int boundary[4];
  const double* src_host;          /* optional host source, canonical complex128               */
  double* x_host;                  /* optional host buffer for the solution, canonical          */
} wd_request;

typedef struct {
  int status;                      /* wd_status of the solve                                    */
  int iterations;
  int reliable_updates;
  int slot;                        /* execution slot that ran it                                */
  double true_rel_residual;
  double queue_ms;                 /* submit -> start                                           */
  double solve_ms;                 /* start -> done (fields generated, solved, copied out)      */
  double latency_ms;               /* submit -> done                                            */
  int batch;                       /* requests solved together in its batch (1 = alone)         */
} wd_result;

typedef struct {
  long long submitted, admitted, completed, failed;
  long long warm_hits;             /* requests that ran on an already resident context          */
  long long evictions;             /* resident contexts freed to make room                      */
  int pending;
  double used_bytes, peak_bytes;   /* device memory charged to resident contexts                */
  long long batches;               /* batches of two or more requests run                        */
  long long batched_requests;      /* requests that ran in such batches                          */
} wd_server_stats;

wd_status wd_server_create(double budget_bytes, int slots, wd_server** out);
wd_status wd_server_submit(wd_server* srv, const wd_request* req, long long* id);
wd_status wd_server_wait(wd_server* srv, long long id, wd_result* out);
wd_status wd_server_poll(wd_server* srv, long long id, wd_result* out, int* done);
wd_status wd_server_set_max_batch(wd_server* srv, int max_batch);
wd_status wd_server_set_policy(wd_server* srv, int policy, double max_wait_ms);
wd_status wd_server_get_stats(wd_server* srv, wd_server_stats* out);
void wd_server_destroy(wd_server* srv);

/*
 * The paper's own method, for comparison on the same GPU (Sec. 2): D in coordinate format and
 * its sparse matrix-vector product. wd_coo_build writes the 49 * 12 * V non-zeros of D (the
 * context's kappa and boundary; U = device canonical complex128 links) into device arrays Row,
 * Col (int32, indices of the canonical vector 12*site + 3*spin + colour) and Val (complex128),
 * ordered by row; capacity = their length in entries, *nnz receives 49 * 12 * V. wd_coo_spmv
 * computes out[Row[k]] += Val[k] * in[Col[k]] over k < nnz, one thread per non-zero with atomic
 * accumulation into the zeroed `out` (canonical complex128; summation order is not fixed).
 * Errors: WD_EINVAL, WD_ECUDA.
 */
wd_status wd_coo_build(wd_ctx* ctx, const double* U, int* row, int* col, double* val, long long capacity,
                       long long* nnz);
wd_status wd_coo_spmv(wd_ctx* ctx, long long nnz, const int* row, const int* col, const double* val,
                      const double* in, double* out);

/* Recursive relative residual ||r_k|| / ||eta|| after each CG iteration k of the last cg_solve
 * (the residual the stopping rule tests: in mixed precision that of the inner solver, before any
 * reliable update of that iteration), for the first min(iterations, WD_OPT_RESIDUAL_HISTORY,
 * max_entries) iterations. out: host array of max_entries doubles; *count: entries written.
 * Returns WD_EINVAL for null pointers or a negative length. */
wd_status wd_get_residual_history(const wd_ctx* ctx, double* out, int max_entries, int* count);

/* Set an option (WD_OPT_*). Returns WD_EINVAL for an unknown key or a value out of range. */
wd_status wd_set_option(wd_ctx* ctx, int key, double value);

/* Statistics of the last cg_solve on this context. */
wd_status wd_get_stats(const wd_ctx* ctx, wd_stats* out);

/*
 * Time the dslash kernel as the CG launches it: `launches` back-to-back launches on the
 * context's internal vectors (dagger as given), bracketed by CUDA events on the context's
 * stream. *avg_ms receives the mean duration of one launch. Requires a loaded gauge field.
 */
wd_status wd_time_dslash(wd_ctx* ctx, int dagger, int launches, double* avg_ms);

/*
 * wd_dslash_noalloc -- out = D in (or D^dagger in) and, optionally, ||out||^2, without allocating.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot call cudaMalloc
 * (code under a framework or pooled allocator that must own every device allocation, plug-ins
 * handed fixed buffers). Such callers cannot create a wd_ctx, so everything is passed in:
 *   dims, kappa, boundary : as for wd_create (boundary NULL = (1, 1, 1, -1)); V <= 2^20 sites.
 *   U    : device, canonical complex128 links [V][4][3][3] (read in place, not converted).
 *   in   : device, canonical complex128 spinor [V][4][3];  out: device, same layout, != in.
 *   norm2_out : device pointer to one double receiving ||out||^2, or NULL for none.
 *   cuda_stream : stream to enqueue on (NULL = legacy default stream).
 * The call only enqueues work (no synchronisation); results are ready when the stream reaches it.
 * The norm's scratch (one partial per 128-site block and a counter, 64 KiB + 256 B) is a fixed
 * array in the library's device memory, held on every GPU that loads the library until the
 * process exits. The first call on each device looks up that array's device address (a one-time
 * set-up per device); make that first call before any stream capture. Every call shares the one
 * array, so calls whose kernels overlap on the GPU (different streams, concurrent threads) race
 * and give wrong norms; serialise them. The cached address belongs to the device's primary context:
 * resetting the device (cudaDeviceReset) after the first call is not supported. The call allocates
 * nothing: no cudaMalloc/cudaFree and no allocating library routine.
 * Errors: WD_EINVAL (null pointer, bad dims, V > 2^20, bad kappa or boundary, in and out
 * overlapping), WD_ECUDA (device or launch failure).
 */
wd_status wd_dslash_noalloc(const int dims[4], double kappa, const int boundary[4], const double* U,
                            const double* in, double* out, int dagger, double* norm2_out,
                            void* cuda_stream);

/*
 * wd_measure_fp64_peak -- FP64 fused multiply-add throughput of the current device, in TFLOP/s.
 *
 * A cross-check of the compute ceiling pi of the roofline P = min(pi, beta I) (Eq. (2), Sec. 3.1)
 * for the FP64 kernels, which on GB300 are bound by the FP64 pipe: a probe kernel runs 8 independent
 * chains of dependent FMAs per thread on 4 blocks of 256 threads per SM and is timed with CUDA events
 * on cuda_stream (NULL = legacy default stream); *tflops receives 2 flops per FMA over the fastest of
 * `repeats` launches (1..1000) after one warm-up launch. On GB300 it reads about 84 % of the unit
 * count (2 DFMA per clock per SM), which the FP64 dslash's mix of instructions comes within 5 % of.
 * Allocates nothing. Errors: WD_EINVAL, WD_ECUDA.
 */
wd_status wd_measure_fp64_peak(void* cuda_stream, int repeats, double* tflops);

/* Message of the last failing call on this thread ("" if none). */
const char* wd_last_error(void);

/* Library version string. */
const char* wd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WD_H */
