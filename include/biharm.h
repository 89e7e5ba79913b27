/*
 * biharm.h -- C ABI of the GB300 multigrid library for the C0 interior-penalty
 * (C0IP) discretization of the clamped biharmonic problem on (0,1)^d
 * (Sec. 2 of "Tensor-product vertex patch smoothers for biharmonic problems",
 * arXiv 2412.05082), with Q_k elements on uniform Cartesian meshes.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - A context owns one multigrid hierarchy: levels l = 1..L, level l has
 *    N = 2^l cells per direction (the coarsest mesh of 2^d cells is one vertex
 *    patch, Sec. 5.1).  Its unknowns are the interior support points,
 *    n = (k N - 1)^d values, stored lexicographically with x fastest.  The
 *    Q_k support points are the Gauss-Lobatto-Legendre points.
 *  - Pointers named *_dev are device pointers owned by the caller: FP64,
 *    contiguous, with the size of the level they refer to.  The library never
 *    frees or keeps them.  Pointers named *_host are host pointers.
 *  - Work is enqueued on the CUDA stream given to bh_create and is
 *    asynchronous unless stated otherwise.  Calls on one context must not
 *    overlap (a context is not thread-safe); distinct contexts are
 *    independent.
 *  - Every call returns a bh_status.  On failure a message is available from
 *    bh_last_error() (thread-local).  The library never aborts, never prints,
 *    never traps on the device, and has no CPU fallback: without a usable
 *    CUDA device bh_create fails with BH_ECUDA.
 */
#ifndef BIHARM_H
#define BIHARM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bh_ctx bh_ctx;

typedef enum {
  BH_OK = 0,
  BH_EINVAL = -1,    /* bad argument (size, level, null pointer, option) */
  BH_ENOMEM = -2,    /* device or host allocation failed */
  BH_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed */
  BH_ENOCONV = -4,   /* the Krylov solver did not reach the tolerance */
  BH_ETIMEOUT = -5,  /* a bounded wait ran out (server: a request's deadline passed) */
  BH_EBUSY = -6,     /* resource in use (server queue full) */
  BH_ECANCELED = -7  /* the request was cancelled before it started */
} bh_status;

/* smoother (Sec. 3): additive vertex-patch smoother with atomic or colored
 * writes (Sec. 5), or the colored multiplicative one. */
enum { BH_AVS_ATOMIC = 0, BH_AVS_COLORED = 1, BH_MVS_COLORED = 2 };
/* local solver: fast diagonalization of the separable A~_v
 * (Eq. (localsolverbila), Sec. 4.1) or the exact inverse of A_v (Sec. 3). */
enum { BH_FDM = 0, BH_EXACT = 1 };
/* precision of the V-cycle: FP64, or FP32 inside FP64 GMRES (Sec. 5.2).
 * BH_MIXED_FP32_R64 keeps the FP32 smoothing, transfers and storage of
 * BH_MIXED_FP32 but evaluates the defect b_l - A_l x before each restriction
 * in FP64 arithmetic (from the FP32 iterate) and restricts it in FP64: the
 * FP32 rounding error of A x is amplified by the coarse-grid correction like
 * the condition number of A_l, which stalls the plain FP32 V-cycle on fine
 * meshes at high degree (2D k >= 5 on 256^2 cells).  BH_MIXED_FP32_RC is
 * BH_MIXED_FP32_R64 with that defect evaluated in compensated FP32
 * arithmetic instead of FP64: every value of the sum factorization is a pair
 * hi + lo of floats, every 1D coefficient c is stored as fl32(c) plus
 * fl32(c - fl32(c)), products with the FP32 iterate are made exact by FMA and
 * sums by TwoSum, so the defect is accurate to about (terms) 2^-48 of
 * sum |terms| (FP64: 2^-53, FP32: 2^-24); the FP64 pipe, which issues 1/64 of
 * the FP32 rate on this GPU, is used only for the final b - (hi + lo).  The
 * restriction stays FP64.  Neither form is in the paper. */
enum { BH_FP64 = 0, BH_MIXED_FP32 = 1, BH_MIXED_FP32_R64 = 2, BH_MIXED_FP32_RC = 3 };
/* GMRES preconditioning side (Sec. 5.1 leaves it open).  BH_RIGHT (the
 * default) keeps the preconditioned directions (flexible form) and stops on the
 * true residual b - A x; its FP64 rounding floor eps ||A|| ||x|| / ||b|| is
 * O(eps) when b = A x* for a rough x*, but exceeds 1e-8 for an i.i.d. random b
 * on the paper's finest meshes (1e-8 .. 3e-7).  BH_LEFT stops on the reduction
 * of the preconditioned residual M^-1 (b - A x), the convention whose iteration
 * counts match the paper's tables. */
enum { BH_RIGHT = 0, BH_LEFT = 1 };
/* Krylov method of bh_solve (Sec. 5.1 pairs conjugate gradients with the
 * additive smoother, whose V-cycle is symmetric, and GMRES with the
 * multiplicative one). */
enum { BH_GMRES = 0, BH_CG = 1 };
/* coarse solver on level 1: the exact dense solve, or a single step of the
 * level's smoother (Sec. 5.1). */
enum { BH_COARSE_EXACT = 0, BH_COARSE_SMOOTH = 1 };
/* right-hand sides for bh_rhs. */
enum { BH_RHS_MANUFACTURED = 0, BH_RHS_PAPER_SINE = 1 };

typedef struct {
  int dim;           /* d = 2 or 3 */
  int degree;        /* k = 2..7 */
  int level;         /* finest level L >= 1 (N = 2^L) */
  double gamma;      /* penalty constant of Eq. (bfc0ip), used as gamma/h; <= 0: k(k+1) */
  int smoother;      /* BH_AVS_ATOMIC | BH_AVS_COLORED | BH_MVS_COLORED */
  int local_solver;  /* BH_FDM | BH_EXACT */
  int pre_steps;     /* smoothing steps before / after the coarse correction */
  int post_steps;
  double omega;      /* damping; <= 0: Sec. 5.1 defaults (AVS 1/4 in 2D, 0.1 in 3D
                        (1/8 exact); MVS 1 in 2D, 0.7 in 3D) */
  int precision;     /* BH_FP64 | BH_MIXED_FP32 | BH_MIXED_FP32_R64 | BH_MIXED_FP32_RC
                        (mixed forms need gmres_side = BH_RIGHT, or krylov = BH_CG) */
  int gmres_restart; /* restart length m (default 50) */
  int gmres_side;    /* BH_RIGHT (default) | BH_LEFT */
  int coarse;        /* BH_COARSE_EXACT (default) | BH_COARSE_SMOOTH */
  int krylov;        /* BH_GMRES (default) | BH_CG (additive smoothers only) */
} bh_params;

/* Fill *out with the defaults above for (dim, degree, level): MVS, FDM,
 * one pre- and one post-smoothing step, FP64, GMRES(50), right side.
 * Host only.  BH_EINVAL for d not in {2,3}, k not in 2..7 or level < 1. */
bh_status bh_default_params(int dim, int degree, int level, bh_params* out);

/* Create a context: host setup of the 1D data in FP64 (Eq. (matrix1d),
 * Sec. 4.1: 1D mass/stiffness/bulk-and-face matrices, the generalized
 * eigenpairs B s = lambda M s, the dense coarse inverse), allocation of every
 * level's device buffers and the GMRES workspace.  stream: a cudaStream_t
 * (NULL = legacy default stream).  The context is returned in *out and must be
 * released with bh_destroy.  Synchronous. */
bh_status bh_create(const bh_params* params, void* stream, bh_ctx** out);

/* Release every device and host resource of ctx (synchronizes its stream). */
bh_status bh_destroy(bh_ctx* ctx);

/* Number of unknowns (k 2^level - 1)^d of a level. Host only. */
bh_status bh_num_unknowns(const bh_ctx* ctx, int level, int64_t* n);

/* y = A_l x: the C0IP operator of Eq. (bfc0ip) on level l, applied
 * matrix-free by sum factorization of its Kronecker form Eq. (c0iptensorvp)
 * (2D) / Eq. (c0iptensorvp3D) (3D).  x_dev and y_dev: n(l) values, must not
 * alias. */
bh_status bh_apply_A(bh_ctx* ctx, int level, const double* x_dev, double* y_dev);

/* r = b - A_l x (Algorithm 1, restriction step).  r_dev must not alias x_dev. */
bh_status bh_residual(bh_ctx* ctx, int level, const double* x_dev, const double* b_dev,
                      double* r_dev);

/* r = b - A_l x for an FP32 iterate x_dev (n(l) floats) and an FP64 b_dev, in
 * the compensated FP32 arithmetic of BH_MIXED_FP32_RC (the defect that form
 * restricts, Algorithm 1's restriction step): the result differs from the
 * exact defect of (double) x by about (terms) 2^-48 of (|A_l| |x| + |b|).  The
 * context must have a mixed precision (it uses the FP32 tables' hi + lo
 * parts).  r_dev (n(l) doubles) must not alias x_dev; it may be b_dev.
 * BH_EINVAL for an FP64 context.  Not in the paper. */
bh_status bh_defect_compensated(bh_ctx* ctx, int level, const float* x_dev, const double* b_dev,
                                double* r_dev);

/* steps smoothing steps x <- S_l(x, b) of the context's smoother (AVS or
 * colored MVS, Sec. 3) with its local solver and damping, in place on x_dev. */
bh_status bh_smooth(bh_ctx* ctx, int level, double* x_dev, const double* b_dev, int steps);

/* Colors first_color .. end_color-1 of one step of the colored multiplicative
 * smoother (Sec. 3, 8 colors in 2D, 16 in 3D, processed in increasing order):
 * for each color, x_v += omega A_v^-1 R_v (b - A_l x) on all its patches at
 * once.  bh_smooth with one step equals the range 0 .. ncolors.  In place on
 * x_dev.  BH_EINVAL for another smoother or a range outside 0..ncolors. */
bh_status bh_smooth_colors(bh_ctx* ctx, int level, double* x_dev, const double* b_dev,
                           int first_color, int end_color);

/* xf += I_{l-1}^up xc: the embedding V_{l-1} -> V_l (Sec. 3).  level is the
 * fine level (>= 2); xc_dev has n(level-1) values, xf_dev n(level). */
bh_status bh_prolongate_add(bh_ctx* ctx, int level, const double* xc_dev, double* xf_dev);

/* bc = (I_{l-1}^up)^T rf: restriction, the transpose of the embedding
 * (Sec. 3).  level is the fine level (>= 2). */
bh_status bh_restrict(bh_ctx* ctx, int level, const double* rf_dev, double* bc_dev);

/* x <- MG_l(x, b): one V-cycle of Algorithm 1 from level l down to the coarse
 * level 1, in the context's precision (FP32 inside, FP64 in and out, for
 * the mixed forms: x += MG_l(0, b - A x) with the FP32 V-cycle).  In place on
 * x_dev. */
bh_status bh_vcycle(bh_ctx* ctx, int level, double* x_dev, const double* b_dev);

/* Tile shape of the fused colored-MVS kernels of this context: patches per
 * thread block (0 = automatic: about two blocks per SM, for FP64 capped at a
 * measured per-degree optimum; larger values are clamped to the kernel's
 * shared-memory budget).  Host only; takes effect on
 * the next smoothing call.  BH_EINVAL for a negative value. */
bh_status bh_set_tile(bh_ctx* ctx, int patches_per_block);

/* Solve A_L x = b on the finest level with a Krylov method preconditioned by
 * one V-cycle (Sec. 5.1), x0 = 0.
 * BH_GMRES: until the Givens estimate of the minimized residual
 * (preconditioned for BH_LEFT, true for BH_RIGHT) has dropped by rtol relative
 * to its initial value, or maxit iterations.  Right preconditioning keeps the
 * preconditioned directions (flexible form), as the FP32 V-cycle requires.
 * BH_CG: preconditioned conjugate gradients until the recursively updated
 * residual ||r_j|| <= rtol ||b||, or maxit iterations; with a mixed precision
 * the Polak-Ribiere coefficient (flexible CG) is used.  BH_ENOCONV also if p.Ap
 * <= 0 (the preconditioner is not positive definite).
 * On return (synchronous) *iters holds the iteration count and *relres the
 * true ||b - A x|| / ||b|| in FP64.  BH_ENOCONV if rtol was not reached (x
 * holds the last iterate). */
bh_status bh_solve(bh_ctx* ctx, const double* b_dev, double* x_dev, double rtol, int maxit,
                   int* iters, double* relres);

/* bh_solve from the initial guess held in x_dev (warm start, and the resume
 * point of an interrupted solve, e.g. after BH_ENOCONV): the correction d of
 * A d = b - A x is solved from zero and added to x, with the tolerance that
 * makes the stopping test the one of bh_solve on b (relative to ||b|| for
 * right GMRES and CG, to ||M^-1 b|| for left GMRES).  *iters counts the
 * iterations of this call; *relres is ||b - A x|| / ||b||.  A guess that
 * already meets the tolerance returns at once with *iters = 0.  The first
 * call allocates two vectors of workspace.  Synchronous.  The paper has no
 * counterpart (Sec. 5.1 solves from zero). */
bh_status bh_solve_guess(bh_ctx* ctx, const double* b_dev, double* x_dev, double rtol, int maxit,
                         int* iters, double* relres);

/* bh_solve with host buffers: copies b_host to the device, solves, copies x
 * back (b_host, x_host: n(L) doubles, pinned or pageable).  Synchronous. */
bh_status bh_solve_host(bh_ctx* ctx, const double* b_host, double* x_host, double rtol,
                        int maxit, int* iters, double* relres);

/* b_i = int f phi_i for f = Delta^2 u of the manufactured u = prod sin^2(pi x_a)
 * (BH_RHS_MANUFACTURED) or of the paper's u = prod sin(pi x_a)
 * (BH_RHS_PAPER_SINE, Sec. 5.1), on level l. */
bh_status bh_rhs(bh_ctx* ctx, int level, int kind, double* b_dev);

/* Counters of the context and the CUDA-event device time of its last
 * bh_solve / bh_solve_host ("last_solve_ms") as a JSON object written to buf
 * (NUL-terminated, truncated to len).  Host only.  Of the last solve:
 * "last_iters", "last_relres" (the true ||b - A x|| / ||b|| that the call
 * returned) and "last_estimate", the ratio its stopping test compared with
 * rtol: the Givens estimate of the minimized residual over its initial value
 * for GMRES (preconditioned for BH_LEFT, true for BH_RIGHT), ||r_j|| / ||b||
 * for CG; for bh_solve_guess, relative to the reference of a solve from zero.
 * The fractional iteration count of Sec. 5.1 is -8 iters / log10(estimate). */
bh_status bh_stats(const bh_ctx* ctx, char* buf, size_t len);

/* Message of the last failed call on this thread ("" if none). */
const char* bh_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (all contexts).  Host only; never fails. */
long long bh_kernel_launches(void);

/* Host-side fault injection, for testing failure handling without a device
 * fault: after `skip` more device allocations by the library succeed, the next
 * `fail` ones fail with BH_ENOMEM as if cudaMalloc had returned an out-of-memory
 * error (cudaMalloc is not called for them).  (0, 0) switches it off.  Global
 * to the process; host only.  The paper has no counterpart. */
bh_status bh_fault_inject_alloc(long long skip, long long fail);

/* Measured FP64 fused-multiply-add rate of the current device in TFLOP/s:
 * 4 blocks per SM of 128 threads, each running four independent chains of
 * dependent FMAs on registers, timed with CUDA events on `stream` (a
 * cudaStream_t; NULL = legacy default stream).  A reference for the FP64
 * kernels' roofline (the paper has no counterpart).  Allocates and frees a
 * small device buffer; synchronous.  BH_ECUDA without a device. */
bh_status bh_fp64_fma_rate(void* stream, double* tflops);

/* The same for the FP64 tensor-core instruction (mma.sync m8n8k4 f64, four
 * independent accumulator tiles per warp): the rate a DMMA formulation of the
 * FP64 contractions could reach on this device.  No paper counterpart. */
bh_status bh_fp64_mma_rate(void* stream, double* tflops);

/* Host-only 1D setup in FP64 on a line of `cells` cells of size 1 (the level
 * scaling is applied by the caller): which = 0, 1, 2 returns the mass M,
 * stiffness L and bulk-plus-face matrix B of Eq. (matrix1d) / Eq. (ev) on the
 * nodes 0..k*cells, row-major into out (ld = k*cells + 1). */
bh_status bh_setup_1d(int degree, double gamma, int cells, int which, double* out);

/* Host-only: the fast-diagonalization data of Sec. 4.1 for the 1D patch
 * matrices (B_v, M_v) of patch type `type` (0 interior, 1 touching x = 0,
 * 2 touching x = 1, 3 both: the single patch of N = 2) on cells of size 1:
 * S (m x m, row-major, columns the M-orthonormal eigenvectors) and lambda (m),
 * m = 2k - 1, with S^T M_v S = I and S^T B_v S = diag(lambda). */
bh_status bh_setup_fdm(int degree, double gamma, int type, double* S, double* lambda);

/* ---- batched form (no counterpart in the paper: a deployment form of the
 * same solver) ------------------------------------------------------------
 * Many independent 2D problems with their own degree and level, solved
 * together.  Every level operation of their V-cycles runs as ONE launch over
 * all problems (a work list of (problem, range) entries dispatched on the
 * degree); the patch work of one color is one launch per degree present,
 * forked into parallel branches so that each uses its own tile shape; the
 * lockstep V-cycle (x_L = MG_L(0, b_L) for every problem, Algorithm 1) is
 * captured once as a CUDA graph.  The V-cycle runs in FP64, or in FP32 with
 * the defect before each restriction evaluated and restricted in FP64
 * (BH_MIXED_FP32_R64).  GMRES(m) (Sec. 5.1) runs in lockstep with one host
 * synchronization per iteration for the whole batch, preconditioned on the
 * left (stopping on the preconditioned residual) or on the right in the
 * flexible form (stopping on the true residual), with restarts.  Each problem
 * follows the arithmetic of its own context, so its result matches bh_solve
 * on the same parameters up to rounding order and does not depend on the
 * other problems of the batch.
 * Calls on one batch must not overlap.  A batch works on its own stream;
 * every call first waits for the work already enqueued on the stream given to
 * bh_batch_create, and work enqueued there after the call returns waits for
 * the call's results. */
typedef struct bh_batch bh_batch;

/* count problems, params[i] each: dim 2, BH_MVS_COLORED, BH_FDM,
 * BH_COARSE_EXACT, BH_GMRES, precision BH_FP64, BH_MIXED_FP32_R64 or
 * BH_MIXED_FP32_RC (the mixed ones with BH_RIGHT; BH_MIXED_FP32_RC in the
 * graph form only); precision, gmres_side, pre_steps and post_steps the
 * same for every problem (BH_EINVAL otherwise); the restart length is the
 * largest gmres_restart.  Allocates every hierarchy, builds the work lists and
 * captures the V-cycle graph.  Synchronous. */
bh_status bh_batch_create(const bh_params* params, int count, void* stream, bh_batch** out);
bh_status bh_batch_destroy(bh_batch* batch);

/* Tile shape of the patch kernel for one degree: patches per thread block
 * (1..32, bounded by the shared-memory budget of the batch's precision).
 * Rebuilds the work lists and re-captures the graph.  Used by the autotuner. */
bh_status bh_batch_set_tile(bh_batch* batch, int degree, int patches_per_block);

/* Mean device time (ms, CUDA events) of one batched V-cycle graph launch on
 * the current right-hand sides, over reps launches after one warm-up. */
bh_status bh_batch_vcycle_time(bh_batch* batch, int reps, double* ms);

/* Persistent form of the batched V-cycle (on = 1; 0: the captured graph, the
 * default): the whole V-cycle runs as ONE cooperative launch whose blocks walk
 * its phases -- every color of the patch kernel, the sweeps, transfers, vector
 * operations and coarse solves of all problems at one depth -- separated by a
 * grid barrier.  Every barrier wait is bounded (2 s of clock cycles); a wait
 * that runs out ends the kernel with a status word that the next call reading
 * it turns into BH_ETIMEOUT.  The graph's arithmetic up to degree 4; above it
 * the persistent kernel solves interior patches by the unfolded fast
 * diagonalization, the graph's per-degree kernels by the folded one (equal up
 * to rounding).  Host only.  BH_EINVAL for a BH_MIXED_FP32_RC batch (its compensated defect sweeps are
 * graph nodes only). */
bh_status bh_batch_set_persistent(bh_batch* batch, int on);

/* Check of the persistent form's failure path: one persistent V-cycle whose
 * grid barrier expects one block more than the launch has, so that the first
 * barrier wait runs out after wait_ms (0 < wait_ms <= 10000) and every block
 * leaves the kernel; returns BH_ETIMEOUT (BH_EINVAL if the barrier had
 * completed).  No device fault, trap or unbounded wait is involved; the
 * batch's internal vectors are left undefined, the caller's are not touched.
 * Synchronous. */
bh_status bh_batch_check_barrier_timeout(bh_batch* batch, double wait_ms);

/* One batched V-cycle from zero: x_dev[i] = MG_L(0, b_dev[i]) (Algorithm 1)
 * for every problem i, by the captured graph in the batch's precision (the
 * preconditioner that bh_batch_solve applies).  b_dev, x_dev: host arrays of
 * device pointers, n_i FP64 values each, not aliased.  Synchronous. */
bh_status bh_batch_vcycle(bh_batch* batch, const double* const* b_dev, double* const* x_dev);

/* Colors first_color .. end_color-1 (0 <= first <= end <= 8) of one colored
 * multiplicative smoothing step (Sec. 3) on the finest level of every problem,
 * in place on x_dev[i] with right-hand side b_dev[i], by the batched patch
 * kernels of the batch's precision (for BH_MIXED_FP32_R64: x and b rounded to
 * FP32, the FP32 kernels, the result widened to FP64).  BH_EINVAL if a
 * problem's finest level is 1 (no smoother there).  Synchronous. */
bh_status bh_batch_smooth_colors(bh_batch* batch, double* const* x_dev,
                                 const double* const* b_dev, int first_color, int end_color);

/* Solve all problems from x = 0: b_dev[i], x_dev[i] are host arrays of device
 * pointers (n_i FP64 values each).  Every problem iterates until its stopping
 * test (the Givens estimate of the minimized residual -- preconditioned for
 * BH_LEFT, true for BH_RIGHT -- at most rtol times its initial value) holds
 * or it has run maxit iterations, restarting every m iterations.  iters[i] and
 * relres[i] (the true ||b - A x|| / ||b|| in FP64) receive each problem's
 * result.  BH_ENOCONV if any problem missed rtol.  Synchronous. */
bh_status bh_batch_solve(bh_batch* batch, const double* const* b_dev, double* const* x_dev,
                         double rtol, int maxit, int* iters, double* relres);

/* bh_batch_solve with host buffers: b_host[i], x_host[i] (pinned or pageable)
 * are copied through device staging buffers inside the call.  Synchronous. */
bh_status bh_batch_solve_host(bh_batch* batch, const double* const* b_host,
                              double* const* x_host, double rtol, int maxit, int* iters,
                              double* relres);

/* Kernel and graph launches issued by the batch so far. */
bh_status bh_batch_stats(const bh_batch* batch, long long* launches);

/* ---- serving form (no counterpart in the paper: a deployment form) --------
 * A request loop of solves with continuous batching: `slots` worker threads
 * each run one solve at a time on a resident hierarchy (pooled by dim,
 * degree, level and precision; each with its own CUDA stream), so solves of
 * different slots overlap on the device.  A request whose shape has no idle
 * hierarchy is admitted when the footprint estimate of a new one fits the
 * memory budget, after evicting idle hierarchies least recently used first;
 * otherwise it waits for running solves to release memory.  A request starts
 * as soon as a slot and its memory are free.  Precision: the FP32 V-cycle
 * with compensated FP32 defects (BH_MIXED_FP32_RC) in flexible FP64 GMRES
 * for degrees <= mixed_max_degree, FP64 otherwise; right preconditioning
 * (true residual).  A request's result does not depend on the other requests
 * in flight. */
typedef struct bh_server bh_server;

typedef struct {
  int slots;                /* concurrent solves (worker threads), 1..64 */
  double mem_budget_bytes;  /* device memory the resident hierarchies may use */
  int mixed_max_degree;     /* FP32 V-cycle (compensated defects) for k <= this, FP64 above
                               (default 7: every degree) */
  double rtol;              /* GMRES relative tolerance (default 1e-8) */
  int maxit;                /* GMRES iteration limit (default 200) */
  int gmres_restart;        /* restart length (default 30) */
  int64_t queue_capacity;   /* submissions beyond this many queued fail with BH_EBUSY */
} bh_server_config;

typedef struct {
  int status;        /* bh_status of the solve (BH_ENOMEM: larger than the budget) */
  int iters;
  double relres;     /* true relative residual */
  double latency_s;  /* completion - submission */
  double service_s;  /* time on a slot (the solve itself) */
} bh_server_result;

/* Defaults: 4 slots, 80 % of the currently free device memory, above. */
bh_status bh_server_default_config(bh_server_config* cfg);
bh_status bh_server_create(const bh_server_config* cfg, bh_server** out);

/* Queue a solve of the (dim, degree, level) problem with right-hand side b_host
 * (n host doubles); the solution is written to x_host.  Both host buffers stay
 * owned by the caller and must stay valid until bh_server_wait returns for
 * the ticket.  Returns at once with *ticket. */
bh_status bh_server_submit(bh_server* server, int dim, int degree, int level,
                           const double* b_host, double* x_host, int64_t* ticket);

/* bh_server_submit with a deadline: a request not started deadline_s seconds
 * after its submission (0: no deadline) is dropped when a slot reaches it, its
 * result status BH_ETIMEOUT; the server goes on with the next request. */
bh_status bh_server_submit_deadline(bh_server* server, int dim, int degree, int level,
                                    const double* b_host, double* x_host, double deadline_s,
                                    int64_t* ticket);

/* Cancel a queued request: it is removed from the queue and its result status
 * is BH_ECANCELED (the ticket must still be released by bh_server_wait).
 * BH_EBUSY if it has already started or finished (a running solve is not
 * interrupted), BH_EINVAL for an unknown ticket. */
bh_status bh_server_cancel(bh_server* server, int64_t ticket);

/* Wait up to timeout_s seconds (< 0: forever) for a ticket; fills *result and
 * releases the ticket.  BH_ETIMEOUT if still running.  Tickets that are never
 * waited for (a client that went away) do not hold up other requests; they
 * are released by bh_server_destroy. */
bh_status bh_server_wait(bh_server* server, int64_t ticket, double timeout_s,
                         bh_server_result* result);

/* Queue, slot and memory counters as a JSON object, with the requests dropped
 * at their deadline, cancelled, and failed (allocation or solve errors). */
bh_status bh_server_stats(bh_server* server, char* buf, size_t len);

/* Finish the queued requests, stop the workers, free every hierarchy. */
bh_status bh_server_destroy(bh_server* server);

/* y = A_l x like bh_apply_A, for callers that cannot allocate device memory:
 * for example a plugin inside a framework that owns every device allocation
 * and forbids allocation while it executes, or a latency-critical loop that
 * cannot afford the synchronization of cudaMalloc.  The paper has no
 * counterpart; it is a deployment variant of the apply_A kernel.
 *  - Needs no context and allocates nothing, on the device or on the host
 *    heap: the operator tables are built once per (degree, gamma) into static
 *    host storage and reused, and the sweep intermediates live in one static
 *    device array of 64 MiB (8 Mi doubles) that every GPU loading the library
 *    holds until the process exits.
 *  - Size limit: 3 (2D) or 6 (3D) times n^d must fit in that array, i.e. at
 *    most 2,796,202 unknowns in 2D and 1,398,101 in 3D, n = k 2^level - 1;
 *    larger problems fail with BH_EINVAL and a message naming the limit.
 *  - dim, degree, level, gamma as in bh_params (gamma <= 0: k(k+1)); x_dev,
 *    y_dev: n^d FP64 device values, caller-owned, not aliased; stream: the
 *    cudaStream_t to enqueue on (asynchronous).
 *  - Every call shares the array: calls whose kernels may overlap on the GPU
 *    (other streams, other host threads) race and must be serialized by the
 *    caller.  Nothing in the array needs to start at zero.
 *  - The first call on a device resolves the array's device address (with
 *    that device current); make that first call before any stream capture.
 *    A cudaDeviceReset of the device invalidates the resolved address without
 *    the library noticing: do not reset a device between calls. */
bh_status bh_apply_A_noalloc(int dim, int degree, int level, double gamma,
                             const double* x_dev, double* y_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BIHARM_H */
