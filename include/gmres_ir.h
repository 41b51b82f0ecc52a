/*
 * gmres_ir.h -- C ABI of the B300 (sm_103a) mixed-precision GMRES library.
 *
 * Method: Loe, Glusa, Yamazaki, Boman, Rajamanickam, "A Study of Mixed
 * Precision Strategies for GMRES on GPUs" (arXiv 2109.01232).
 *   - gmres_solve     : restarted GMRES(m) with CGS2 orthogonalisation in FP64
 *                       (Algorithm 1; CGS2 as described in Section 3.1).
 *   - gmres_ir_solve  : GMRES-IR (Algorithm 2, Section 3.2): FP64 residual and
 *                       update around a low-precision GMRES(m) cycle.
 *   - polynomial      : right preconditioning with the GMRES polynomial,
 *                       M^{-1} = p(A) (Section 3.4).
 * The problem statement is that of Algorithm 1: A in R^{n x n} (CSR), b, an
 * initial guess x0 and a relative residual tolerance; the output is x with
 * ||b - A x||_2 / ||b||_2 <= rtol.
 *
 * Conventions for every entry point:
 *   - Pointers named as DEVICE are device memory owned by the caller; the
 *     library never frees them.  HOST pointers are ordinary host memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous in their kernel launches but return only after the final
 *     status has been read back, so results are ready when a call returns.
 *   - Nothing is printed and nothing throws across the ABI: every function
 *     returns a gmres_status code.  Invalid arguments are rejected with
 *     GMRES_ERR_INVALID before any launch.
 *   - The library allocates its own workspace (Krylov basis, low-precision
 *     copy of A, Hessenberg data) with cudaMalloc; plans keep it between
 *     solves, the one-shot calls free it before returning.
 *   - Matrices use int32 indices: n < 2^31 and nnz < 2^31.  Column indices
 *     must lie in [0, n) and row_ptr must be nondecreasing with row_ptr[0] = 0
 *     (checked on the device before the first solve; violations give
 *     GMRES_ERR_INVALID).
 */
#ifndef GMRES_IR_H
#define GMRES_IR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
  GMRES_OK = 0,              /* converged: ||b - A x|| / ||b|| <= rtol (explicit FP64 residual) */
  GMRES_NOT_CONVERGED = 1,   /* max_iters reached; x holds the last iterate */
  GMRES_BREAKDOWN = 2,       /* singular least-squares factor after a breakdown (A singular) */
  GMRES_NONFINITE = 3,       /* NaN/Inf met in A, b or a reduction */
  GMRES_ERR_INVALID = 4,     /* bad argument (null pointer, size, parameter, CSR structure) */
  GMRES_ERR_OOM = 5,         /* device allocation failed */
  GMRES_ERR_CUDA = 6,        /* any other CUDA runtime error */
  GMRES_ERR_TOO_LARGE = 7,   /* a size exceeds a documented maximum */
  GMRES_ERR_DEVICE_TIMEOUT = 8 /* a kernel's bounded wait on its own copies expired (the kernel
                                  stopped and reported instead of waiting further) */
} gmres_status;

/* Storage precision of the inner solve: the Krylov basis V and the copy of A
 * used by the inner SpMV.  FP16/BF16 store 16-bit values and accumulate in
 * FP32; FP16 scales A by 1/max|a_ij| and each basis vector by s_v, the largest
 * power of two with s_v^2 <= 2n (about sqrt(n)). */
typedef enum { GMRES_FP64 = 0, GMRES_FP32 = 1, GMRES_FP16 = 2, GMRES_BF16 = 3 } gmres_prec;

/* CSR matrix, FP64 values (the master copy used by every FP64 residual).
 * All three arrays are DEVICE pointers, caller-owned, read only. */
typedef struct {
  int32_t n;                /* rows = columns */
  int32_t nnz;              /* row_ptr[n] */
  const int32_t* row_ptr;   /* n+1 entries */
  const int32_t* col_idx;   /* nnz entries */
  const double* vals;       /* nnz entries */
} gmres_csr;

/* Solver parameters; gmres_default_params() fills the paper's defaults
 * (Section 5: m = 50, rtol = 1e-10, FP32 inner precision, no preconditioner). */
typedef struct {
  int32_t restart_m;        /* m: Arnoldi steps per cycle, 1..GMRES_MAX_RESTART */
  double rtol;              /* outer relative residual tolerance (explicit FP64 residual) */
  double inner_rtol;        /* IR: end an inner cycle once |g_{j+1}| <= inner_rtol * ||r||;
                               0 = always m steps (the paper's GMRES-IR) */
  int64_t max_iters;        /* cap on the total number of Arnoldi steps */
  int32_t inner_prec;       /* gmres_prec of the inner cycle (IR only) */
  int32_t poly_degree;      /* degree d of the GMRES polynomial preconditioner; 0 = none */
  uint64_t seed;            /* SplitMix64 seed of the polynomial's start vector */
  int32_t record_history;   /* nonzero: keep |g_{j+1}| per iteration in gmres_stats */
  int32_t cgs_kernel;       /* gmres_cgs_kernel: how the CGS2 update kernels read V */
  int32_t poly_in_fp32;     /* nonzero: apply the polynomial preconditioner in FP32 (an FP32
                               copy of A, FP32 vectors, cast in and out) under an FP64 cycle --
                               the paper's FP64 GMRES with an FP32 polynomial (Section 5.4);
                               ignored when the cycle is not FP64 */
  int32_t bj_block;         /* block size k of the block-Jacobi right preconditioner
                               (Section 5.8, "J k"), 1..GMRES_MAX_BJ_BLOCK; 0 = none.  The
                               diagonal blocks [q k, min((q+1) k, n)) are LU-factored with
                               partial pivoting in FP64 at plan creation and applied in the
                               cycle's working precision (FP64 for FP64 plans, FP32
                               otherwise).  Not combined with poly_degree > 0. */
  int32_t bj_rcm;           /* nonzero: reorder the system with reverse Cuthill-McKee at
                               plan creation (Section 5.8; before the blocks are taken);
                               b, x0 and x stay in the caller's numbering */
  int32_t max_outer;        /* cap on the restart cycles (GMRES) / refinement steps
                               (GMRES-IR) of a solve; 0 = none (max_iters alone).  A solve
                               stopped by it returns GMRES_NOT_CONVERGED with x the last
                               iterate.  Must be 0 for the batched solver. */
  int64_t tma_wait_cycles;  /* bound, in SM clocks, of each wait of the TMA-fed CGS kernels
                               (cgs_kernel = GMRES_CGS_TMA) for a stage of copies or a
                               released stage; 0 = the default, 2^31 clocks (about a second).
                               A wait that expires ends the solve with
                               GMRES_ERR_DEVICE_TIMEOUT; the kernel still waits for the copies
                               it has issued, with the default bound, before it returns */
  int32_t tma_test_withhold; /* test hook of that timeout path, 0 in normal use: nonzero makes
                               the TMA producer of every CGS launch issue the copies of its
                               first row block only, so the consumers' wait for the second
                               block can only end by the bound */
} gmres_params;

/* Forms of the two CGS2 update kernels (the same arithmetic per row; both produce the
 * same partial-sum layout for the next kernel). */
typedef enum {
  GMRES_CGS_REGISTER = 0,  /* vector loads into registers (default: the faster form on a
                              B300 at every step length measured) */
  GMRES_CGS_TMA = 1        /* cp.async.bulk copies into a shared-memory ring, one producer
                              warp; used for the steps whose basis block fits two stages,
                              the register form for the others */
} gmres_cgs_kernel;

#define GMRES_MAX_RESTART 512
#define GMRES_MAX_POLY_DEGREE 96
#define GMRES_MAX_BJ_BLOCK 64

/* Solve statistics (written by every solve entry point when non-NULL). */
typedef struct {
  int32_t status;           /* gmres_status of the solve */
  int64_t iters;            /* total Arnoldi steps (inner iterations) */
  int32_t outer_iters;      /* restarts = refinement steps */
  double rel_resid;         /* final explicit ||b - A x||_2 / ||b||_2 in FP64 */
  double t_solve_ms;        /* device time of the solve (CUDA events) */
  double t_setup_ms;        /* device time of set-up: low-precision copy of A, polynomial */
  int64_t history_len;      /* entries written to history (<= history_cap) */
  double* history;          /* HOST buffer supplied by the caller, or NULL: relative
                               residual estimate after every Arnoldi step */
  int64_t history_cap;      /* capacity of history */
} gmres_stats;

void gmres_default_params(gmres_params* p);
const char* gmres_status_string(int status);
/* The last CUDA failure recorded by this thread (call site and the runtime's
 * message) behind a GMRES_ERR_CUDA / GMRES_ERR_OOM status; "" if none. */
const char* gmres_last_error(void);

/* FP64 restarted GMRES(m) (Algorithm 1 with CGS2).  b: DEVICE, n doubles.
 * x: DEVICE, n doubles, initial guess on entry, solution on exit.  The cycle
 * ends early when the Givens residual reaches rtol*||b||; convergence is then
 * confirmed by the explicit residual.  p->inner_prec is ignored. */
int gmres_solve(const gmres_csr* A, const double* b, double* x, const gmres_params* p,
                gmres_stats* stats, void* stream);

/* GMRES-IR (Algorithm 2): r = b - A x [FP64]; u = GMRES(m) cycle on A u = r in
 * p->inner_prec; x += u [FP64]; repeat while ||r|| / ||b|| > rtol.  Same
 * pointer conventions as gmres_solve. */
int gmres_ir_solve(const gmres_csr* A, const double* b, double* x, const gmres_params* p,
                   gmres_stats* stats, void* stream);

/* GMRES-FD (Section 3.3): restarted GMRES(m) entirely in single precision (b, A, x, the
 * basis and the explicit residual rounded to FP32, FP32 arithmetic) for switch_iters
 * iterations, rounded up to whole cycles so that the switch happens at a restart, then
 * FP64 GMRES(m) (as gmres_solve) from that iterate for the remaining p->max_iters.
 * Pointers as in gmres_solve.  stats_fp32 / stats_fp64 (either may be NULL) describe the
 * two stages; the return value is the FP64 stage's status.  switch_iters = 0 is plain
 * FP64 GMRES; no preconditioner or reordering (p->poly_degree, p->bj_block and p->bj_rcm
 * must be 0, else GMRES_ERR_INVALID). */
int gmres_fd_solve(const gmres_csr* A, const double* b, double* x, const gmres_params* p,
                   int64_t switch_iters, gmres_stats* stats_fp32, gmres_stats* stats_fp64,
                   void* stream);

/* Same solves with HOST pointers: A's arrays, b and x live in host memory
 * (pinned memory gives the fastest copies).  The call copies A, b and x0 to
 * the device, solves, and copies x back before returning. */
int gmres_ir_solve_host(const gmres_csr* A_host, const double* b, double* x,
                        const gmres_params* p, gmres_stats* stats, void* stream);
int gmres_solve_host(const gmres_csr* A_host, const double* b, double* x,
                     const gmres_params* p, gmres_stats* stats, void* stream);

/* ---- Plans: keep the workspace, the low-precision copy of A, the polynomial
 * and the captured CUDA graph of one cycle between solves. ----------------- */
typedef struct gmres_plan_s* gmres_plan;

/* kind: 0 = FP64 GMRES, 1 = GMRES-IR with p->inner_prec, 2 = GMRES entirely in FP32
 * (GMRES-FD's first stage; p->inner_prec ignored, no polynomial, block Jacobi or
 * reordering).  A's arrays must stay valid until gmres_plan_destroy.  Set-up on the
 * stream: CSR check, the low-precision SELL-32 copy of A, with bj_rcm the reordering
 * (host) and the plan's reordered copy, the polynomial roots, the block factors, the
 * graph capture.  GMRES_ERR_INVALID for a malformed CSR, bad parameters or a singular
 * diagonal block (bj_block > 0); GMRES_ERR_OOM / GMRES_ERR_CUDA on allocation / runtime
 * failure (nothing is leaked). */
int gmres_plan_create(gmres_plan* plan, const gmres_csr* A, int32_t kind, const gmres_params* p,
                      void* stream);
int gmres_plan_solve(gmres_plan plan, const double* b, double* x, gmres_stats* stats,
                     void* stream);
int gmres_plan_destroy(gmres_plan plan);
/* Times y = A x with the plan's SELL-32 inner copy of A, the SpMV alone (no dot products,
 * no basis store; Section 5.5's fp64-vs-fp32 experiment): one warm-up launch, then `reps`
 * launches between CUDA events on `stream`.  x, y: DEVICE, n values of the plan's working
 * type (double for FP64 plans, float otherwise), not overlapping.  *ms_out = mean ms per
 * SpMV. */
int gmres_plan_spmv_timed(gmres_plan plan, const void* x, void* y, int32_t reps, float* ms_out,
                          void* stream);
/* Changes the stopping parameters of later solves on the plan (rtol, inner_rtol,
 * max_iters as in gmres_params); the captured cycle does not depend on them. */
int gmres_plan_set_tolerances(gmres_plan plan, double rtol, double inner_rtol, int64_t max_iters);

/* ---- Building blocks on a plan (the hot-path kernels, exposed for tests) - */

/* y = A v with the plan's inner copy of A: v is DEVICE, n doubles; it is
 * scaled and rounded to the plan's storage precision exactly as a basis
 * vector is; y is DEVICE, n values of the working type (double for FP64
 * plans, float otherwise).  Runs the fused SpMV kernel of the Arnoldi step. */
int gmres_plan_spmv(gmres_plan plan, const double* v, void* y, void* stream);

/* Arnoldi with CGS2 from v0 (DEVICE, n doubles) for `steps` steps (<= m),
 * the cycle kernels of the solver without the stopping test.  V_out: DEVICE,
 * (steps+1) columns of n values in the storage type (double, float, half or
 * bfloat16; FP16 values are scaled by s_v, see gmres_prec).  H_out: HOST, (steps+1) x
 * steps FP64, column-major.  *k_out = steps taken (fewer after a breakdown). */
int gmres_plan_arnoldi(gmres_plan plan, const double* v0, int32_t steps, void* V_out,
                       double* H_out, int32_t* k_out, void* stream);

/* GMRES-polynomial set-up (Section 3.4): `degree`+1 FP64 Arnoldi steps on
 * the GPU from the SplitMix64 vector of `seed` (or from v0 if non-NULL,
 * DEVICE, n doubles), harmonic Ritz values on the host, Leja ordering.
 * roots_re/roots_im: HOST arrays of degree+1 entries; *nroots = roots
 * written (fewer after an Arnoldi breakdown). */
int gmres_poly_roots(const gmres_csr* A, int32_t degree, uint64_t seed, const double* v0,
                     double* roots_re, double* roots_im, int32_t* nroots, void* stream);

/* y = p(A) v with the plan's GMRES polynomial (Section 3.4; the plan must have
 * poly_degree > 0): the product form over the Leja-ordered roots, d SpMVs with
 * the plan's inner copy of A, in the working precision.  v: DEVICE, n doubles;
 * y: DEVICE, n values of the polynomial's working type (double for FP64 plans,
 * float otherwise and for FP64 plans created with poly_in_fp32). */
int gmres_plan_poly_apply(gmres_plan plan, const double* v, void* y, void* stream);

/* y = M^{-1} v with the plan's block-Jacobi factors (Section 5.8; the plan must have
 * bj_block > 0): per block, the pivoted forward and back substitutions in the working
 * precision.  v: DEVICE, n doubles; y: DEVICE, n values of the working type (double for
 * FP64 plans, float otherwise).  Both in the plan's numbering (reordered when bj_rcm).
 * Asynchronous on `stream` (y is ready in stream order).  GMRES_ERR_INVALID without
 * block Jacobi or with a NULL pointer. */
int gmres_plan_bj_apply(gmres_plan plan, const double* v, void* y, void* stream);

/* The plan's reverse Cuthill-McKee permutation: *reordered = 1 and, if perm is not NULL,
 * perm[new] = old (HOST, n entries) when the plan was created with bj_rcm; *reordered = 0
 * otherwise (perm untouched).  The plan's test entry points (spmv, arnoldi, bj_apply,
 * poly_apply) work in the reordered numbering; solves take and return the caller's. */
int gmres_plan_perm(gmres_plan plan, int32_t* perm, int32_t* reordered);

/* Reverse Cuthill-McKee ordering of a CSR structure (Section 5.8), on the host: all
 * arrays HOST; perm[new] = old, n entries, written by the call.  The graph is the
 * structure of A + A^T without the diagonal; vertices rank by (degree, index); each
 * connected component (in the order of its lowest-ranked vertex) starts from the
 * pseudo-peripheral vertex of the George-Liu iteration and is ordered by a breadth-first
 * search that takes unvisited neighbours in rank order; the whole order is reversed.
 * GMRES_ERR_INVALID for a malformed structure (row_ptr[0] != 0, decreasing row_ptr,
 * column out of range) or a NULL pointer with n > 0; GMRES_ERR_OOM when the host memory
 * of the graph (about 8 bytes per stored entry) cannot be allocated. */
int gmres_rcm(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t* perm);

/* The plan's polynomial roots (HOST arrays of at least poly_degree+1 entries,
 * either may be NULL) in the order they are applied; *nroots = 0 without a
 * preconditioner. */
int gmres_plan_poly_roots(gmres_plan plan, double* roots_re, double* roots_im, int32_t* nroots);

/* Profiling aid for the per-kernel time breakdown of one cycle (the kernel
 * classes of the paper's Section 5.2 breakdown and Table 1: SpMV, the two
 * transposed/plain GEMV passes of CGS2, norm, least squares, update).  Runs
 * the FP64 residual of x0 (DEVICE, n doubles) against b (DEVICE) and one
 * restart cycle kernel by kernel, not through the graph, with CUDA events
 * around every launch.  ms_out: HOST, 3m+3 doubles; ms_out[3j+0/1/2] = fused
 * SpMV / first CGS update / second CGS update of Arnoldi step j,
 * ms_out[3m+0/1/2] = least squares / x update / residual; -1 for steps the
 * cycle did not reach. */
int gmres_plan_profile_cycle(gmres_plan plan, const double* b, const double* x0, double* ms_out,
                             void* stream);
/* The same breakdown measured as a solve runs the cycle: one restart cycle captured as
 * a CUDA graph with an event-record node (cudaEventRecordExternal) before every kernel
 * and after the last, launched once; ms_out[i] = time between the events around kernel
 * i (same layout and -1 convention as gmres_plan_profile_cycle).  Instantiates a
 * graph per call (not for use inside a solve loop); synchronises the stream. */
int gmres_plan_profile_cycle_graph(gmres_plan plan, const double* b, const double* x0,
                                   double* ms_out, void* stream);
/* The cycle of gmres_plan_profile_cycle_graph captured with event-record nodes only
 * before its first kernel and after its last, so that no event node sits between two
 * kernels: ms_out (HOST, 2 doubles) = {milliseconds of the whole cycle, Arnoldi steps
 * it took}.  With the per-kernel times of gmres_plan_profile_cycle_graph this gives each
 * kernel's share of a cycle that runs as in a solve.  Same inputs, state reset and
 * synchronisation as gmres_plan_profile_cycle_graph. */
int gmres_plan_time_cycle_graph(gmres_plan plan, const double* b, const double* x0,
                                double* ms_out, void* stream);

/* Plan geometry: info_out (HOST, 8 int64) = n, nnz, leading dimension ld,
 * m, storage precision, grid of the SpMV kernel, grid of the CGS kernels,
 * grid of the residual kernel. */
int gmres_plan_info(gmres_plan plan, int64_t* info_out);

/* SplitMix64 vector on the device: out[i] in [-1, 1) (DEVICE, n doubles). */
int gmres_splitmix64_fill(double* out, int64_t n, uint64_t seed, void* stream);

/* y = A v in FP64 without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc
 * -- code whose GPU memory is owned by another allocator that reserved it up
 * front, latency-critical loops that cannot take the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree, and plug-ins that may not allocate.
 * It runs the library's CSR SpMV kernel (plans use a SELL-32 copy of A, which
 * this entry point cannot allocate; the products are summed in CSR order, so y
 * agrees with gmres_plan_spmv on an FP64 plan to rounding).  Its scratch -- a
 * device state with the flag of the structure check, and room to stage v when
 * y overlaps it -- lives in a fixed device array of about 8 MB that every GPU
 * loading this library keeps until the process exits.
 *   A: DEVICE CSR (FP64 values), n <= GMRES_NOALLOC_MAX_N, else
 *      GMRES_ERR_TOO_LARGE (checked before any device work).  The structure is
 *      checked on the device first (row_ptr[0] = 0, row_ptr[n] = nnz,
 *      non-decreasing row_ptr, 0 <= col_idx < n): a malformed one returns
 *      GMRES_ERR_INVALID with y untouched.
 *   v: DEVICE, n doubles; y: DEVICE, n doubles.  y may overlap v (then v is
 *      copied into the scratch array before the product).
 * Each call looks up the array's address on the current device
 * (cudaGetSymbolAddress) and returns only after the stream has finished the
 * work, so the call is synchronous: it cannot be made on a stream that is
 * being captured into a graph.  All calls share the one array: calls that may
 * overlap on the GPU (different streams, or several host threads) race and
 * must be serialised by the caller. */
#define GMRES_NOALLOC_MAX_N (1 << 20)
int gmres_spmv_fp64_noalloc(const gmres_csr* A, const double* v, double* y, void* stream);

/* ---- Batched GMRES-IR: many independent small systems -------------------
 * Each system A_i x_i = b_i is solved by GMRES-IR (Algorithm 2: FP64 residual and
 * update, inner GMRES(m) cycle of Algorithm 1 with CGS2 in p->inner_prec) exactly as
 * gmres_ir_solve would, but all systems run in ONE persistent kernel: every thread-block
 * cluster takes the next unsolved system (largest first, through a device counter) and
 * carries out its whole solve, its CTAs splitting the rows and combining their sums
 * through distributed shared memory, so no system waits for another and no cluster waits
 * for another cluster.  Meant for systems of up to a few 10^5 rows (the per-cluster
 * workspace is (m+1) columns of the largest system); restart_m <= GMRES_BATCH_MAX_M.
 *
 * The systems are one concatenated CSR:
 *   row_off, nnz_off: HOST, nsys+1 int64 each, non-decreasing, row_off[0] = nnz_off[0]
 *                     = 0: system i has rows [row_off[i], row_off[i+1]) of the
 *                     concatenated vectors and nonzeros [nnz_off[i], nnz_off[i+1]).
 *   row_ptr: DEVICE, row_off[nsys] + nsys int32: system i's n_i + 1 LOCAL row pointers
 *            (starting at 0) begin at row_ptr[row_off[i] + i].
 *   col_idx: DEVICE, LOCAL column indices (0 <= c < n_i); vals: DEVICE FP64.
 * The caller owns these arrays; a plan reads them until it is destroyed. */
#define GMRES_BATCH_MAX_M 32
typedef struct {
  int32_t nsys;
  const int64_t* row_off;
  const int64_t* nnz_off;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const double* vals;
} gmres_csr_batch;

/* Per-system results (HOST arrays of nsys entries each, any may be NULL). */
typedef struct {
  int32_t* status;     /* gmres_status of each system */
  int64_t* iters;      /* inner iterations */
  int32_t* outer;      /* refinement steps */
  double* rel_resid;   /* final explicit FP64 ||b_i - A_i x_i|| / ||b_i|| */
  double t_solve_ms;   /* device time of the whole batch (CUDA events) */
} gmres_batch_stats;

typedef struct gmres_batch_plan_s* gmres_batch_plan;

/* Creates the workspace (FP32 copy of the values, per-cluster basis and vectors), chooses
 * the CTA size (256 or 512 threads) and the cluster size (1, 2, 4 or 8 CTAs per system) --
 * if autotune is nonzero by timing each pair on a sample of the systems (every 8th by
 * size, b = ones) and the two fastest once more on all the systems (two extra solves of
 * the whole batch at set-up), else 256 threads in clusters of 4 -- and captures the launch
 * as a CUDA graph.  p: restart_m (<= GMRES_BATCH_MAX_M), rtol, inner_rtol, max_iters (per system),
 * inner_prec (GMRES_FP32, or GMRES_FP64 for plain FP64 GMRES(m) per system).
 * Errors: INVALID (bad sizes/offsets/structure/params), TOO_LARGE (m), OOM, CUDA. */
int gmres_batch_plan_create(gmres_batch_plan* plan, const gmres_csr_batch* A,
                            const gmres_params* p, int32_t autotune, void* stream);
/* b: DEVICE, row_off[nsys] doubles; x: DEVICE, the same, initial guesses on entry,
 * solutions on exit.  Returns OK when every system converged, else the first non-OK
 * status in system order (per-system codes in stats->status). */
int gmres_batch_plan_solve(gmres_batch_plan plan, const double* b, double* x,
                           gmres_batch_stats* stats, void* stream);
/* out[0..6] = threads per CTA, CTAs, candidates timed by the autotuner, largest system's
 * rows, basis leading dimension, inner precision, CTAs per cluster. */
int gmres_batch_plan_info(gmres_batch_plan plan, int64_t* out);
int gmres_batch_plan_destroy(gmres_batch_plan plan);
/* One-shot: plan (no autotuning), solve, destroy. */
int gmres_ir_solve_batched(const gmres_csr_batch* A, const double* b, double* x,
                           const gmres_params* p, gmres_batch_stats* stats, void* stream);

/* ---- Learned parameter selector -------------------------------------------
 * Picks the restart length, polynomial degree, inner precision and inner tolerance of
 * GMRES-IR from 16 cheap features of A with a 16-64-64-32 MLP (ReLU, softmax over 32
 * classes).  The paper has no such component.  Its network is trained on sweep timings of
 * this solver (paper_2109_01232_b300/selector.py) by gmres_mlp_train; without a model, or
 * below the model's confidence threshold, the fixed default is used: m = 50, no
 * polynomial, FP32 inner storage, inner tolerance 1e-4. */
#define GMRES_SEL_FEATURES 16
#define GMRES_SEL_CLASSES 32
#define GMRES_SEL_PARAMS 7328   /* W1[16][64] b1[64] W2[64][64] b2[64] W3[64][32] b3[32], W row-major */

/* The 16 features of A (DEVICE CSR, n >= 1) into features (HOST, 16 floats), with
 * d_i = a_ii (0 if absent), s_i = sum_j |a_ij|, lg(x) = log10(max(x, 1e-30)):
 *  0 lg n, 1 lg nnz, 2 nnz/n, 3 max row length, 4 mean |d_i|/s_i, 5 min |d_i|/s_i,
 *  6 share of rows with |d_i| >= s_i - |d_i|, 7 lg max s_i, 8 lg ||A||_F, 9 lg max|a_ij|,
 *  10 lg mean |d_i|, 11 lg max|d_i| - lg min nonzero |d_i|,
 *  12 sum (a_ij - a_ji)^2 / sum (a_ij^2 + a_ji^2) over the off-diagonal pattern,
 *  13 mean over rows with d_i != 0 of (sum_{j != i} a_ij) / d_i,
 *  14 log10(1 + mean |i - j| over the nonzeros), 15 log10(1 + max |i - j|).
 * Statistics are accumulated in FP64 in a fixed order. */
int gmres_matrix_features(const gmres_csr* A, float* features, void* stream);
/* Class probabilities (HOST, nsamp x 32) of the rows of X (HOST, nsamp x 16, already
 * normalised) under params (HOST, GMRES_SEL_PARAMS). */
int gmres_mlp_forward(const float* params, const float* X, int32_t nsamp, float* probs, void* stream);
/* Mean cross-entropy of X against labels (HOST, nsamp ints in [0, 32)) and its gradient
 * (HOST, GMRES_SEL_PARAMS floats, the params layout). */
int gmres_mlp_loss_grad(const float* params, const float* X, const int32_t* labels, int32_t nsamp,
                        float* loss, float* grad, void* stream);
/* Full-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8, step lr) for `epochs` steps on the
 * device: params (HOST) in = initial weights, out = trained; losses (HOST, epochs, or
 * NULL) = the loss before each step. */
int gmres_mlp_train(float* params, const float* X, const int32_t* labels, int32_t nsamp,
                    int32_t epochs, float lr, float* losses, void* stream);

typedef struct {
  const float* params;             /* HOST, GMRES_SEL_PARAMS, or NULL: always the default */
  const float* feat_mean;          /* HOST, 16: the network's input is */
  const float* feat_scale;         /* HOST, 16:   (feature - mean) * scale */
  const int32_t* class_m;          /* HOST, 32: restart length of each class */
  const int32_t* class_degree;     /* HOST, 32: polynomial degree */
  const int32_t* class_prec;       /* HOST, 32: gmres_prec of the inner cycle */
  const double* class_inner_rtol;  /* HOST, 32: inner tolerance */
  float min_confidence;            /* below this top probability, use the default */
} gmres_selector;

/* Sets p->restart_m, poly_degree, inner_prec and inner_rtol for A: the selector's class
 * if it has a model and is confident, else the default (*class_out = -1).  Other fields
 * of p are left as they are.  confidence_out: the top class probability (0 without a
 * model).  Either output may be NULL. */
int gmres_select_params(const gmres_csr* A, const gmres_selector* sel, gmres_params* p,
                        int32_t* class_out, float* confidence_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GMRES_IR_H */
