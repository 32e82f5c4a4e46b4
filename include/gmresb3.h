/*
 * gmresb3 -- multiprecision restarted GMRES for one NVIDIA B300 (sm_103a).
 *
 * C ABI of the solver library (libgmresb3.so).  The method is GMRES(m) with two passes of
 * classical Gram-Schmidt per iteration (Algorithm 1 and Section III-A of Loe et al.,
 * "Experimental Evaluation of Multiprecision Strategies for GMRES on GPUs") and its iterative-
 * refinement form GMRES-IR (Algorithm 2, Section III-B): the inner GMRES(m) cycle runs in FP32
 * (with the Krylov basis stored in FP32 or BF16), the residual r = b - A x and the update
 * x = x + u run in FP64.  An optional GMRES-polynomial right preconditioner p(A)
 * (Section III-D) is built in FP64 at create time and applied as repeated SpMVs.
 *
 * Conventions shared by every call:
 *  - Return value: 0 (GMRES_OK) on success; negative = caller or CUDA error; positive =
 *    numerical outcome of a solve (the solution buffer then holds the best iterate reached).
 *  - Device pointers are CUDA global-memory pointers on the device that was current when the
 *    handle was created; host pointers are plain (pageable or pinned) host memory.  Where a call
 *    accepts either, the library tells them apart with cudaPointerGetAttributes.
 *  - The library never prints and keeps no global state except the handles it returns and the
 *    fixed scratch array of gmres_precond_apply_noalloc.  Each handle runs its work on a private
 *    non-blocking stream, ordered after the caller's stream when a call starts and before it
 *    when the call ends (the caller's stream is the legacy default stream unless
 *    gmres_set_stream names another).
 *  - Vectors are dense, contiguous, length n.  Matrices are square CSR with int32 row pointers
 *    and column indices (Section V-D: 4-byte indices in every precision); columns need not be
 *    sorted within a row.
 */
#ifndef GMRESB3_H
#define GMRESB3_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------------------------- */
enum {
    GMRES_OK = 0,
    GMRES_ERR_INVALID_ARG = -1,   /* bad pointer, size, CSR structure or parameter            */
    GMRES_ERR_OOM = -2,           /* device allocation failed                                  */
    GMRES_ERR_CUDA = -3,          /* a CUDA runtime call failed (no device, launch error, ...) */
    GMRES_ERR_UNSUPPORTED = -4,   /* valid request that the library does not implement        */
    GMRES_NOT_CONVERGED = 1,      /* maxiter or the time limit reached before tol              */
    GMRES_NAN = 2,                /* a NaN/Inf appeared in a norm; the solve stopped            */
    GMRES_LOSS_OF_ACCURACY = 3,   /* FP64 GMRES: implicit residual met tol but the explicit one
                                     did not, more often than max_loss_of_accuracy (Sec. V-F)  */
    GMRES_STAGNATION = 4,         /* GMRES-IR: the explicit residual stopped decreasing        */
    GMRES_TIMEOUT = 5             /* a kernel's bounded wait for a bulk copy gave up (after
                                     200 ms); the solve stopped, x holds the last good iterate  */
};

/* ---- precisions ---------------------------------------------------------------------------- */
typedef enum { GMRES_F64 = 0, GMRES_F32 = 1, GMRES_BF16 = 2, GMRES_F16 = 3 } gmres_prec_t;

/* Precisions of a handle.  matrix = F32 and inner = F32: the FP32 copy of A and the FP32
 * arithmetic of the GMRES-IR inner cycle (dot products accumulate in FP32); gmres_solve_fp64
 * always uses the FP64 values.  basis: storage of the GMRES-IR Krylov basis, F32, BF16 or F16
 * (FP16 columns are stored scaled to entries of order one -- the cycle's first vector by
 * sqrt(n) / ||r||, each new one by sqrt(n) / ||A z||, never past FP16's range -- and the scale is
 * folded into the per-column scale; the paper names half precision as future work, Section VI).
 * precond: the precision in which gmres_solve_fp64 applies the polynomial preconditioner, F64 or
 * F32 (GMRES-IR always applies it in FP32).  The outer residual and the solution update are
 * always FP64.  Other combinations give GMRES_ERR_UNSUPPORTED. */
typedef struct {
    gmres_prec_t matrix, inner, basis, precond;
} gmres_precisions_t;

/* ---- matrix -------------------------------------------------------------------------------- */
/* Square CSR matrix.  rowptr[n+1] (rowptr[0] = 0, non-decreasing, rowptr[n] = nnz),
 * colidx[nnz] in [0, n), val[nnz] finite FP64.  on_device = 0: host arrays, 1: device arrays.
 * gmres_create copies the matrix; the caller keeps ownership of these arrays. */
typedef struct {
    int64_t n, nnz;
    const int32_t *rowptr;
    const int32_t *colidx;
    const double *val;
    int on_device;
} gmres_csr_t;

/* ---- solve parameters ---------------------------------------------------------------------- */
typedef struct {
    int m;                    /* restart length for the next solves; 0 = the create-time m;
                                 must not exceed the create-time m                              */
    int64_t maxiter;          /* cap on inner iterations (default 200000)                       */
    double time_limit_s;      /* wall-clock cap per solve in seconds; 0 = none                  */
    double inner_tol;         /* GMRES-IR: end an inner cycle once its implicit residual is
                                 <= inner_tol * ||r||; 0 (default) = always m steps (Sec. III-B) */
    int use_graphs;           /* 1 (default): one CUDA graph per restart cycle, replayed        */
    int profiling;            /* 1: time kernel classes with CUDA events (runs without graphs)  */
    int stagnation_cycles;    /* GMRES-IR: STAGNATION after this many consecutive cycles whose
                                 residual did not fall below 0.9x the best so far; 0 = off      */
    int max_loss_of_accuracy; /* FP64 GMRES: stop with LOSS_OF_ACCURACY after this many
                                 implicit/explicit mismatches (default 20)                      */
    int orth;                 /* orthogonalisation: 0 (default) = CGS2, two classical Gram-
                                 Schmidt passes per step (Section III-A); 1 = DCGS2, the second
                                 pass delayed by one step and merged with the next step's first
                                 (Bielich et al. 2022): the same Arnoldi factorisation in exact
                                 arithmetic, A DIFFERENT ALGORITHM in floating point, one global
                                 reduction and two basis reads per step instead of three of
                                 each.  Not with an F16 basis (GMRES_ERR_UNSUPPORTED).           */
} gmres_params_t;

/* ---- launch shapes (autotuner) ---------------------------------------------------------------- */
/* Launch shapes of the single-system kernels.  0 in a field = the built-in heuristic.  They change
 * how rows and tiles are grouped over CTAs, so FP32 partial sums (and the last bits of the inner
 * iterates) depend on them; every choice reaches the same FP64 tolerance. */
typedef struct {
    int sweep_stage_kb;       /* target size of one CGS2 sweep pipeline stage in KB (0 = 24)    */
    int sweep_ctas_per_sm;    /* resident sweep CTAs per SM the stage count is sized for
                                 (0 = the first of 4, 2, 1 that gives >= 2 stages; max 4)      */
    int spmv_ctas_per_sm;     /* CTAs per SM of the SpMV and polynomial kernels
                                 (0 = the occupancy limit)                                     */
    int spmv_lanes_per_row;   /* lanes per matrix row in the SpMV kernels: 1 = a row per thread,
                                 2, 4, 8, 16 or 32 = a group of lanes per row (coalesced loads of
                                 long rows); 0 = from the mean nonzeros per row w (1 up to
                                 w = 12, else the power of two with about five per lane)       */
    int cluster_cycle;        /* small systems: 0 (default) = each restart cycle of
                                 gmres_ir_solve (FP32 or BF16 basis) and gmres_solve_fp64 is one
                                 kernel on one thread-block cluster when the system qualifies --
                                 no preconditioner, CGS2, at most 16 CTAs of 256 or 512 rows
                                 whose shared memory holds their rows of all m + 1 basis columns
                                 (FP64 at m = 50: up to 4096 rows); the cycle's global sums are
                                 cluster barriers over distributed shared memory instead of
                                 kernel boundaries.  -1 = always the per-step kernels.          */
} gmres_tuning_t;

/* ---- statistics ---------------------------------------------------------------------------- */
enum {  /* indices of gmres_stats_t.t_kernel (seconds, filled when profiling = 1) */
    GMRES_T_SPMV = 0,         /* inner SpMV w = A z (FP32 arithmetic: fused with the first
                                 projection and ||w||)                                         */
    GMRES_T_CGS_PASS2 = 1,    /* first update fused with the second projection                  */
    GMRES_T_CGS_UPDATE = 2,   /* second update, norm, basis store and Givens step               */
    GMRES_T_PRECOND = 3,      /* polynomial preconditioner SpMV steps                           */
    GMRES_T_RESIDUAL = 4,     /* FP64 residual r = b - A x and its norm                          */
    GMRES_T_SOLUTION = 5,     /* least-squares back substitution and x = x + p(A) V y           */
    GMRES_T_CGS_PROJ = 6,     /* FP64 solver: first projection h1 = V^T w and ||w|| (in FP32
                                 arithmetic it runs inside GMRES_T_SPMV)                       */
    GMRES_T_OTHER = 7
};

typedef struct {
    int64_t iters;            /* inner iterations (Arnoldi steps) over all cycles               */
    int64_t cycles;           /* restart cycles                                                 */
    double rel_res_explicit;  /* final ||b - A x||_2 / ||b||_2 in FP64                          */
    double rel_res_implicit;  /* last implicit (Givens) residual / ||b|| (FP64 GMRES) or
                                 / ||r|| of the last cycle (GMRES-IR)                            */
    int status;               /* same value the solve returned                                  */
    int64_t loss_of_accuracy; /* implicit/explicit mismatches seen (Sec. V-F)                    */
    int64_t breakdowns;       /* lucky breakdowns                                               */
    double *res_history;      /* caller-owned host buffer or NULL: explicit relative residual
                                 at the start and after every cycle                              */
    int64_t res_history_cap;  /* capacity of res_history                                        */
    int64_t res_history_len;  /* entries written                                                 */
    double t_kernel[8];       /* see GMRES_T_*                                                   */
    int64_t kernel_launches;  /* kernels this library launched during the solve                  */
    double solve_seconds;     /* host wall-clock time of the solve                              */
} gmres_stats_t;

typedef struct gmres_ctx *gmres_handle_t;

/* ---- lifecycle ----------------------------------------------------------------------------- */

/* gmres_default_params: fill *p with the defaults listed in gmres_params_t. */
void gmres_default_params(gmres_params_t *p);

/* gmres_create: copy A to the current device, make its FP32 copy (round to nearest; Section
 * III-B keeps both copies; when slices of 32 rows padded to their longest row add at most a
 * quarter to the nonzeros, also a sliced SELL-32 copy of the FP32 values, read by the fused SpMV
 * of GMRES-IR), allocate the workspace for restart length m (1 <= m <= 128) and,
 * if poly_degree > 0, build the GMRES polynomial of that degree (Section III-D): poly_degree+1
 * FP64 Arnoldi steps from poly_start (n doubles, host or device; NULL = all ones), harmonic
 * Ritz values as roots, modified Leja order.  The build and the copies are not part of any
 * solve time.  *out receives the handle.  Errors: INVALID_ARG (CSR checks fail, m or degree
 * out of range, unsupported precision mix), OOM, CUDA. */
int gmres_create(const gmres_csr_t *A, int m, int poly_degree, gmres_precisions_t prec,
                 const double *poly_start, gmres_handle_t *out);

/* gmres_set_tuning / gmres_get_tuning: the launch shapes of later solves on h (the cycle graph
 * is rebuilt when they change).  Fields out of range give GMRES_ERR_INVALID_ARG. */
int gmres_set_tuning(gmres_handle_t h, const gmres_tuning_t *t);
int gmres_get_tuning(gmres_handle_t h, gmres_tuning_t *t);

/* gmres_autotune: time GMRES-IR cycles of h on right-hand side b (host or device, n doubles) under
 * a grid of launch shapes and keep the fastest on h.  Candidates: sweep stage target
 * {24 (default), 16, 32} KB x sweep CTAs per SM {auto, 1, 2, 3} x SpMV CTAs per SM {occupancy, 4},
 * then, with the best of those, SpMV lanes per row from a quarter to four times the automatic
 * choice.
 * Each candidate runs one untimed cycle (capturing its graph) and then `cycles` timed cycles from
 * x = 0 with tolerance 0 and full inner cycles; the cost is wall seconds per inner iteration.
 * best (may be NULL) receives the chosen shapes; best_s_per_iter and default_s_per_iter (may be
 * NULL) the cost of the chosen and of the all-default shapes.  h's solve parameters are left as
 * they were.  1 <= cycles <= 100. */
int gmres_autotune(gmres_handle_t h, const double *b, int cycles, gmres_tuning_t *best,
                   double *best_s_per_iter, double *default_s_per_iter);

/* gmres_set_block_jacobi: right-precondition later solves of h with block Jacobi (Section III-D;
 * Section V-G uses block sizes 1 and 42 after a reverse Cuthill-McKee reordering).  With
 * reorder = 1 the unknowns are ordered by RCM (symmetric pattern of A + A^T; components in turn,
 * each started at its unvisited node of smallest degree, smallest index on ties, neighbours in
 * increasing (degree, index) order, then the whole order reversed); block b is the index set
 * I_b = order[b k, (b+1) k) (the last may be shorter) and M^{-1} v sets z[I_b] = A[I_b, I_b]^{-1} v[I_b].
 * Nothing is permuted: b, x and every other entry point keep the caller's ordering.  The block
 * inverses are formed on the host in FP64 (Gauss-Jordan with partial pivoting, all host threads)
 * and kept in FP64 and FP32; GMRES-IR applies them in FP32, gmres_solve_fp64 in prec.precond.
 * block_size: 1..64, or 0 to remove the preconditioner.  A handle with a polynomial gets
 * INVALID_ARG; a singular block gives INVALID_ARG.  gmres_precond_apply applies it;
 * gmres_precond_apply_noalloc returns UNSUPPORTED for it. */
int gmres_set_block_jacobi(gmres_handle_t h, int block_size, int reorder);

/* gmres_block_jacobi_perm: copy the ordering (order[new] = old, n entries) into perm
 * (cap >= n).  INVALID_ARG if no block Jacobi is set. */
int gmres_block_jacobi_perm(gmres_handle_t h, int32_t *perm, int64_t cap);

/* gmres_destroy: free every device and host resource of the handle.  NULL is accepted. */
int gmres_destroy(gmres_handle_t h);

/* gmres_set_stream: the caller's stream (a cudaStream_t; NULL = the legacy default stream) that
 * further calls on h are ordered after (inputs) and before (outputs). */
int gmres_set_stream(gmres_handle_t h, void *cuda_stream);

/* gmres_set_params: replace the solve parameters (validated; INVALID_ARG on bad values). */
int gmres_set_params(gmres_handle_t h, const gmres_params_t *p);

/* ---- solves -------------------------------------------------------------------------------- */

/* gmres_ir_solve: GMRES-IR (Algorithm 2).  b: n FP64 values (host or device, read only);
 * x: n FP64 values (host or device), initial guess on entry, solution on return.  The FP64
 * residual is checked only at restarts; the solve ends when ||b - A x|| / ||b|| <= tol.
 * stats may be NULL.  Returns OK, NOT_CONVERGED, NAN, STAGNATION or an error. */
int gmres_ir_solve(gmres_handle_t h, const double *b, double *x, double tol, gmres_stats_t *stats);

/* gmres_solve_fp64: plain FP64 GMRES(m) (Algorithm 1 with CGS2), right-preconditioned by the
 * polynomial when one was built, applied in prec.precond: F64, or F32 (FP32 matrix values and
 * vectors inside an otherwise FP64 solve, variant (a) of Section III-D).  Stops inside a cycle when the implicit residual reaches
 * tol ||b||, then checks the explicit residual (Section V-F).  Same buffers and returns as
 * gmres_ir_solve, plus LOSS_OF_ACCURACY. */
int gmres_solve_fp64(gmres_handle_t h, const double *b, double *x, double tol,
                     gmres_stats_t *stats);

/* gmres_status_string: static text for a status code (never NULL). */
const char *gmres_status_string(int status);

/* ---- building blocks (device pointers; used by tests and tools) ---------------------------- */

/* gmres_solve_fp32: single-precision GMRES(m): Algorithm 1 with CGS2 entirely in FP32 (b and x0
 * rounded to FP32, FP32 residual, basis and update; x holds FP32 values), stop rules as
 * gmres_solve_fp64 with the relative residual measured in FP32.  It cannot in general reach
 * FP64-level tolerances; it is the first phase of GMRES-FD.  Requires basis = F32.  Buffers and
 * returns as gmres_ir_solve, plus LOSS_OF_ACCURACY. */
int gmres_solve_fp32(gmres_handle_t h, const double *b, double *x, double tol, gmres_stats_t *stats);

/* gmres_fd_solve: GMRES-FD (Section III-C; studied in Section V-A): single-precision GMRES(m)
 * for switch_iters iterations (or until it meets tol), then FP64 GMRES(m) from that iterate
 * until ||b - A x|| / ||b|| <= tol (the FP64 phase stops at once if the iterate qualifies).
 * switch_iters = 0 is plain FP64 GMRES.  params.maxiter caps the total.  stats (may be NULL) sums both phases; its residual
 * history holds the FP32 phase's entries followed by the FP64 phase's.  fp32_iters (may be NULL)
 * receives the iterations of the FP32 phase.  Returns the FP64 phase's status or an error. */
int gmres_fd_solve(gmres_handle_t h, const double *b, double *x, double tol, int64_t switch_iters,
                   gmres_stats_t *stats, int64_t *fp32_iters);

/* gmres_spmv: y = A x with the handle's matrix.  prec = F64: x, y are double; prec = F32:
 * float values, float x and y, FP32 accumulation (the inner SpMV of Section III-B). */
int gmres_spmv(gmres_handle_t h, gmres_prec_t prec, const void *x, void *y);

/* gmres_precond_apply: z = p(A) v with the handle's polynomial in precision prec (F32: float
 * vectors; F64: double vectors).  Without a polynomial, z = v. */
int gmres_precond_apply(gmres_handle_t h, gmres_prec_t prec, const void *v, void *z);

/* gmres_poly_roots: copy the Leja-ordered roots theta_k of the residual polynomial
 * pi(t) = prod_k (1 - t / theta_k) = 1 - t p(t) into re[], im[] (host, capacity cap).  *count
 * receives degree+1 (0 without a polynomial). */
int gmres_poly_roots(gmres_handle_t h, double *re, double *im, int cap, int *count);

/* gmres_arnoldi: run k <= m steps of the inner Arnoldi process (Algorithm 1 with fused CGS2)
 * from r0 (device, n doubles) in the given mode: inner = F64 uses the FP64 kernels, F32 the
 * FP32 kernels with the handle's basis precision.  H (host, (k+1) x k column-major FP64)
 * receives the Hessenberg matrix; V (device, n x (k+1) column-major FP64, or NULL) receives the
 * normalised basis (with params.orth = 1 its last column is the candidate before its delayed
 * second pass, not a basis vector).  *steps receives the steps taken (fewer than k after a lucky
 * breakdown). */
int gmres_arnoldi(gmres_handle_t h, gmres_prec_t inner, int k, const double *r0, double *H,
                  double *V, int *steps);

/* gmres_test_expire_wait: testing hook of the bounded waits.  The pipelined sweeps wait for
 * their bulk copies with a time limit (200 ms) instead of forever; when one gives up, the CTA
 * waits (bounded) for its other copies in flight, flags the cycle, and the solve returns
 * GMRES_TIMEOUT.  With armed = 1 the next solve on h (gmres_ir_solve, gmres_solve_fp64,
 * gmres_solve_fp32) has one CTA of its first second-pass sweep skip one bulk copy, so that wait
 * runs out for real; the hook then disarms itself.  Costs about half a second.  Only for tests
 * of that path; nothing else changes. */
int gmres_test_expire_wait(gmres_handle_t h, int armed);

/* gmres_hessenberg_eigvals: eigenvalues of a real upper Hessenberg k x k matrix (host,
 * column-major) by the implicit double-shift QR algorithm; the host routine of the polynomial
 * build.  re/im (host, k each).  Returns INVALID_ARG if it fails to converge. */
int gmres_hessenberg_eigvals(int k, const double *H, double *re, double *im);

/* ---- batched block GMRES-IR ---------------------------------------------------------------- */

typedef struct gmres_batch_ctx *gmres_batch_t;

typedef struct {
    int status;               /* OK when every system converged                                 */
    int64_t cycles;           /* block cycles run (all systems in lock step)                    */
    int64_t block_steps;      /* block Arnoldi steps summed over systems                        */
    int64_t converged_systems;
    int64_t breakdowns;       /* Cholesky-QR breakdowns (the system's cycle ended early)         */
    double max_rel_res;       /* largest ||b - A x|| / ||b|| over all columns of all systems      */
    double *per_system_rel;   /* caller buffer (or NULL): per system, largest column residual    */
    int64_t *per_system_cycles; /* caller buffer (or NULL): cycles each system ran              */
    int64_t per_system_cap;   /* capacity of the two buffers                                    */
    int64_t kernel_launches;
    double solve_seconds;
    double t_kernel[4];       /* with profiling on: seconds per kernel class (GMRES_BT_*)       */
    int64_t class_launches[4];/* with profiling on: launches per kernel class                   */
} gmres_batch_stats_t;

enum {  /* kernel classes of a block cycle (gmres_batch_stats_t.t_kernel) */
    GMRES_BT_SPMM = 0,        /* block SpMV W = A Q_k                                           */
    GMRES_BT_SWEEP = 1,       /* block CGS2 sweeps (projection, update + projection, update)    */
    GMRES_BT_SMALL = 2,       /* per-system small kernels (coefficients, Cholesky QR, Givens)   */
    GMRES_BT_CYCLE = 3        /* cycle start and end (start block, solution, FP64 residual)     */
};

/* gmres_batch_create: nsys independent square CSR systems A[0..nsys) (host or device arrays each),
 * solved together by block GMRES-IR with nrhs right-hand sides each (nrhs must be 8) and m block
 * steps per cycle (1..32).  Block Arnoldi with block CGS2 (Algorithm 1 / Section III-A applied to
 * a block of vectors), Cholesky QR of each new block, FP32 inner arithmetic with a BF16 basis
 * (prec must be {F32, F32, BF16, F32}), FP64 residual and update (Algorithm 2).  The paper has no
 * batched or block method; this follows its GMRES-IR per block.  Errors as gmres_create. */
int gmres_batch_create(int nsys, const gmres_csr_t *A, int nrhs, int m, gmres_precisions_t prec,
                       gmres_batch_t *out);

/* gmres_batch_destroy: free the batch (NULL accepted). */
int gmres_batch_destroy(gmres_batch_t b);

/* gmres_batch_set_stream: order the batch's work after / before cuda_stream. */
int gmres_batch_set_stream(gmres_batch_t b, void *cuda_stream);

/* gmres_batch_set_profiling: 1 = later solves launch each block cycle directly (no graph) and
 * time the kernel classes with CUDA events on the batch's stream (stats.t_kernel); 0 = graphs. */
int gmres_batch_set_profiling(gmres_batch_t b, int on);

/* Launch shapes of the batched solver.  0 in a field = the default.  The chunk size groups tiles
 * into sweep work items, so the FP32 partial Gram and projection sums (and the last bits of the
 * inner iterates) depend on it; every choice reaches the same FP64 tolerance. */
typedef struct {
    int chunk_tiles;          /* 128-row tiles per sweep work item (0 = 16; 4..64); cycles with
                                 few tiles left use items of half this size (at least 4)       */
    int sweep_smem_kb;        /* shared memory a sweep CTA's pipeline is sized for, in KB
                                 (0 = 64, three CTAs per SM; 64..220)                          */
    int sweep_max_stages;     /* pipeline stages at most (0 = 3; 2..8; at least 2 are used)     */
    int reserved;             /* must be 0                                                     */
} gmres_batch_tuning_t;

/* gmres_batch_set_tuning / gmres_batch_get_tuning: the launch shapes of later solves on b (the
 * cycle graph is rebuilt; a new chunk size reallocates the per-chunk partial sums).  Fields out
 * of range give GMRES_ERR_INVALID_ARG and leave the shapes unchanged. */
int gmres_batch_set_tuning(gmres_batch_t b, const gmres_batch_tuning_t *t);
int gmres_batch_get_tuning(gmres_batch_t b, gmres_batch_tuning_t *t);

/* gmres_batch_autotune: solve the batch from X = 0 with right-hand sides B (host or device, the
 * layout of gmres_batch_ir_solve) under a grid of launch shapes and keep the fastest on b.
 * Candidates: chunk tiles {16 (default), 8, 32} x sweep pipeline {default, 100 KB with up to 4
 * stages, 220 KB (one CTA per SM) with up to 8 stages}.  Each candidate runs one cycle (capturing
 * its graph), then one timed solve to tol or max_cycles; the cost is its wall time.  best (may be
 * NULL) receives the chosen shapes; best_seconds and default_seconds (may be NULL) the solve time
 * of the chosen and of the default shapes.  Allocates one solution-sized device buffer while it
 * runs.  On an error the previous shapes are restored. */
int gmres_batch_autotune(gmres_batch_t b, const double *B, double tol, int max_cycles,
                         gmres_batch_tuning_t *best, double *best_seconds, double *default_seconds);

/* gmres_batch_ir_solve: B and X (host or device) hold the systems one after another, system s an
 * n_s x nrhs column-major block (each column contiguous); X is the initial guess on entry and the
 * solution on return.  Every column of every system is solved to ||b - A x|| / ||b|| <= tol, or
 * until max_cycles block cycles have run.  One CUDA graph replays a block cycle of all systems;
 * converged systems are skipped.  stats may be NULL.  Returns OK or NOT_CONVERGED, or an error. */
int gmres_batch_ir_solve(gmres_batch_t b, const double *B, double *X, double tol, int max_cycles,
                         gmres_batch_stats_t *stats);

/* ---- learned parameter controller (small MLP, own FP32 kernels) ------------------------------ */
/* The paper tunes restart length, inner tolerance and polynomial degree by hand (Sections V-E,
 * V-F); this network proposes them.  Architecture 12 -> 64 (ReLU) -> 64 (ReLU) -> 9 outputs:
 * [0..2] logits of m in {25, 50, 100}, [3] log10 inner tolerance, [4..7] logits of the polynomial
 * degree in {0, 10, 25, 40}, [8] log of the predicted time ratio against the default parameters.
 * Parameters: one FP32 array W1[64][12], b1[64], W2[64][64], b2[64], W3[9][64], b3[9]. */
typedef struct gmres_mlp_ctx *gmres_mlp_t;

/* gmres_mlp_num_params: length of the parameter array (5577). */
int gmres_mlp_num_params(void);

/* gmres_mlp_create: a network with the given initial parameters (host or device array). */
int gmres_mlp_create(const float *params, gmres_mlp_t *out);

/* gmres_mlp_destroy: free the network (NULL accepted). */
int gmres_mlp_destroy(gmres_mlp_t c);

/* gmres_mlp_get_params: copy the current parameters into params (host or device). */
int gmres_mlp_get_params(gmres_mlp_t c, float *params);

/* gmres_mlp_forward: Y[B][9] = net(X[B][12]), row-major; X, Y host or device (1 <= B <= 65536).
 * Device inputs must be complete before the call: the network runs on its own stream, which the
 * call synchronises before it returns. */
int gmres_mlp_forward(gmres_mlp_t c, const float *X, int B, float *Y);

/* gmres_mlp_gradient: gradient (nparams, host or device) of the mean loss
 * CE(m) + (y3 - tl)^2 + CE(d) + (y8 - rt)^2 over the batch; X, labels host or device (staged
 * into the network's own buffers): mc, dc class indices (-1 or out of range = no label), tl, rt targets.  loss4 (host, 4 floats, may be NULL) receives the
 * four batch-mean terms.  Deterministic (fixed summation order). */
int gmres_mlp_gradient(gmres_mlp_t c, const float *X, const int *mc, const float *tl,
                       const int *dc, const float *rt, int B, float *grad, float *loss4);

/* gmres_mlp_train_step: one Adam step (beta 0.9 / 0.999, eps 1e-8) with learning rate lr on the
 * same loss; inputs as gmres_mlp_gradient. */
int gmres_mlp_train_step(gmres_mlp_t c, const float *X, const int *mc, const float *tl,
                         const int *dc, const float *rt, int B, float lr, float *loss4);

/* ---- learned parameter controller for C callers ---------------------------------------------- */
/* The trained network of a checkpoint chooses (m, inner tolerance, polynomial degree) for a system
 * (the parameters Sections V-E and V-F tune by hand).  Features (12, in this order): log10 n; mean
 * and max nonzeros per row; min over rows of |a_ii| / sum_{j != i} |a_ij|; ||A - A^T||_F /
 * ||A||_F; log10(max |(A - A^T)_ij| / dscale + 1e-12); min and max over rows of
 * (a_ii -+ sum_{j != i} |a_ij|) / dscale (Gershgorin); the largest and smallest |eigenvalue| of
 * H_k of a k = min(10, n - 1)-step FP64 Arnoldi run from b, / dscale; log10 of the relative
 * residual drop of one default GMRES-IR cycle (FP32 basis, m = 50, full cycle, no polynomial)
 * from x = 0; log10 of that cycle's wall time in seconds (second run, its CUDA graph captured by
 * the first).  dscale = sum |a_ii| / n (1 if that is 0).  The matrix must not hold duplicate
 * entries. */
typedef struct gmres_ctrl_ctx *gmres_ctrl_t;

typedef struct {
    int m;                    /* restart length: 25, 50 or 100                                  */
    double inner_tol;         /* GMRES-IR inner tolerance (gmres_params_t.inner_tol); 0 = full
                                 inner cycles                                                   */
    int poly_degree;          /* polynomial degree 0, 10, 25 or 40 (a create-time parameter)     */
    int choice;               /* 0: the network's choice; 1: the default (m = 50, full cycles,
                                 no polynomial), taken when the predicted best time is >= 0.95 x
                                 the default's; 2: the checkpoint's best fixed setting, taken when
                                 the predicted gain is not beyond that setting's median gain on
                                 the training systems (predicted ratio >= its ratio / 0.95)      */
    double predicted_ratio;   /* exp(output 8): predicted best time / default time               */
    double outputs[9];        /* raw network outputs (FP32 forward pass)                         */
    double features[12];      /* the features the decision used                                  */
} gmres_suggestion_t;

/* gmres_controller_load: read a checkpoint: "GMRESMLP", then little-endian u32 version (1 or 2),
 * u32 number of parameters (5577), f64 feature means[12], f64 standard deviations[12], f32
 * parameters (the layout of gmres_mlp_create), version 2 only: i32 m, f64 inner tolerance, i32
 * degree, f64 median time ratio of the best fixed setting; last a u32 CRC-32 (zlib's) of the bytes
 * between the magic and the CRC.  The network is created on the current device.  Errors:
 * INVALID_ARG (no such file, bad magic, size, version or CRC), OOM, CUDA. */
int gmres_controller_load(const char *path, gmres_ctrl_t *out);

/* gmres_controller_destroy: free the controller (NULL accepted). */
int gmres_controller_destroy(gmres_ctrl_t c);

/* gmres_controller_features: the 12 features of h's matrix with right-hand side b (n doubles,
 * host or device).  GPU work on h's device and the stream set with gmres_set_stream: one row
 * kernel over the FP64 CSR, and on a temporary handle (a copy of the matrix, released before the
 * call returns) the Arnoldi run and two default IR cycles.  features: host, 12 doubles.  The last
 * feature is a wall time, so it varies between calls. */
int gmres_controller_features(gmres_handle_t h, const double *b, double *features);

/* gmres_controller_decide: the suggestion for given features (host, 12 doubles): standardised
 * with the checkpoint's means and deviations, rounded to FP32, one forward pass with the
 * library's MLP kernels, then the rule described at gmres_suggestion_t.choice (argmax of the m
 * and degree logits; inner tolerance 10^clip(output 3, -6, -2)).  Deterministic. */
int gmres_controller_decide(gmres_ctrl_t c, const double *features, gmres_suggestion_t *out);

/* gmres_controller_suggest: gmres_controller_features, then gmres_controller_decide.  To use it:
 * create the solving handle with poly_degree = out.poly_degree and set params.m = out.m,
 * params.inner_tol = out.inner_tol. */
int gmres_controller_suggest(gmres_ctrl_t c, gmres_handle_t h, const double *b,
                             gmres_suggestion_t *out);

/* gmres_precond_apply_noalloc: the same z = p(A) v as gmres_precond_apply, for callers that
 * must not allocate device memory while they run (a memory pool or arena that owns the GPU, a
 * real-time loop where cudaMalloc's implicit synchronisation is not allowed, a plug-in whose
 * host forbids allocation).  The paper has no counterpart; this is a service of the library.
 * v, z: device vectors of n values (double for F64, float for F32); z must not overlap v
 * (GMRES_ERR_INVALID_ARG otherwise: z is written while other rows of v are still being read).
 * The work vectors live in a fixed 12 MiB (+256 bytes) array in the library's device image,
 * present on every GPU that loads the library until the process exits; nothing is allocated.
 * Limit: n <= 524288 (2^19), larger handles get GMRES_ERR_INVALID_ARG.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture on the device.  All calls share the one array, which keeps the last call's
 * contents: calls whose GPU work overlaps (other streams, other threads, other handles on the
 * same device) race and must be serialised by the caller.  Every call synchronises the handle's
 * stream and returns with z complete. */
int gmres_precond_apply_noalloc(gmres_handle_t h, gmres_prec_t prec, const void *v, void *z);

#ifdef __cplusplus
}
#endif

#endif /* GMRESB3_H */
