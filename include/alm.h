/*
 * alm.h -- C ABI of the GB300 (sm_103a) ALM-BM hot path.
 *
 * The library solves the semidefinite program (P) of arXiv 2505.15775, Sec. 1.2,
 *
 *     min <C, X>   s.t.   [A(X)]_k = <A_k, X> = b_k  (k = 0..m-1),   X >= 0,
 *
 * through the Burer-Monteiro factorisation X = R R^T (R is n x r, the paper's F)
 * and the augmented Lagrangian
 *
 *     L_sigma(R R^T, y) = <C, RR^T> + <y, b - A(RR^T)> + sigma/2 ||A(RR^T) - b||^2
 *
 * (Eq. AL / AL-BM; the paper's penalty rho is called sigma here).  Throughout:
 *
 *     w = y - sigma (A(RR^T) - b)       the ALM multiplier update (Eq. ALM)
 *     S = C - A^*(w) = grad_X L_sigma   the dual slack map Z(w) at w
 *     G = grad_R L_sigma = 2 S R        the BM gradient (Sec. 4.2)
 *
 * Conventions
 * -----------
 * - Symmetric matrices (C and every A_k) are given by upper-triangle entries
 *   (i <= j).  An off-diagonal entry v at (i, j) means M_ij = M_ji = v, so it
 *   contributes 2 v X_ij to <M, X>.  Repeated entries add up.
 * - C may carry a low-rank part sum_l s_l u_l u_l^T (u_l dense, length n); the
 *   Lovasz theta SDP's -J is s = -1, u = 1.
 * - Device arrays (R, D, G, v, y, AX) are caller-owned device memory.  R, D and G
 *   are row-major n x ldr in the handle's precision (double for ALM_FP64, float
 *   for ALM_FP32); only columns 0..r-1 are read; ldr * element size must be a
 *   multiple of 16 bytes and the base address 16-byte aligned.  Outputs G write
 *   zeros into columns r..ldr-1.  y and AX are double, length m.
 * - Every call runs on the handle's stream.  Calls that return host scalars
 *   (pointers documented "host") synchronise that stream before returning.
 * - Every call returns an alm_status; on error, alm_last_error(h) gives a
 *   one-line message.  No C++ exception crosses this boundary.  A handle is not
 *   thread-safe: calls on one handle must not overlap.
 */
#ifndef ALM_H
#define ALM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct alm_handle alm_handle;
typedef void *alm_stream_t; /* a cudaStream_t; NULL = the legacy default stream */

typedef enum {
    ALM_OK = 0,
    ALM_ERR_INVALID_ARG = 1,   /* bad size, index, pointer alignment or option */
    ALM_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has the name) */
    ALM_ERR_OOM = 3,           /* device or host allocation failed */
    ALM_ERR_NUMERIC = 4,       /* non-finite value in a reduction or step */
    ALM_ERR_NOT_CONVERGED = 5, /* outer/inner iteration cap reached; stats filled */
    ALM_ERR_TIMEOUT = 6,       /* a bounded wait ran out */
    ALM_ERR_UNBOUNDED = 7      /* L_sigma unbounded below along a direction */
} alm_status;

enum { ALM_FP64 = 0, ALM_FP32 = 1 };           /* arithmetic of R, D, G, S and the SpMV */
enum { ALM_INNER_CG = 0, ALM_INNER_GD = 1 };   /* inner direction */
enum { ALM_SIGMA_FIXED = 0, ALM_SIGMA_ADAPTIVE = 1 };

/* Problem data of (P), host arrays copied by alm_create (the caller keeps them). */
typedef struct {
    int64_t n, m;
    int64_t c_nnz;                 /* upper-triangle COO of C */
    const int32_t *c_i, *c_j;
    const double *c_v;
    int32_t c_lr_k;                /* number of low-rank terms of C (0..4) */
    const double *c_lr_u;          /* c_lr_k x n, row-major */
    const double *c_lr_s;          /* c_lr_k */
    int64_t a_nnz;                 /* entries of the A_k: constraint a_k[e], upper (a_i[e], a_j[e]) */
    const int32_t *a_k, *a_i, *a_j;
    const double *a_v;
    const double *b;               /* m */
} alm_problem;

/* Options (alm_default_options fills every field).  The readings of what the
 * paper leaves open are documented beside each field. */
typedef struct {
    int32_t precision;        /* ALM_FP64 or ALM_FP32 (FP32 bulk, FP64 reductions/dual) */
    int32_t r_max;            /* rank cap of the solve, 1..32 */
    double sigma0;            /* initial penalty */
    int32_t sigma_rule;       /* ALM_SIGMA_FIXED, or ALM_SIGMA_ADAPTIVE: sigma <- min(2 sigma,
                                 sigma_max) when the primal KKT term fell by < 4x */
    double sigma_max;
    double eps;               /* stop when the relative KKT error (Sec. 6) <= eps */
    int32_t max_outer;        /* ALORA iterations (Alg. 1 "repeat") */
    int32_t max_inner;        /* inner steps per outer iteration */
    int32_t inner_method;     /* ALM_INNER_CG (Polak-Ribiere+) or ALM_INNER_GD */
    double inner_rel;         /* tau_in = max(inner_floor*eps, min(inner_rel*KKT_prev, */
    double inner_floor;       /*          inner_decay*tau_in_prev)); inner stop when    */
    double inner_start;       /*          ||G||_F/(1+||C||_F) <= tau_in; tau_in starts at */
    double inner_decay;       /*          inner_start                                     */
    int32_t lanczos_k;        /* Lanczos basis length per restart cycle, 2..64 */
    int32_t lanczos_max_restarts;
    double lanczos_tol;       /* stop when ||S v - theta v|| <= tol * ||S||_est */
    uint64_t seed;            /* Lanczos start vector (SplitMix64 counter generator) */
    int32_t chunk;            /* inner steps enqueued between two host checks */
    int32_t use_graph;        /* capture each chunk of inner steps as a CUDA graph */
    int32_t profile;          /* time the SpMM launches with CUDA events */
    int32_t verbose;          /* 1: one line per outer iteration on stderr */
    int32_t inner_precond;    /* 1: row-block Jacobi preconditioned CG (P_i = 2 S_ii I + 4 sigma a_i^2
                                 r_i r_i^T, the row block of the Hessian); 0: plain */
    int32_t lanczos_warm;     /* 1: inside a solve, start each Lanczos from the previous outer
                                 iteration's Ritz vector plus a seeded perturbation of norm 0.05;
                                 0 (default): from a fresh seeded vector every time.  Measured on
                                 the MaxCut workloads (-24% to -45% Lanczos products); off by
                                 default because it is not validated on general constraints */
    int32_t fallback_inner;   /* batched solver only: an instance that has taken more than this many
                                 inner steps without converging restarts once from a seeded cold
                                 start (uniform rows, normalised; y = 0); 0 (default) = never.  The
                                 cold start is the fallback of a learned warm start. */
    int32_t growth_k;         /* directions per rank-growth step (Alg. 1 grows along the
                                 eigenvectors of grad_X L with negative eigenvalues and an r x r SDP):
                                 1 (default) = the smallest eigenpair and its closed-form step;
                                 2..4 = up to that many eigenpairs below -tau_lambda (Lanczos with the
                                 found ones deflated) and the k x k SDP over the PSD cone, then
                                 R <- [R, V S^{1/2}].  Several directions need every constraint to
                                 be a diagonal selector X_ii = b_i (the MaxCut form); other problems
                                 grow by one direction. */
} alm_options;

/* Solve statistics (alm_solve fills it). */
typedef struct {
    int32_t status;           /* alm_status of the solve */
    int32_t outer, inner_total, rank;
    double sigma;             /* final penalty */
    double kkt[3];            /* primal, dual, gap terms of the relative KKT error */
    double objective;         /* <C, X> at the end */
    double lambda_min;        /* last lambda_min(C - A^* y) estimate */
    int64_t lanczos_matvecs;
    int64_t kernel_launches;  /* kernels this library launched inside the solve */
    int64_t spmm_launches;    /* SpMM launches timed with CUDA events (profile mode: the
                                 first SpMM of every chunk of inner steps) */
    double spmm_ms;           /* their total device time (ms) */
    double spmm_bytes;        /* their total algorithmic bytes: row pointers, column
                                 indices and values of S, diag(S), and the n x r_pad
                                 blocks R, G_prev, D_prev read and G written */
    int32_t spmm_rank_pad;    /* padded rank of the last timed SpMM */
    int32_t growth_steps;
    double time_ms;           /* wall time of the solve on the host */
    double step_ms[5];        /* profile mode: device time of the kernels of the timed inner
                                 steps, by class: slack/constraint map, SpMM, direction,
                                 line search, update (summed over the timed steps) */
    double lanczos_ms;        /* wall time spent in the Lanczos eigensolves */
    double ls_bytes;          /* profile mode: algorithmic bytes of the timed line-search
                                 launches (step_ms[3]): the n x r_pad blocks R, Z, D_old
                                 read and D_new written, the strict upper pattern's column
                                 indices and values, and the per-row selector record */
} alm_stats;

/* Fill *o with the defaults. */
void alm_default_options(alm_options *o);

/* Validate the problem (indices in range, i <= j, finite values, n, m >= 1),
 * build the aggregated sparsity pattern of C and the A_k (Sec. 1.2's data in
 * the upper-triangle CSR, full symmetric CSR and constraint-map layouts the
 * kernels read) and upload it.  s is the stream every later call uses.
 * On error *h is NULL and the status says why (ALM_ERR_INVALID_ARG, ALM_ERR_OOM,
 * ALM_ERR_CUDA); alm_last_error(NULL) then returns the message.
 *
 * Host-side fault injection, for testing the error paths without a GPU fault: when the
 * environment variable ALM_FAULT_INJECT is set when alm_create runs, the call
 *   "nan_b"  validates a copy of the problem whose b[0] is NaN (ALM_ERR_INVALID_ARG),
^ *   "csr"    validates a copy whose first constraint entry has row index n, out of range
 *            (ALM_ERR_INVALID_ARG),
 *   "oom"    fails its first device allocation as cudaMalloc would (ALM_ERR_OOM),
 * and frees what it allocated.  Any other value is rejected with ALM_ERR_INVALID_ARG.  The
 * caller's arrays are never modified. */
alm_status alm_create(alm_handle **h, const alm_problem *p, const alm_options *o, alm_stream_t s);

/* Free every device and host resource of h (NULL is allowed). */
void alm_destroy(alm_handle *h);

/* Last error message of h, or of the last failed alm_create when h is NULL. */
const char *alm_last_error(const alm_handle *h);

/* Sizes of the built pattern: [n, m, nnz of the strict upper pattern, nnz of the
 * full off-diagonal pattern, number of selector constraints, number of general
 * constraints, 1 if S's off-diagonal values depend on y].  out: host, 7 entries. */
alm_status alm_pattern_info(const alm_handle *h, int64_t *out);

/* One inner step of the solver's inner loop (Sec. 4.2: the BM gradient of Eq. AL-BM,
 * preconditioned Polak-Ribiere+ directions, the exact step along them from the quartic of
 * Eq. AL), run from a caller-given state with the very kernels alm_solve uses, for problems
 * whose constraints are all X_ii = b_i and whose rows have at most 16 entries:
 *   R_out = R + alpha D                      (the pending step of the previous line search)
 *   S_ii  = C_ii - (y_i - sigma (|r_out,i|^2 - b_i)),  G = 2 S R_out
 *   Z     = P^{-1} G  (row blocks P_i = 2 max(S_ii, f) I + 4 sigma a_i^2 r_i r_i^T) when the
 *           handle's inner_precond is on, else Z = G
 *   beta  = max(0, (<Z, G> - <G, Z_old>) / zg_prev), and 0 when zg_prev <= 0 or when
 *           -<Z, G> + beta <G, D> >= 0 (not a descent direction)
 *   D_new = -Z + beta D,  q1..q4 the quartic coefficients of L(R_out + t D_new) (q1 =
 *           <G, D_new>), alpha_new = argmin_{t >= 0} of that quartic.
 *   R, D, R_out, Z, D_new  device, n x ldr in the working precision, r columns; Z holds Z_old
 *                          on entry and Z on return; R_out, Z, D_new are separate buffers.
 *   y                      device, m doubles;  diag_out: device, n doubles (may be NULL): S_ii.
 *   out                    host, 11 doubles: |G|^2, <G, Z_old>, <G, D>, <Z, G>, beta, q0 (not
 *                          computed: the solver does not need it), q1, q2, q3, q4, alpha_new.
 * Synchronises the handle's stream.  Other problems: ALM_ERR_INVALID_ARG. */
alm_status alm_cg_step(alm_handle *h, const void *R, const void *D, int32_t r, int32_t ldr, const double *y,
                       double sigma, double alpha, double zg_prev, void *R_out, void *Z, void *D_new,
                       double *diag_out, double *out);

/* Launch shape of the two kernels of an inner CG step in the fused ELL form (problems
 * whose constraints are all X_ii = b_i and whose rows have at most 8 off-diagonal entries,
 * at ranks of 16 or more columns; other cases always use variant 0): variant 0 loads each
 * row group's rows into registers; variant 1 stages them in shared memory with
 * asynchronous copies, `stages` buffers per row group (2..4; rows in flight = stages - 1),
 * `threads` per CTA (128 or 256).  The paper has no counterpart (it is a property of this
 * implementation, not of Alg. 1); every shape computes the same iteration up to FP
 * rounding order. */
typedef struct {
    int32_t variant, stages, threads;
} alm_inner_shape;
/* Set / read the shape of h (the default: variant 1, 2 stages, 128 threads).  Invalid shapes
 * are rejected with ALM_ERR_INVALID_ARG. */
alm_status alm_set_inner_shape(alm_handle *h, const alm_inner_shape *shape);
alm_status alm_get_inner_shape(const alm_handle *h, alm_inner_shape *shape);
/* The autotuner's candidate shapes in the order alm_autotune times them; returns their
 * count and writes them to out when out is not NULL (it has room for 16). */
int32_t alm_inner_shapes(alm_inner_shape *out);
/* Autotuner: time `steps` (even, 2..256) inner CG steps of the fused loop from the factor R
 * (device, n x ldr, r columns) and dual y (device, m doubles) at sigma0, in every candidate
 * shape, and keep the fastest on h.  times_ms (host, may be NULL, room for 16) gets each
 * shape's time, best (may be NULL) the chosen shape, count the number of shapes timed (0
 * when the problem does not use the fused loop, or when the shape came from the cache).
 * cache_path (may be NULL): a JSON-lines file of tuned shapes keyed by (n, nnz of the full
 * pattern, r, precision, ELL widths); a hit sets the cached shape without timing
 * (*from_cache = 1), a miss tunes and appends a line.  R and y are not modified; on a miss
 * the handle's solver buffers are (so a later alm_checkpoint needs a new solve first). */
alm_status alm_autotune(alm_handle *h, const void *R, int32_t r, int32_t ldr, const double *y, int32_t steps,
                        const char *cache_path, alm_inner_shape *best, double *times_ms, int32_t *count,
                        int32_t *from_cache);

/* Constraint map and augmented Lagrangian at X = R R^T (Eq. AL; (a) of the hot
 * path: the fused SDDMM over the aggregated pattern with the scatter into A(X)).
 *   R      device, n x ldr, r columns used.
 *   y      device, m doubles.
 *   L_out  host, may be NULL: L_sigma(RR^T, y).
 *   AX_out device, may be NULL: A(RR^T), m doubles.
 *   CX_out host, may be NULL: <C, RR^T>. */
alm_status alm_eval(alm_handle *h, const void *R, int32_t r, int32_t ldr, const double *y,
                    double sigma, double *L_out, double *AX_out, double *CX_out);

/* Gradient G = 2 S R with S = C - A^*(y - sigma(A(RR^T) - b)) ((b) of the hot
 * path; Sec. 4.2's grad h(F) = 2 grad f(FF^T) F).
 *   G          device, n x ldr (same layout as R; may not alias R).
 *   gnorm2_out host, may be NULL: ||G||_F^2. */
alm_status alm_grad(alm_handle *h, const void *R, int32_t r, int32_t ldr, const double *y,
                    double sigma, void *G, double *gnorm2_out);

/* Exact line search along D ((c) of the hot path): the coefficients of
 * phi(alpha) = L_sigma((R + alpha D)(R + alpha D)^T, y) = sum_k q_k alpha^k,
 * from A(RD^T + DR^T), A(DD^T), <C, RD^T + DR^T> and <C, DD^T>, and
 * alpha* = argmin_{alpha >= 0} phi (smallest among equal minima; 0 if phi does
 * not decrease; +inf and ALM_ERR_UNBOUNDED when phi is unbounded below).
 *   D          device, same layout as R.
 *   coeffs_out host, may be NULL: q0..q4.
 *   alpha_out  host, may be NULL. */
alm_status alm_linesearch(alm_handle *h, const void *R, const void *D, int32_t r, int32_t ldr,
                          const double *y, double sigma, double *coeffs_out, double *alpha_out);

/* Smallest eigenpair of S = C - A^*(w), w = y - sigma(A(RR^T) - b) ((d) of the
 * hot path; Alg. 1's eigenvector of grad_X L, Sec. 6's lambda_min(C - A^* y)
 * when sigma = 0).  Lanczos with full (twice-applied classical Gram-Schmidt)
 * reorthogonalisation, restarted from the Ritz vector.  R may be NULL (r = 0):
 * then A(RR^T) = 0.
 *   lambda_out host: the Ritz value (an upper bound of lambda_min).
 *   v_out      device, may be NULL: unit Ritz vector, n entries (precision of h).
 *   resid_out  host, may be NULL: ||S v - lambda v||_2. */
alm_status alm_lambda_min(alm_handle *h, const void *R, int32_t r, int32_t ldr, const double *y,
                          double sigma, double *lambda_out, void *v_out, double *resid_out);

/* ALORA (Alg. 1) with the options of h: repeat { inner solve of (AL-BM) at
 * fixed y; smallest eigenpair of grad_X L; rank-one growth if lambda_min <
 * -eps(1+||C||_F) and r < r_max; y <- y + sigma(b - A(RR^T)) } until the
 * relative KKT error <= eps.
 *   R       device, n x ldr with ldr >= r_max: in, columns 0..*r_inout-1 hold R0;
 *           out, columns 0..*r_inout-1 hold the final factor.
 *   r_inout host: initial rank in (1..r_max), final rank out.
 *   y       device, m doubles: initial multiplier in, final multiplier out.
 *   stats   host, may be NULL.
 * Returns ALM_OK on convergence, ALM_ERR_NOT_CONVERGED at the outer cap. */
alm_status alm_solve(alm_handle *h, void *R, int32_t ldr, int32_t *r_inout, double *y,
                     alm_stats *stats);

/* Save the ALORA state at the end of the last alm_solve / alm_resume on h (the factor and
 * its rank, y, sigma, the inner tolerance, the last KKT values, the counters and the last
 * Ritz vector that starts the next Lanczos) to the file `path` (raw binary, this build
 * only).  ALM_ERR_INVALID_ARG when there is no state or the file cannot be written. */
alm_status alm_checkpoint(alm_handle *h, const char *path);
/* Per-outer-iteration log of alm_solve and alm_resume: when `path` is set, every later
 * solve appends one JSON object per outer iteration (one line each) to the file:
 *   outer, inner (steps of this iteration's inner solve), inner_total, rank, sigma (the
 *   penalty this iteration used), lambda_min (null when the eigensolve was skipped),
 *   grew (a rank-growth step was taken), kkt [p, d, g] (Sec. 6's relative residuals of
 *   the iterate after the dual update; d is 0 when lambda_min is null), objective
 *   (<C, RR^T>), alpha_last (the last exact step of the inner solve), time_ms {inner,
 *   lanczos, total}.  Non-finite numbers are written as null.  The file is opened in append
 *   mode at each solve and flushed after every line.  path NULL or "" switches it off.
 * ALM_ERR_INVALID_ARG when the file cannot be opened for appending. */
alm_status alm_set_log(alm_handle *h, const char *path);
/* Continue a saved ALORA trajectory: load `path` (written by alm_checkpoint for a handle of
 * the same problem and precision) and run the remaining outer iterations (from the saved
 * count up to this handle's max_outer) exactly as the uninterrupted solve would have.
 * R, ldr, y and stats as in alm_solve (outputs only); r_out gets the final rank.  The
 * checkpoint carries a 64-bit fingerprint of the problem arrays (C, the A_k, b): a file
 * saved for another problem, even of the same n, m and precision, is rejected with
 * ALM_ERR_INVALID_ARG. */
alm_status alm_resume(alm_handle *h, const char *path, void *R, int32_t ldr, int32_t *r_out, double *y,
                      alm_stats *stats);
/* Gradient G = 2 S R of the augmented Lagrangian, S = C - A^*(y - sigma(A(RR^T) - b)),
 * for problems whose constraints are X_ii = b_i, one per row (the MaxCut SDP form),
 * computed from caller-owned device arrays WITHOUT ANY DEVICE ALLOCATION.  The paper
 * has no counterpart: this entry point serves callers that cannot call cudaMalloc (a
 * fixed memory budget reserved up front, an allocator that must not be re-entered, a
 * deployment that forbids allocation after start-up) and so cannot use alm_create.
 * It gives the same G as alm_grad on a handle of the same problem.
 *   precision     ALM_FP64 (arrays double) or ALM_FP32 (R, G, val, cdiag float).
 *   n             rows, 1..1048576 (the limit of the scratch array below; larger n is
 *                 rejected with ALM_ERR_INVALID_ARG).
 *   rowptr, col   device int32, the off-diagonal pattern of C in full symmetric CSR
 *                 (both (i,j) and (j,i)), n+1 and rowptr[n] entries; val its values C_ij.
 *   cdiag         device, C_ii (n).   b, y: device double (n).   sigma: penalty >= 0.
 *   R, G          device, n x ldr row-major, 16-byte aligned, ldr * element size a
 *                 multiple of 16; G gets zeros in columns r..ldr-1; G may not alias R.
 *   s             stream of the two kernel launches (asynchronous; nothing is synchronised).
 * Scratch: diag(S) lives in a file-scope device array of 1048576 doubles (8 MiB) that
 * every GPU which loads the library keeps until the process exits.  The first call on
 * each device looks up that array's device address (cudaGetSymbolAddress) with the
 * device current: make that first call before any stream capture.  Under CUDA's lazy
 * module loading (the default) that first call is also when the device allocates the
 * 8 MiB, so a caller with a fixed budget makes it once at start-up, before the budget
 * is fixed.  The address is cached per device index; after cudaDeviceReset it is stale,
 * so a process that resets a device must not call this entry point on it again.  In FP32
 * the off-diagonal sum is a plain FP32 accumulation (alm_grad compensates it), so the two
 * agree to FP32 rounding of |S||R|, not of |G|.  Every call writes the
 * entries it reads, so nothing carries over; but all calls share the one array, so calls
 * that overlap on the GPU (two streams, two host threads) race.  Errors: a status code,
 * and alm_last_error(NULL) gives the message. */
alm_status alm_grad_unitdiag_noalloc(int32_t precision, int64_t n, const int32_t *rowptr, const int32_t *col,
                                     const void *val, const void *cdiag, const double *b, const double *y,
                                     double sigma, const void *R, int32_t r, int32_t ldr, void *G,
                                     alm_stream_t s);

/* ------------------------------------------------------------------------------------
 * Batched solver: many small unit-diagonal SDPs in one persistent launch.
 *
 * Each instance b is  min <C_b, X_b>  s.t.  X_ii = 1 for every i,  X_b >= 0  (the MaxCut
 * SDP of Sec. 6.1 and any other C_b with the same constraints), solved by the same ALORA
 * iteration as alm_solve (Alg. 1: preconditioned CG inner solves with the exact quartic
 * step, Lanczos lambda_min, rank-one growth, y <- w, the relative KKT of Sec. 6) in the
 * FP32-bulk / FP64-scalar form.  One kernel launch processes the whole batch: every CTA
 * takes instances from a work counter, largest first, and solves each one alone.  The
 * launch (and the reset of the counter) is captured once as a CUDA graph and replayed.
 * The factor of instance b occupies rows row_off[b] .. row_off[b+1]-1 of one row-major
 * float matrix with a fixed row stride of 32 (ALM_BATCH_LDR) floats.
 * ------------------------------------------------------------------------------------ */
typedef struct alm_batch alm_batch;
enum { ALM_BATCH_LDR = 32 };
/* Problem data, host arrays copied by alm_batch_create. */
typedef struct {
    int32_t count;              /* instances, >= 1 */
    const int64_t *row_off;     /* count + 1, row_off[0] = 0: n_b = row_off[b+1] - row_off[b] >= 1 */
    const int64_t *nnz_off;     /* count + 1: instance b's entries are [nnz_off[b], nnz_off[b+1]) */
    const int32_t *c_i, *c_j;   /* upper-triangle COO of C_b with LOCAL indices 0 <= i <= j < n_b */
    const double *c_v;
} alm_batch_problem;
/* Per-instance result (alm_batch_solve fills one per instance). */
typedef struct {
    int32_t status;             /* ALM_OK, ALM_ERR_NOT_CONVERGED, ALM_ERR_NUMERIC or ALM_ERR_UNBOUNDED */
    int32_t outer, inner_total, rank;
    int32_t lanczos_matvecs, growth_steps;
    double kkt[3];              /* primal, dual, gap terms of the relative KKT error */
    double objective;           /* <C_b, X_b> at the end */
    double lambda_min;          /* last lambda_min(C_b - Diag(y_b)) estimate */
    double sigma;               /* final penalty */
    double device_ms;           /* time its CTA spent on it (GPU global timer) */
    int32_t fell_back;          /* 1 if it restarted from the cold start (fallback_inner) */
    int32_t reserved;
} alm_instance_stats;
/* Whole-batch statistics. */
typedef struct {
    int32_t status;             /* ALM_OK when every instance converged, else the first failing
                                   instance's status */
    int32_t converged;          /* instances with relative KKT <= eps */
    int32_t threads;            /* threads per CTA of the launch */
    int32_t ctas_per_sm, grid;  /* resident CTAs per SM and CTAs launched */
    int64_t kernel_launches;    /* kernels this library launched inside the call */
    int64_t inner_total, lanczos_matvecs;  /* sums over the instances */
    double device_ms;           /* CUDA-event time of the persistent launch */
    double time_ms;             /* host wall time of the call */
} alm_batch_stats;
/* Validate the batch (indices in range, i <= j, finite values, n_b >= 1), build
 * each instance's off-diagonal pattern in full symmetric CSR and the queue order, and
 * upload them.  Options: alm_options with precision ALM_FP32 (the only form of this
 * solver); chunk, use_graph, profile and verbose are ignored; o = NULL gives the
 * defaults with precision ALM_FP32 and lanczos_warm = 1.  s is the stream of every
 * later call.  On error *hb is NULL and alm_batch_last_error(NULL) gives the message. */
alm_status alm_batch_create(alm_batch **hb, const alm_batch_problem *p, const alm_options *o, alm_stream_t s);
void alm_batch_destroy(alm_batch *hb);
const char *alm_batch_last_error(const alm_batch *hb);
/* Solve every instance (instances of at most 16384 rows; larger ones are for alm_solve,
 * and a batch holding one is rejected here with ALM_ERR_INVALID_ARG).
 *   R     device float, (row_off[count]) x 32 row-major, 16-byte aligned: in, columns
 *         0..rank[b]-1 of instance b's rows hold its R0; out, its final factor, with zeros
 *         in columns rank[b]..31.
 *   rank  device int32, count: initial ranks in (clamped to 1..r_max), final ranks out.
 *   y     device double, row_off[count]: initial multipliers in, final multipliers out.
 *   stats host, may be NULL.   per_instance host, count entries, may be NULL.
 * Returns ALM_OK when every instance converged, else ALM_ERR_NOT_CONVERGED (or the
 * first instance error); the per-instance statuses say which. */
alm_status alm_batch_solve(alm_batch *hb, float *R, int32_t *rank, double *y, alm_batch_stats *stats,
                           alm_instance_stats *per_instance);
/* Choose the threads per CTA (256, 512 or 1024) of the persistent launch by timing
 * each candidate on a sample of the batch (about two instances per resident CTA, spread
 * over the size range, from the given R, rank, y, which are not modified; one outer
 * iteration each) and keep the fastest for later alm_batch_solve calls.  Without a call
 * the launch uses 512.  times_ms: host, may be NULL, 3 entries: the candidates' times. */
alm_status alm_batch_autotune(alm_batch *hb, const float *R, const int32_t *rank, const double *y,
                              int32_t *threads_out, double *times_ms);
/* Fix the threads per CTA of later alm_batch_solve calls (256, 512 or 1024). */
alm_status alm_batch_set_threads(alm_batch *hb, int32_t threads);
/* ------------------------------------------------------------------------------------
 * Learned warm start for the batched solver.
 *
 * A message-passing network on the pattern of C predicts (R0, y0) for every instance of
 * a batch (the paper has no network; its local convergence analysis of the BM subproblem
 * in Sec. 4.2 is why a starting point near a solution and a multiplier near y* pay off).
 * Per instance, with deg_i = off-diagonal entries of row i, s_i = sum_j C_ij,
 * dbar = max(mean deg, 1), cbar = mean |C_ij| (off-diagonal; 1 if none), sbar = mean |s_i|
 * (1 if 0):
 *   x_i  = [1, deg_i/dbar, s_i/sbar, log(n)/8, u_1(i), u_2(i), u_3(i), u_4(i)], u_k(i) the
 *          SplitMix64 uniform on [-1, 1) of stream feat_seed + k at the local row index i
 *   three layers  h'_i = relu(Ws h_i + Wn agg_i + b),  agg_i = sum_j (C_ij/cbar) h_j / max(deg_i, 1),
 *          width 8 -> 64 -> 64 -> 64
 *   heads  rhat_i = W_R h_i (32 columns),  yhat_i = w_y . h_i + b_y
 *   warm start  R0_i = rhat_i / |rhat_i|,  y0_i = cbar yhat_i
 * Training loss against solutions (R*, y*) of the same batch, X* = R* R*^T, P = the
 * diagonal and the strict upper pattern:
 *   L = sum_P (rhat_i . rhat_j - X*_ij)^2 / |P| + lam sum_i (yhat_i - y*_i / cbar)^2 / rows
 * Activations are stored in BF16 (ALM_GNN_BF16) or FP32 (ALM_GNN_FP32); all products
 * accumulate in FP32.  Parameters are one float vector (alm_gnn_num_params entries): per
 * layer Ws (64 x din), Wn (64 x din), b (64), then W_R (32 x 64), w_y (64), b_y.
 * Row-major matrices; din = 8 for the first layer.  The network runs on its own stream
 * s; every call below synchronises it before returning.
 * ------------------------------------------------------------------------------------ */
typedef struct alm_gnn alm_gnn;
enum { ALM_GNN_FP32 = 0, ALM_GNN_BF16 = 1 };
int32_t alm_gnn_num_params(void);
/* Weights start as U(-1, 1) sqrt(3 / fan_in) from the SplitMix64 stream init_seed (biases 0). */
alm_status alm_gnn_create(alm_gnn **g, int32_t storage, uint64_t feat_seed, uint64_t init_seed, alm_stream_t s);
void alm_gnn_destroy(alm_gnn *g);
const char *alm_gnn_last_error(const alm_gnn *g);
/* theta: host float vector (alm_gnn_num_params).  set_params also resets the Adam state. */
alm_status alm_gnn_set_params(alm_gnn *g, const float *theta);
alm_status alm_gnn_get_params(alm_gnn *g, float *theta);
/* The heads on every row of hb: rhat device float rows x 32, yhat device float rows (each may be NULL). */
alm_status alm_gnn_forward(alm_gnn *g, const alm_batch *hb, float *rhat, float *yhat);
/* Warm start for alm_batch_solve: R0_i = normalise(rhat_i/|rhat_i| + mix u_i/|u_i|), u_i a
 * uniform row from the SplitMix64 stream feat_seed ^ 0x3a1d (mix = 0: the network's rows
 * alone; mixing keeps R0 of full rank), y0 = cbar yhat.  R0 device float rows x 32
 * (16-byte aligned), rank device int32 count (set to min(32, r_max)), y0 device double rows.
 * Pair it with the option fallback_inner of the batch, so that an instance on which the
 * warm start does badly restarts from the cold start. */
alm_status alm_gnn_warm_start(alm_gnn *g, const alm_batch *hb, double mix, float *R0, int32_t *rank, double *y0);
/* Loss and gradient at the current parameters: Rstar device float rows x 32 (columns
 * beyond each instance's rank zero), ystar device double rows.  loss_out host (may be
 * NULL); grad_out host, alm_gnn_num_params floats (may be NULL). */
alm_status alm_gnn_loss_grad(alm_gnn *g, const alm_batch *hb, const float *Rstar, const double *ystar, double lam,
                             double *loss_out, float *grad_out);
/* `steps` full-batch Adam steps (Kingma and Ba; beta 0.9, 0.999, eps 1e-8, step size lr)
 * on the loss above.  loss_out: host, `steps` entries (the loss before each step), may be NULL. */
alm_status alm_gnn_train(alm_gnn *g, const alm_batch *hb, const float *Rstar, const double *ystar, double lam,
                         int32_t steps, double lr, double *loss_out);
/* Library build tag ("sm_103a ..."). */
const char *alm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ALM_H */
