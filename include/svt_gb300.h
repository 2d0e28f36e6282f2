/*
 * svt_gb300.h -- C ABI of the GB300 (sm_103a) implementation of fast singular value
 * thresholding with the recycling rank-revealing randomized SVD (Li & Yu,
 * "A Fast Implementation of Singular Value Thresholding Algorithm using Recycling
 * Rank Revealing Randomized Singular Value Decomposition").
 *
 * Problem (eq. (1)-(3)): complete an m x n matrix A from the entries observed on the
 * index set Lambda.  The solver runs the Uzawa / linearized-Bregman iteration of
 * eq. (4), X = D_tau(Y), Y <- Y + delta P_Lambda(A - X), with the shrinkage operator
 * D_tau of eq. (5) evaluated through R4SVD (Algorithm 3; Algorithm 2 on the first
 * iteration) and the cooled precision threshold of Section 2.5 (Algorithm 4).
 *
 * Conventions shared by every entry point
 *  - Indices are 0-based int32; nnz < 2^31.  Lambda is a set: duplicate (row, col)
 *    pairs and out-of-range indices are errors.
 *  - Dense matrices are row-major: element (i, j) of an R x C matrix with leading
 *    dimension ld lives at p[i * ld + j], ld >= C.
 *  - Values observed on Lambda are kept in CSR order (sorted by row, then column);
 *    a vector "in CSR order" has one entry per observed position in that order.
 *  - Precision SVT_FP64 computes everything in binary64.  SVT_MIXED_FP32 keeps the
 *    observed values, Y and the tall-skinny blocks in binary32 and computes the
 *    Gram matrices, Cholesky factors, the small eigenproblem and all norms and
 *    threshold decisions in binary64 (or binary64-accurate arithmetic).
 *  - Work is queued on `stream` (a cudaStream_t; NULL is the legacy default stream).
 *    Every call returns after the work it queued has finished.
 *  - A call that fails returns a negative svt_status; svt_last_error() then gives a
 *    message for the calling thread.  No entry point terminates the process, and
 *    none leaves work running on the GPU when it returns.
 *  - Inputs and outputs are owned by the caller.  Device scratch memory of svt_complete,
 *    svt_complete_eval and svt_r4svd comes from a caller-owned workspace when one is
 *    passed (size from svt_workspace_size / svt_r4svd_workspace_size); with a NULL
 *    workspace, and in the other entry points, the library takes stream-ordered
 *    allocations from the device's default pool and returns them before the call ends.
 */
#ifndef SVT_GB300_H
#define SVT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum svt_status {
  SVT_OK = 0,              /* converged (residual < tol) or the call finished      */
  SVT_NOT_CONVERGED = 1,   /* maxit iterations done; the last iterate is returned   */
  SVT_ERR_ARG = -1,        /* invalid argument (sizes, parameters, capacities)      */
  SVT_ERR_INDEX = -2,      /* an observed index lies outside [0,m) x [0,n)          */
  SVT_ERR_DUPLICATE = -3,  /* an observed (row, col) pair occurs twice              */
  SVT_ERR_CUDA = -4,       /* a CUDA runtime call failed, or a bounded device wait  */
                           /* (tensor-core pipeline, grid barrier) ran out          */
  SVT_ERR_NUMERIC = -6,    /* non-finite input value, or a non-finite iterate       */
  SVT_ERR_UNSUPPORTED = -8 /* size beyond what this build supports                  */
} svt_status;

typedef enum svt_precision {
  SVT_FP64 = 0,
  SVT_MIXED_FP32 = 1
} svt_precision;

/* Which left singular vectors of D_tau's SVD seed the next R4SVD call (Section 2.3).
 * SVT_RECYCLE_ALL is the paper's method (Algorithm 3 with the r revealed vectors).
 * SVT_RECYCLE_KEPT recycles only the k vectors above tau.  SVT_RECYCLE_NONE starts every
 * call from Gaussian blocks (Algorithm 2); with t = r_max that is the fixed-rank
 * randomized SVD of Section 2.1 (one block of r_max columns, n_power power iterations). */
typedef enum svt_recycle {
  SVT_RECYCLE_ALL = 0,
  SVT_RECYCLE_KEPT = 1,
  SVT_RECYCLE_NONE = 2
} svt_recycle;

/* Stop rule of svt_complete: SVT_STOP_RESIDUAL ends when the relative residual
 * ||P_Lambda(A - X^(i))||_F / ||P_Lambda(A)||_F falls below tol (Algorithm 4);
 * SVT_STOP_MAE when the mean absolute error over the observed entries,
 * (1/|Lambda|) sum |A_ij - X^(i)_ij|, falls below tol (the rule of Section 3). */
typedef enum svt_stop {
  SVT_STOP_RESIDUAL = 0,
  SVT_STOP_MAE = 1
} svt_stop;

/* Solver options.  Defaults (svt_default_options) follow Section 3: t =
 * floor(0.05 min(m,n)), dt = 10, beta = 0.95; no power iterations. */
typedef struct svt_options {
  int32_t t;            /* width of the first Gaussian block; <= 0: floor(0.05 min(m,n)), at least 1 */
  int32_t dt;           /* width of each further block (Algorithms 2-3: Delta t)        */
  int32_t n_power;      /* power iterations X <- Y (Y^T X) per block (np)              */
  int32_t r_max;        /* rank cap; r <= min(m, n, r_max); <= 0: min(m, n)            */
  int32_t power_steps;  /* power steps for ||P_Lambda(A)||_2 in the initialisation     */
  int32_t precision;    /* svt_precision                                               */
  int32_t recycle;      /* svt_recycle (svt_complete)                                   */
  int32_t stop;         /* svt_stop (svt_complete)                                      */
  int32_t core_rows;    /* SVT_MIXED_FP32 only: rows of the dense core of the fused update
                           (the fullest rows, stored as a dense panel and updated on the
                           tensor cores); -1 automatic (rows with at least n/10 observed
                           entries, in whole tiles of 128), 0 none, > 0 that many rows    */
  int32_t reserved;     /* zero                                                          */
  double beta;          /* cooling factor for the precision threshold (0 < beta < 1)   */
  double eps_thr0;      /* initial error-percentage threshold                          */
  uint64_t seed;        /* key of the counter-based Gaussian generator                 */
  void* stream;         /* cudaStream_t                                                */
} svt_options;

/* Per-iteration record (the analogue of the paper's per-iteration timing plots). */
typedef struct svt_iter_log {
  int32_t iter;         /* SVT iteration i (1-based)                                   */
  int32_t r;            /* revealed rank of R4SVD                                      */
  int32_t k;            /* singular values above tau (rank of X^(i))                   */
  int32_t blocks;       /* Gaussian blocks drawn in this iteration                     */
  int32_t cooled;       /* 1 if the threshold was multiplied by beta after this step   */
  int32_t exhausted;    /* 1 if a block found the range of Y exhausted                 */
  double eps;           /* final error percentage of the QB decomposition              */
  double eps_thr;       /* threshold used in this iteration                            */
  double rel_residual;  /* ||P_Lambda(A - X^(i))||_F / ||P_Lambda(A)||_F               */
  double mae;           /* mean |A - X^(i)| over the observed entries                  */
  double sigma_max;     /* largest singular value of Y^(i)                             */
  double seconds;       /* wall time of the iteration (host clock, after its sync)     */
  double mae_eval;      /* mean |A - X^(i)| over the evaluation set of svt_complete_eval
                           (entries outside Lambda), NaN without one                    */
} svt_iter_log;

typedef struct svt_result {
  int32_t status;       /* svt_status of the call                                      */
  int32_t iters;        /* iterations run                                              */
  int32_t k;            /* rank of the returned X                                      */
  int32_t r;            /* last revealed rank                                          */
  int32_t k0;           /* kick-start multiple of the initialisation                   */
  int32_t log_len;      /* entries written to the log buffer                           */
  double rel_residual;  /* residual of the returned X                                  */
  double mae;
  double spec_norm;     /* ||P_Lambda(A)||_2 estimate used by the initialisation       */
  double eps_thr;       /* threshold at exit                                           */
  double seconds_pattern; /* time spent building the sorted pattern                    */
  double seconds_total;
} svt_result;

typedef struct svt_pattern svt_pattern;   /* opaque: the observed set on the device */

/* ------------------------------------------------------------------ utilities */
int svt_abi_version(void);
void svt_default_options(svt_options* opt);
const char* svt_status_string(int status);
/* Message describing the last failure on the calling thread (never NULL). */
const char* svt_last_error(void);

/* ------------------------------------------------------------------ pattern */
/* Build the observed set Lambda (P_Lambda of eq. (4)) from device COO arrays rows[nnz],
 * cols[nnz].  Sorts into CSR (row, col) and CSC (col, row) orders with a stable radix
 * sort; rejects out-of-range indices (SVT_ERR_INDEX) and duplicates
 * (SVT_ERR_DUPLICATE).  *out receives a handle owned by the caller. */
svt_status svt_pattern_create(int64_t m, int64_t n, int64_t nnz, const int32_t* rows,
                              const int32_t* cols, void* stream, svt_pattern** out);
void svt_pattern_destroy(svt_pattern* p);
int64_t svt_pattern_nnz(const svt_pattern* p);
/* Copy the sorted pattern into caller device buffers (any may be NULL):
 * row_ptr[m+1], col_idx[nnz] (CSR), csr_src[nnz] (input position of each CSR slot),
 * col_ptr[n+1], row_idx[nnz] (CSC), perm[nnz] (CSR slot of each CSC slot). */
svt_status svt_pattern_export(const svt_pattern* p, int32_t* row_ptr, int32_t* col_idx,
                              int32_t* csr_src, int32_t* col_ptr, int32_t* row_idx,
                              int32_t* perm, void* stream);

/* ------------------------------------------------------------------ building blocks */
/* Gaussian test block Omega (Algorithms 2-3): n x w standard normals, binary64,
 * row-major with leading dimension ld, device memory.  Entry (j, c) comes from
 * Philox4x32-10 (Salmon et al., SC'11) with counter (j, c/2, iter, block) and key
 * (seed low 32 bits, seed high 32 bits), turned into normals by Box-Muller. */
svt_status svt_gaussian_block(uint64_t seed, uint32_t iter, uint32_t block, int64_t n,
                              int32_t w, double* out, int64_t ld, void* stream);

/* Sparse times tall-skinny block with Y supported on Lambda (the matrix-block
 * products of Algorithms 1-3).  y_csr: values in CSR order (double for SVT_FP64,
 * float for SVT_MIXED_FP32).  transpose = 0: out (m x w) = Y W with W n x w;
 * transpose = 1: out (n x w) = Y^T W with W m x w.  W and out have the element type
 * of y_csr; all pointers are device pointers. */
svt_status svt_spmm(const svt_pattern* p, int precision, int transpose, const void* y_csr,
                    const void* W, int64_t ldw, int32_t w, void* out, int64_t ldo,
                    void* stream);

/* svt_spmm without any device allocation (the paper has no counterpart: this serves
 * callers, not the method).  Same arguments, results and errors as svt_spmm, but its
 * scratch memory comes from one fixed 32 MiB array inside this library instead of a fresh
 * allocation, for callers that cannot allocate device memory when they need the product:
 * a process whose other runtime has reserved nearly all GPU memory for its own pool, a
 * latency-critical loop where an allocation or free would stall the device, or an
 * application that only allows allocations at start-up.  A product whose scratch need
 * (partial rows of its entry chunks, plus a column-order copy of Y when transpose = 1)
 * exceeds the array returns SVT_ERR_UNSUPPORTED without queuing work.  Every GPU that
 * loads the library keeps the array until the process exits.  All calls share it and
 * its contents persist from call to call; nothing in it needs to start at zero, but
 * calls that overlap on the GPU race on it.  The first call on a device looks up the
 * array's address there and caches it for the process, so a device reset
 * (cudaDeviceReset) while the library is in use is not supported; make that first call
 * before any stream capture.
 * y_csr must hold the pattern's nnz values and W its n (transpose = 0) or m
 * (transpose = 1) rows: the library cannot check buffer sizes. */
svt_status svt_spmm_noalloc(const svt_pattern* p, int precision, int transpose,
                            const void* y_csr, const void* W, int64_t ldw, int32_t w, void* out,
                            int64_t ldo, void* stream);

/* One sampled shrinkage-and-update pass (eq. (4)-(5) restricted to Lambda): for each
 * observed (p, q) in CSR order, x = sum_{j<k} U[p, j] * W[q, j], d = a - x,
 * y += delta * d.  U (m x k, ldu) and W (n x k, ldw) hold X^(i) = U W^T.  sums[0..2]
 * (host memory) receive sum d^2, sum |d| and sum y_new^2 (binary64).  Element type
 * of a_csr, y_csr, U and W as in svt_spmm. */
svt_status svt_sampled_update(const svt_pattern* p, int precision, const void* U,
                              int64_t ldu, const void* W, int64_t ldw, int32_t k,
                              const void* a_csr, void* y_csr, double delta, double* sums,
                              void* stream);

/* The same pass in CSC order fused with the next iteration's recycled product: R4SVD
 * with recycling (Algorithm 3) starts from the basis U that defines X^(i), so
 * B^T = (Y^(i+1))^T U can be formed while the update gathers U's rows.  For each observed
 * (p, q) in CSC order: x = sum_{j<k} U[p, j] * W[q, j], d = a - x, y += delta * d; then
 * Bt[q, :r] = sum over column q of y_new * U[p, :r].
 *   U      m x r basis (ldu), device, 16-byte aligned, ldu a multiple of 4 (binary32) or
 *          2 (binary64) elements and at least r rounded up to that multiple;
 *   W      n x k (ldw), device, same alignment rule for k;
 *   a_csc, y_csc  observed values and Y in the pattern's CSC order (device, nnz each);
 *          y_csc is updated in place;
 *   Bt     n x r (ldb >= r), device, overwritten (rows of empty columns are zero);
 *   sums   host, as in svt_sampled_update.
 * 1 <= r <= 512 (binary32) or 256 (binary64) and 0 <= k <= r, else SVT_ERR_ARG;
 * misaligned U or W gives SVT_ERR_UNSUPPORTED.  Bt does not depend on scheduling. */
svt_status svt_sampled_update_recycle(const svt_pattern* p, int precision, const void* U,
                                      int64_t ldu, int32_t r, const void* W, int64_t ldw,
                                      int32_t k, const void* a_csc, void* y_csc, double delta,
                                      void* Bt, int64_t ldb, double* sums, void* stream);

/* ------------------------------------------------------------------ workspaces */
/* Device bytes that svt_complete / svt_complete_eval take from a caller workspace for a
 * solve of an m x n matrix with nnz observed entries, n_eval evaluation entries (0 for
 * svt_complete), output capacity cap and options opt (precision, rank cap, blocks,
 * core_rows matter).  The figure covers the device copies of host inputs whether or not
 * they will be needed, the sorted patterns and their sort scratch, the solver's arrays
 * with the largest dense core the automatic choice could pick (at most 4096 rows), and
 * the staging of host outputs; the solve itself uses at most this much.  0 for invalid
 * arguments.  The workspace is caller-owned device memory, at least 256-byte aligned. */
size_t svt_workspace_size(int64_t m, int64_t n, int64_t nnz, int64_t n_eval, int32_t cap,
                          const svt_options* opt);
/* Device bytes that svt_r4svd takes from a caller workspace (its work buffers). */
size_t svt_r4svd_workspace_size(int64_t m, int64_t n, int64_t nnz, const svt_options* opt);

/* ------------------------------------------------------------------ R4SVD */
/* One call of R4SVD (Algorithm 3; Algorithm 2 when s == 0) on Y given in CSR order
 * on the pattern.  U_prev: m x s recycled left singular vectors (ld_prev), may be NULL
 * when s == 0.  The basis grows by Gaussian blocks drawn as svt_gaussian_block(
 * opt->seed, iter, b, n, w) until the error percentage (||Y||_F^2 - ||B||_F^2) /
 * ||Y||_F^2 is at most eps_thr or the rank reaches min(m, n, r_max).
 * Outputs (device, element type of y_csr): U (m x r, ldu) = Q U_B, V (n x r, ldv) the
 * right singular vectors, S[r] (binary64, host or device) the singular values in
 * descending order.  Capacities ldu, ldv and S must hold min(m, n, r_max) columns.
 * *r_out, *eps_out and *blocks_out are host pointers.  workspace (device, ws_bytes) may be
 * NULL; otherwise the call allocates no device memory and takes its scratch from it, and
 * a workspace smaller than svt_r4svd_workspace_size(m, n, nnz, opt) returns SVT_ERR_ARG
 * before any work is queued.  The workspace must not be in use by other work meanwhile. */
svt_status svt_r4svd(const svt_pattern* p, const void* y_csr, const void* U_prev,
                     int64_t ld_prev, int32_t s, double eps_thr, uint32_t iter,
                     const svt_options* opt, void* U, int64_t ldu, double* S, void* V,
                     int64_t ldv, int32_t* r_out, double* eps_out, int32_t* blocks_out,
                     void* workspace, size_t ws_bytes);

/* ------------------------------------------------------------------ fast SVT */
/* Algorithm 4: complete the m x n matrix from nnz observed entries (rows, cols, vals).
 * rows/cols/vals may be host or device pointers (detected per pointer); vals is
 * double for SVT_FP64 and float for SVT_MIXED_FP32.  tau > 0 is the threshold of
 * eq. (3), delta > 0 the step of eq. (4); the iteration stops when the quantity of
 * opt->stop (by default the relative residual ||P_Lambda(A - X^(i))||_F /
 * ||P_Lambda(A)||_F) falls below tol, or after maxit iterations (SVT_NOT_CONVERGED).
 * Output X = U diag(S) V^T with U (m x cap), S[cap], V (n x cap), binary64, row-major,
 * host or device memory; the first res->k columns are valid.  cap must be at least
 * min(m, n, r_max).  log (host, may be NULL) receives up to log_cap iteration records.
 * res (host) is always written.  workspace (device, ws_bytes) may be NULL: the solve then
 * takes stream-ordered allocations.  Otherwise it allocates no device memory: every
 * device array of the solve (input copies, patterns, iterates, the dense core) is carved
 * from the workspace, and a workspace smaller than svt_workspace_size(m, n, nnz, 0, cap,
 * opt) returns SVT_ERR_ARG before any work is queued.  Small page-locked host buffers
 * for the solver's per-iteration reads are taken from a process-wide cache (allocated
 * the first time a solve needs one, then reused).  The workspace must not be in use by
 * other work meanwhile. */
svt_status svt_complete(int64_t m, int64_t n, int64_t nnz, const int32_t* rows,
                        const int32_t* cols, const void* vals, double tau, double delta,
                        double tol, int32_t maxit, const svt_options* opt, double* U,
                        double* S, double* V, int32_t cap, svt_result* res,
                        svt_iter_log* log, int32_t log_cap, void* workspace, size_t ws_bytes);

/* svt_complete with an evaluation set: n_eval entries (eval_rows, eval_cols, eval_vals;
 * host or device, element type of vals) that the solver never reads as data.  After each
 * iteration the mean absolute error of X^(i) on them goes to log[i].mae_eval: the
 * held-out ("testing set") MAE curve of Section 3.2.  The entries need not be disjoint
 * from Lambda, but must be distinct and in range (else SVT_ERR_DUPLICATE or
 * SVT_ERR_INDEX).  n_eval = 0 gives svt_complete.  The workspace as in svt_complete, sized
 * by svt_workspace_size(m, n, nnz, n_eval, cap, opt). */
svt_status svt_complete_eval(int64_t m, int64_t n, int64_t nnz, const int32_t* rows,
                             const int32_t* cols, const void* vals, int64_t n_eval,
                             const int32_t* eval_rows, const int32_t* eval_cols,
                             const void* eval_vals, double tau, double delta, double tol,
                             int32_t maxit, const svt_options* opt, double* U, double* S,
                             double* V, int32_t cap, svt_result* res, svt_iter_log* log,
                             int32_t log_cap, void* workspace, size_t ws_bytes);

/* ------------------------------------------------------------------ unrolled SVT */
typedef struct svt_unrolled_params {
  int32_t steps;             /* unrolled iterations T >= 1                                   */
  int32_t checkpoint_every;  /* forward state kept every this many iterations (default 5)   */
  int32_t cg_maxit;          /* step cap of each batched CG solve (default 1000)             */
  int32_t ritz_maxit;        /* cap on refinement steps per iteration (default 100); 0 turns
                                the refinement off and differentiates plain R4SVD output     */
  double cg_tol;             /* relative residual at which a CG column stops (default 1e-10
                                for SVT_FP64, 1e-6 for SVT_MIXED_FP32)                       */
  double ritz_tol;           /* refinement stops once ||Y v_i - s_i u_i|| <= ritz_tol * s_1
                                for every kept triplet (default 1e-11 for SVT_FP64, 2e-6 for
                                SVT_MIXED_FP32); the first dropped one needs only to be
                                placed below tau                                             */
} svt_unrolled_params;

typedef struct svt_unrolled_info {
  int32_t k0;            /* kick-start multiple of the initialisation (held fixed)        */
  int32_t k_final;       /* rank of X^(T)                                                 */
  int32_t r_final;       /* revealed rank of the last R4SVD                              */
  int32_t cg_iters;      /* conjugate-gradient steps over all adjoint solves             */
  int32_t cg_capped;     /* adjoint solves that stopped at cg_maxit before cg_tol        */
  int32_t ritz_steps;    /* refinement steps over the forward pass                       */
  int32_t ritz_capped;   /* forward iterations whose refinement stopped short of ritz_tol
                            (step cap, or residuals stalled at the rounding floor)        */
  int32_t ritz_grown;    /* blocks appended to certify a kept set (no dropped Ritz value) */
  double loss;
  double seconds_forward;
  double seconds_total;
} svt_unrolled_info;

/* Defaults above for the given precision (SVT_FP64 or SVT_MIXED_FP32); steps = 20. */
void svt_unrolled_default_params(svt_unrolled_params* p, int precision);

/* Unrolled SVT and its gradient (the paper differentiates nothing; this builds on its
 * iteration, eq. (4), with D_tau of eq. (5) evaluated by R4SVD, Algorithm 3).  Runs
 * T = p->steps iterations Y^(1) = k0 delta P_Lambda(A), X^(i) = D_tau(Y^(i)),
 * Y^(i+1) = Y^(i) + delta P_Lambda(A - X^(i)) with no stop test (k0 as in svt_complete,
 * then held fixed), evaluates L = mean over the nheld held-out entries of
 * (X^(T) - A)^2, and returns dL/dvals (grad_vals[nnz], caller order),
 * out3 = {L, dL/dtau, dL/ddelta} and X^(T) on the held-out entries (x_held[nheld]).
 *
 * Forward.  Each R4SVD result is refined by power steps Q <- orth(Y Y^T Q) on its whole
 * basis (the power scheme of Algorithms 1-3), each followed by a Rayleigh-Ritz step,
 * until the kept triplets meet the residual bound ritz_tol and the first dropped one is
 * placed below tau (or the residuals stop falling: the rounding floor);
 * D_tau is then that of Y to this bound and the gradient is that of exact unrolled SVT.
 * While every Ritz value exceeds tau the basis grows by Gaussian blocks of opt->dt
 * columns, as in R4SVD; at the rank cap the kept set cannot be certified and the call
 * fails with SVT_ERR_UNSUPPORTED (raise opt->r_max).  The refined basis is what the next
 * iteration recycles.
 *
 * Reverse.  The forward state (Y, the recycled basis, the cooled threshold) is kept every
 * checkpoint_every iterations and each segment is replayed from it.  The adjoint of D_tau
 * (its Jacobian is symmetric) is a closed form on the kept block and, for the coupling
 * with the rest of the spectrum, shifted systems (s_i^2 - Y_perp^T Y_perp) w_i = b_i
 * solved by batched conjugate gradients with sparse products of Y only.
 *
 * Index and value arrays may be host or device memory (values double for SVT_FP64, float
 * for SVT_MIXED_FP32); outputs are binary64, host or device.  grad_vals NULL skips the
 * reverse pass (out3 = {L, NaN, NaN}).  p NULL means the defaults;
 * info (host) may be NULL.  Errors: SVT_ERR_ARG (sizes, tau/delta <= 0, bad parameters),
 * the pattern errors of svt_pattern_create for either index set, SVT_ERR_NUMERIC
 * (non-finite iterate or CG residual, basis breakdown), SVT_ERR_UNSUPPORTED (see above
 * and svt_complete's rank cap), SVT_ERR_CUDA. */
/* The same computation split for reverse-mode automatic differentiation.  The forward
 * pass runs the T iterations, writes X^(T) on the held-out entries (x_held[nheld],
 * binary64, caller order, host or device) and, when tape is not NULL, returns in *tape the
 * state the reverse pass replays: the checkpoints every checkpoint_every iterations, the
 * patterns and the last iterate, all in device memory owned by the tape (about
 * (T / checkpoint_every + 3 checkpoint_every) copies of Y and of the basis).  With tape
 * NULL only the forward runs and nothing is kept.  Arguments and errors as in
 * svt_unrolled_grad; held-out values are not needed (the loss is the caller's). */
typedef struct svt_unrolled_tape svt_unrolled_tape;
svt_status svt_unrolled_forward(int64_t m, int64_t n, int64_t nnz, const int32_t* rows,
                                const int32_t* cols, const void* vals, int64_t nheld,
                                const int32_t* held_rows, const int32_t* held_cols, double tau,
                                double delta, const svt_unrolled_params* p,
                                const svt_options* opt, double* x_held, svt_unrolled_info* info,
                                svt_unrolled_tape** tape);
/* Reverse pass: given g_held[nheld] = dL/dX^(T) on the held-out entries (binary64, caller
 * order, host or device), writes grad_vals[nnz] = dL/dvals (caller order, binary64, host
 * or device, may be NULL) and grad_tau_delta[2] = {dL/dtau, dL/ddelta} (host or device, may
 * be NULL).  Runs on the stream of the forward call; a tape serves one backward call
 * (SVT_ERR_ARG on a second). */
svt_status svt_unrolled_backward(svt_unrolled_tape* tape, const double* g_held, double* grad_vals,
                                 double* grad_tau_delta, svt_unrolled_info* info);
/* Releases the tape's device memory (after waiting for its stream). */
void svt_unrolled_tape_destroy(svt_unrolled_tape* tape);

svt_status svt_unrolled_grad(int64_t m, int64_t n, int64_t nnz, const int32_t* rows,
                             const int32_t* cols, const void* vals, int64_t nheld,
                             const int32_t* held_rows, const int32_t* held_cols,
                             const void* held_vals, double tau, double delta,
                             const svt_unrolled_params* p, const svt_options* opt,
                             double* grad_vals, double* x_held, double* out3,
                             svt_unrolled_info* info);

/* ------------------------------------------------------------------ profiling */
/* Per-kernel-class timing (no counterpart in the paper; the analogue of its
 * per-iteration timing figures).  When enabled, the solver brackets each kernel class
 * with CUDA events on the launching stream and adds the algorithmic bytes the class
 * must move.  svt_profile_read copies up to cap entries: names (cap x 32 chars,
 * NUL-padded), launch counts, total milliseconds and total algorithmic bytes; it
 * returns the number of entries.  All pointers are host pointers, any may be NULL. */
void svt_profile_enable(int on);
void svt_profile_reset(void);
int svt_profile_read(int cap, char* names, int64_t* launches, double* ms, double* bytes);
/* Number of CUDA kernels this library has launched in the process so far. */
int64_t svt_launch_count(void);

/* ------------------------------------------------------------------ testing hook */
/* Failure detection (no counterpart in the paper).  The cooperative-grid Jacobi used for
 * revealed ranks above what one CTA's shared memory holds waits at a grid barrier after
 * every rotating step; each wait gives up after a bounded number of polls (2^24 by
 * default, about a second), sets a status flag and ends the kernel, and the solver then
 * returns SVT_ERR_CUDA with a message naming the grid Jacobi.  This call sets that bound
 * for later launches in the process (values below 1 count as 1) and returns the previous
 * one, so that a test can make a wait run out and check that the error is reported and
 * the device stays usable.  Not thread-safe with respect to solves running meanwhile. */
unsigned svt_test_set_grid_wait_limit(unsigned polls);

#ifdef __cplusplus
}
#endif

#endif /* SVT_GB300_H */
