/*
 * libsvt — GB300 (sm_103a) implementation of the data-parallel hot path of the Singular Value
 * Thresholding algorithm for matrix completion (Cai, Candes & Shen, "A Singular Value
 * Thresholding Algorithm for Matrix Completion", 2008).
 *
 * One SVT iteration (Sec. 2.2, eq. (2.7); Algorithm 1 of Sec. 5.1.5):
 *     X^k = D_tau(Y^{k-1})                      shrink: soft-threshold the singular values
 *     Y^k = Y^{k-1} + delta P_Omega(M - X^k)    dual step on the sampled set Omega only
 * D_tau(Y) = U diag((sigma_i - tau)_+) V^T (Sec. 2.1, eq. (2.2)) is evaluated by a
 * rank-adaptive block Lanczos partial SVD of the sparse iterate (Sec. 5.1.1), X^k is kept as
 * factors and evaluated on Omega only, and the dual step, the residual of eq. (5.5) and the
 * stop test are fused into one pass over Omega.
 *
 * Conventions for every entry point
 *   - Dimensions: m = number of rows (n1 in the paper), n = number of columns (n2); the paper
 *     writes m for |Omega|, called nnz here.
 *   - Matrices are row-major.  Index arrays are int32 and zero-based.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global memory of the
 *     current device.  The library copies every input it keeps; the caller keeps ownership of
 *     every buffer it passes.  Outputs are written to caller-allocated buffers.
 *   - Every call returns an svt_status.  No call aborts, exits or traps the GPU.  After an
 *     error, svt_last_error(ctx) returns a message (or svt_last_error(NULL) for calls that
 *     failed before a context existed).
 *   - Work is ordered after everything already queued on svt_options.stream (0 = legacy default
 *     stream) and everything queued there afterwards runs after the library's work; calls that
 *     return host data wait for their own work to finish.
 *   - A context is single-threaded.  Distinct contexts may be used concurrently from distinct
 *     threads on distinct streams.
 */
#ifndef SVT_H_
#define SVT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct svt_ctx svt_ctx;

typedef enum svt_status {
  SVT_OK = 0,
  SVT_ERR_ARG = 1,            /* invalid argument (size, pointer, option, index out of range) */
  SVT_ERR_DUP_INDEX = 2,      /* the same (row, col) pair appears twice in Omega */
  SVT_ERR_OOM = 3,            /* device or host allocation failed */
  SVT_ERR_CUDA = 4,           /* a CUDA runtime call failed (message has the CUDA error) */
  SVT_ERR_RANK_LIMIT = 5,     /* more than max_rank singular values exceed tau */
  SVT_ERR_NOT_CONVERGED = 6,  /* k_max iterations without meeting the stopping rule */
  SVT_ERR_NUMERIC = 7,        /* NaN/Inf or loss of positive definiteness in the Lanczos basis */
  SVT_ERR_TIMEOUT = 8,        /* a bounded device wait expired */
  SVT_ERR_INTERNAL = 9,       /* internal consistency check failed */
  SVT_STOPPED = 10            /* svt_step: the stopping rule eq. (5.5) holds at this iterate */
} svt_status;

/* Arithmetic of the per-nonzero work (Y, M values, the two sparse products, X on Omega and the
 * dual step).  The Lanczos basis, its reorthogonalisation and the projected SVD that fixes the
 * singular values compared against tau are float64 in every mode. */
enum { SVT_FP64 = 0, SVT_FP32 = 1, SVT_BF16 = 2 };
/* Shrink engines (svt_options.shrink_engine).  SVT_SHRINK_LANCZOS: the rank-adaptive block
 * Lanczos partial SVD (Sec. 5.1.1).  SVT_SHRINK_RANDOMIZED: the first alternative of Sec. 6, a
 * randomized range finder: with l = min(32, s_k + rsvd_oversample rounded up to a multiple of 8)
 * test columns Omega (the previous shrink's right singular vectors, then uniform(-1, 1) columns:
 * element (i, c) of the n x l block is (SplitMix64 output number i l + c + 1 at seed
 * rsvd_seed + 1000 k + pass) >> 11 times 2^-52, minus 1, k the SVT iteration and pass the rank
 * policy's pass counted from 0), Q = orth(Y Omega), rsvd_power steps Q <- orth(Y orth(Y^T Q)),
 * then D_tau(Q Q^T Y) from the SVD of Q^T Y; the rank policy of Sec. 5.1.1 sets s_k.  Exact when
 * l >= rank(Y); otherwise an approximation of D_tau(Y) (the paper leaves its accuracy open).
 * Needs min(m, n) >= 32 and s_k + rsvd_oversample <= 32 (else SVT_ERR_RANK_LIMIT). */
enum { SVT_SHRINK_LANCZOS = 0, SVT_SHRINK_RANDOMIZED = 1 };
/* SVT_BF16: float32 values and dual iterate as SVT_FP32, plus bfloat16 copies of Y (written by the
 * fused update) that the sparse products read, with float32 accumulation, while the relative
 * residual of eq. (5.5) is at or above svt_options.bf16_switch; once it falls below, the products
 * read the float32 values for the rest of the solve.  bfloat16 rounding of Y (8 significant bits)
 * perturbs the shrink by about 4e-3 |Y_ij| per entry, which stalls the residual well above 1e-4,
 * hence the switch.  The Dantzig-selector form runs in float32 throughout. */

typedef struct svt_options {
  int precision;          /* SVT_FP64 (default) or SVT_FP32 */
  int block;              /* lower bound on the Lanczos block size b (rounded up to a multiple of 8,
                             at most 32); 0 = automatic: wanted triplets + max(4, wanted / 4) */
  int ell;                /* rank increment l of Sec. 5.1.1 (default 5) */
  int k_max;              /* maximum SVT iterations after the kick (default 1000) */
  int lanczos_steps;      /* block steps J per Lanczos cycle (default 3; J b <= 128; raised where a thick restart
                             keeps several blocks of Ritz pairs, beyond 28 wanted triplets) */
  int max_cycles;         /* restarted Lanczos cycles per shrink before SVT_ERR_NUMERIC (default 40) */
  double lanczos_tol;     /* Ritz residual tolerance relative to sigma_1 (0 = 1e-6 FP64: agreement with a
                             float64 SVT with exact partial SVDs to ~1e-7 on the final X; 1e-4 FP32 and BF16,
                             where the float32 products' own rounding dominates) */
  int indices_on_device;  /* rows/cols/M_omega given to svt_create are device pointers */
  int use_graphs;         /* replay each Lanczos cycle as a captured CUDA graph (default 1) */
  uint64_t seed;          /* seed of the random start columns of the Lanczos blocks */
  void* stream;           /* cudaStream_t the caller orders work on; NULL = default stream.  The
                             library works on a stream of its own and joins it to this stream with
                             events at the start and end of every call. */
  int fused_orth;         /* 1 (default): each block orthonormalisation runs as one cooperative
                             kernel with grid barriers where the device supports cooperative
                             launches; 0: as a sequence of eight kernels (same arithmetic) */
  int restart_steps;      /* block steps J of a cycle that thick-restarts a non-converged one (block 0
                             = the leading Ritz pairs, block 1 = the residual block); 0 = same as
                             lanczos_steps */
  double bf16_switch;     /* SVT_BF16 only: relative residual below which the sparse products move
                             from the bfloat16 copies to the float32 values (default 1e-2) */
  int orth_grid;          /* upper bound on the CTAs of the cooperative orthonormalisation; 0
                             (default) = two per SM.  Contexts that run side by side on one GPU
                             (the serving runtime) cap it so that their cooperative kernels are
                             resident together.  The row chunks of the Gram sums follow the grid,
                             so results are reproducible for a given value (not across values). */
  double orth_repass;     /* orthonormality defect max |P^T P - I| of a block after its CGS2 + Cholesky QR pass
                             above which the cooperative orthonormalisation repeats the whole pass on the result
                             (Cholesky QR2; a block with nearly dependent columns loses orthogonality as
                             cond(P)^2 eps in one pass); 0 = default 1e-6, < 0 = never */
  /* Device allocator hook (both or neither; NULL = cudaMalloc / cudaFree): every device allocation
   * of the context goes through device_alloc(bytes, alloc_user), which returns a device pointer
   * aligned to 256 bytes or NULL when it cannot allocate (the call then fails with SVT_ERR_OOM and
   * releases what it holds); device_free(ptr, alloc_user) is called only after the context's work on
   * that memory has finished.  Lets a caller place the context in its own memory pool (a framework's
   * caching allocator). */
  void* (*device_alloc)(size_t bytes, void* alloc_user);
  void (*device_free)(void* ptr, void* alloc_user);
  void* alloc_user;
  int shrink_engine;      /* SVT_SHRINK_LANCZOS (default) or SVT_SHRINK_RANDOMIZED */
  int rsvd_oversample;    /* randomized engine: test columns beyond s_k (default 8, 1 .. 24) */
  int rsvd_power;         /* randomized engine: power steps (default 1, 0 .. 8) */
  uint64_t rsvd_seed;     /* randomized engine: base seed of the random test columns (default 0) */
  int device_loop;        /* 1 (default): each SVT iteration is one CUDA graph -- the shrink's Lanczos cycles
                             under a conditional `while` node whose condition a device kernel sets from the
                             convergence test and rank policy, then the Ritz vectors and the fused update,
                             the rank read on the device -- with one host synchronisation per iteration
                             (the host finishes an iteration whose rank policy grows s_k); 0: the host
                             decides after every Lanczos cycle.  Not used with profiling
                             (svt_set_profile), use_graphs = 0 or the randomized engine. */
  int orth_tf32;          /* coefficients of the first classical Gram-Schmidt pass of the cooperative
                             orthonormalisation (C1 = Q^T P) from split-TF32 tensor-core products (about
                             float32 accuracy); the projection, the second pass and a repeated pass are
                             float64, so the basis stays orthonormal to float64 rounding.  0 (default): on
                             for FP32 / BF16 values, off for FP64; 1: on; -1: off.  Needs orth_repass >= 0
                             (off otherwise) */
  int jacobi_cluster;     /* FP64 projected SVD: 0 (default) a thread-block cluster of 8 CTAs where the device
                             allows it (the dense products, right vectors and residual estimates spread over
                             the cluster), else one CTA; 1: always one CTA (the same arithmetic but for the
                             grouping of sums) */
} svt_options;

/* Per-iteration record (Algorithm 1, one pass of the for-loop body). */
typedef struct svt_step_info {
  int64_t k;              /* iteration index after the kick (1-based) */
  int r;                  /* r_k = #{sigma_j(Y^{k-1}) > tau} */
  int s;                  /* s_k: triplets computed in the final pass of the rank policy */
  int passes;             /* passes of the repeat-until loop of the rank policy */
  int lanczos_cycles;     /* restarted Lanczos cycles used by this shrink */
  int spmm_calls;         /* sparse products (Y V and Y^T U) issued by this shrink */
  double residual;        /* ||P_Omega(X^k - M)||_F / ||P_Omega M||_F  (eq. (5.5)) */
  double sigma1;          /* largest singular value of Y^{k-1} */
  double ms;              /* wall time of the step on the device (CUDA events), milliseconds */
} svt_step_info;

/* Per-solve record. */
typedef struct svt_result {
  int64_t iterations;     /* k at exit of Algorithm 1 (after the kick) */
  int64_t k0;             /* kick count of eq. (5.3) */
  int rank;               /* rank of X^opt */
  int converged;          /* 1 if the stopping rule eq. (5.5) was met */
  double residual;        /* final ||P_Omega(X - M)||_F / ||P_Omega M||_F */
  double norm2_M;         /* ||P_Omega M||_2 (Sec. 5.1.3) */
  double normF_M;         /* ||P_Omega M||_F */
  double ms;              /* wall time of the solve (kick + iterations), milliseconds */
  int64_t spmm_calls;     /* total sparse products */
  int64_t lanczos_cycles; /* total Lanczos cycles */
} svt_result;

/* Fills *opt with the defaults listed above. */
void svt_default_options(svt_options* opt);

/* Options of svt_batch_solve. */
typedef struct svt_batch_options {
  int spmm_grid;          /* CTAs of the persistent batched sparse-product launches (0: 16 per SM) */
  int update_grid;        /* CTAs of the persistent batched update launches (0: 8 per SM) */
  int autotune;           /* 1: the warps per segment of every batched sparse product (1, 2, 4 or 8) are
                             timed on the first product of each class (precision, block width,
                             direction, mean segment length rounded to a power of two) and the fastest
                             is kept for the process; 0 (default): the fixed rule of the solo path */
  int concurrent;         /* 1 (default): each job's own kernels (orthonormalisations, projected SVDs, Ritz
                             vectors) run on its library stream, the batched launches on a stream of the
                             batch, ordered by events, and each job's cooperative orthonormalisation gets
                             max(16, 2 SMs / n) CTAs so that the jobs' kernels overlap on the GPU; 0: all
                             work in issue order on the first job's stream with the solo launch shapes,
                             so that with autotune = 0 every iterate equals the job's solo iterate (shrink
                             decided on the host) */
} svt_batch_options;

/* Fills *opt with the batch defaults. */
void svt_batch_default_options(svt_batch_options* opt);

/*
 * Builds a context for one completion problem: stores Omega (Sec. 2.2: Y^k vanishes off Omega,
 * so only Omega is ever stored) in row-major (CSR) and column-major (CSC) order with the
 * permutation between them, and the sampled entries M_ij, (i,j) in Omega.
 *   m, n       matrix dimensions (n1, n2), 1 <= m, n < 2^31, m*n < 2^62
 *   nnz        |Omega|, 1 <= nnz < 2^31
 *   rows, cols nnz indices each, any order; host pointers, or device pointers when
 *              opt->indices_on_device
 *   M_omega    nnz sampled values (float64), same order as rows/cols, same memory space
 *   opt        may be NULL (defaults)
 *   out        receives the context; NULL on error
 * Errors: SVT_ERR_ARG (bad sizes, NULL pointers, an index outside [0,m) x [0,n)),
 * SVT_ERR_DUP_INDEX (a pair given twice), SVT_ERR_OOM, SVT_ERR_CUDA.
 */
svt_status svt_create(int64_t m, int64_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
                      const double* M_omega, const svt_options* opt, svt_ctx** out);

/*
 * Upper estimate of the device memory a context of this size takes (its persistent buffers, the
 * peak scratch of the structure build in svt_create, and a fixed allowance), for admission
 * control by memory.  Host-only: touches no device.  0 for invalid sizes.  A Dantzig-selector
 * context (svt_set_dantzig) needs 4 nnz value-bytes more.
 */
size_t svt_estimate_device_bytes(int64_t m, int64_t n, int64_t nnz, const svt_options* opt);

/* Releases all device and host memory of the context.  NULL is ignored. */
void svt_destroy(svt_ctx* ctx);

/* Message of the last error on ctx (or of the last failed svt_create when ctx is NULL). */
const char* svt_last_error(const svt_ctx* ctx);

/*
 * Sets the parameters of Algorithm 1 (Sec. 5.1.5) and applies the kicking device of Sec. 5.1.3:
 * computes ||P_Omega M||_2 by the Lanczos partial SVD, k0 = the integer with
 * tau / (delta ||P_Omega M||_2) in (k0 - 1, k0] (eq. (5.3)), and sets Y^0 = k0 delta P_Omega M,
 * r_0 = 0, k = 0.
 *   tau       threshold; <= 0 selects 5 sqrt(m n) (Sec. 5.2.1: tau = 5n for square matrices)
 *   delta     step size; <= 0 selects 1.2 m n / nnz (eq. (5.1))
 *   eps       tolerance of the stopping rule eq. (5.5); <= 0 selects 1e-4
 *   max_rank  capacity for the rank of X^k (1 .. 64); exceeding it returns SVT_ERR_RANK_LIMIT
 *   k0        >= 0 uses this kick count instead of eq. (5.3); -1 = eq. (5.3)
 * Errors: SVT_ERR_ARG, SVT_ERR_NUMERIC, SVT_ERR_CUDA.
 */
svt_status svt_configure(svt_ctx* ctx, double tau, double delta, double eps, int max_rank, int64_t k0);

/*
 * Stopping rule for noisy data (Sec. 5.2.1, noisy model eq. (5.9): B_ij = M_ij + Z_ij on Omega with
 * Z white Gaussian noise of standard deviation sigma; the values given to svt_create are B).
 * With sigma > 0, svt_step / svt_solve stop at the first X^k that is consistent with the data,
 *   ||P_Omega(X^k - B)||_F^2 <= (1 + eps_noise) nnz sigma^2          (eq. (5.10)),
 * instead of the relative-residual rule eq. (5.5); sigma <= 0 restores eq. (5.5).  eps_noise is
 * the paper's small parameter (it is not given a value there); it must be >= 0.  The rule stays in
 * force for later svt_configure / svt_solve calls on the context.
 * Errors: SVT_ERR_ARG (NULL ctx, eps_noise < 0 or not finite).
 */
svt_status svt_set_noise_stop(svt_ctx* ctx, double sigma, double eps_noise);

/*
 * Matrix Dantzig selector (Sec. 3.3, problem (DS) for matrix completion): minimise tau ||X||_* +
 * 1/2 ||X||_F^2 subject to |B_ij - X_ij| <= E on Omega (B = the values given to svt_create), by the
 * SVT iteration (iterDS2) with the multipliers Y_+, Y_- >= 0 of the two one-sided constraints:
 *   X^k = D_tau(Y_+^{k-1} - Y_-^{k-1}),
 *   Y_+^k = [Y_+^{k-1} + delta P_Omega((B - X^k) - E)]_+,  Y_-^k = [Y_-^{k-1} + delta P_Omega(-(B - X^k) - E)]_+.
 * E > 0 switches the context to this iteration (and allocates Y_+ and Y_-, ping-pong); E <= 0
 * returns to Algorithm 1.  Either way the context must be configured again (svt_configure or
 * svt_solve).  Readings where the paper is silent:
 *   kick: the first k steps from Y_+ = Y_- = 0 keep X^k = 0 and give Y_+ - Y_- = k delta soft_E(B)
 *         with soft_E(b) = sign(b) (|b| - E)_+; svt_configure therefore starts at
 *         k0 = ceil(tau / (delta ||P_Omega soft_E(B)||_2)) (eq. (5.3) on soft_E(B)),
 *         Y_+ = k0 delta [B - E]_+, Y_- = k0 delta [-B - E]_+;
 *   stop: the relative constraint violation ||[|B - X^k| - E]_+||_F / ||P_Omega B||_F <= eps
 *         (the analogue of eq. (5.5); svt_step_info.residual reports it).  The noisy-data rule of
 *         svt_set_noise_stop does not apply in this mode.
 * The float32 path keeps Y_+ and Y_- in float32.  svt_save_state / svt_load_state carry them.
 * Errors: SVT_ERR_ARG (NULL ctx, E not finite), SVT_ERR_OOM.
 */
svt_status svt_set_dantzig(svt_ctx* ctx, double E);

/*
 * One pass of the for-loop body of Algorithm 1: rank policy s_k = r_{k-1} + 1, then + l until a
 * computed singular value is <= tau (Sec. 5.1.1); X^k = sum_{j<=r_k} (sigma_j - tau) u_j v_j^T;
 * residual eq. (5.5); if residual <= eps returns SVT_STOPPED and leaves Y unchanged (the
 * break of Algorithm 1), else commits Y^k = Y^{k-1} + delta P_Omega(M - X^k) and returns SVT_OK.
 * info may be NULL.  Requires a prior svt_configure (or svt_solve).
 */
svt_status svt_step(svt_ctx* ctx, svt_step_info* info);

/*
 * Algorithm 1 in full: svt_configure(ctx, tau, delta, eps, max_rank, -1) followed by svt_step
 * until SVT_STOPPED or k_max iterations.  Returns SVT_OK when the stopping rule was met,
 * SVT_ERR_NOT_CONVERGED after k_max iterations (factors of the last iterate are kept), or the
 * first error of a step.  out may be NULL.
 */
svt_status svt_solve(svt_ctx* ctx, double tau, double delta, double eps, int max_rank, svt_result* out);

/*
 * Continuation (Sec. 6): the problem for a larger tau is started from the solution for the previous
 * tau.  svt_set_tau changes tau for the following svt_step calls and keeps the dual iterate Y, the
 * factors of X^k, the rank and the warm start; the iteration count restarts at 0.
 * Errors: SVT_ERR_ARG (NULL ctx, tau not positive and finite, context not configured).
 */
svt_status svt_set_tau(svt_ctx* ctx, double tau);

/*
 * Batched solve: Algorithm 1 (Sec. 5.1.5) for n independent completion problems at once (the paper
 * solves one problem at a time; this is the batched form of its iteration).  jobs: n distinct
 * contexts (1 <= n <= 32), all with the same value precision (FP64 or FP32; not BF16), the Lanczos
 * shrink engine, no noise stop and no Dantzig selector.  tau, delta: n values each, or NULL (a zero
 * or NULL entry takes the job's default, as in svt_configure); eps, max_rank: common to all jobs.
 * Each job is configured (kick of Sec. 5.1.3), then all unfinished jobs advance one SVT iteration
 * at a time in lockstep: the Lanczos cycles of their shrinks run together, and the sparse products
 * of all jobs at the same block step, and the fused updates of all jobs, are one persistent launch
 * each over the ragged job list.  Every job follows its own rank policy, thick restarts and stop
 * rule, and leaves the batch when it stops, fails or reaches its k_max.  Each job's stream is
 * synchronised on entry and on return (see svt_batch_options.concurrent for where the work runs).
 * Outputs: results[i] as
 * svt_solve's (ms = time from the batch's start to the end of the iteration in which job i left
 * it), status[i] the job's own status.  Returns SVT_OK when every job met the stopping rule, else
 * the first failing job's status (SVT_ERR_NOT_CONVERGED for k_max); SVT_ERR_ARG on a bad batch.
 * svt_get_factors and the other per-context calls work on each job afterwards.
 */
svt_status svt_batch_solve(svt_ctx* const* jobs, int n, const double* tau, const double* delta, double eps,
                           int max_rank, const svt_batch_options* opt, svt_result* results, svt_status* status);

/*
 * Continuation in full: svt_configure(ctx, taus[0], delta, eps, max_rank, -1) (the kick of eq. (5.3)
 * at taus[0]), then for i = 0 .. n_tau - 1: tau = taus[i] (svt_set_tau from the second stage on) and
 * svt_step until the stopping rule eq. (5.5) holds (at most k_max steps per stage).  Each stage
 * starts from the dual iterate at which the previous one stopped.  stage_iters (n_tau entries, may
 * be NULL) receives each stage's iterations; out (may be NULL) the totals, with iterations summed
 * over the stages.  Returns SVT_OK when the last stage met the stopping rule,
 * SVT_ERR_NOT_CONVERGED when a stage ran k_max steps, or the first error of a step.
 */
svt_status svt_solve_continuation(svt_ctx* ctx, const double* taus, int n_tau, double delta, double eps,
                                  int max_rank, int64_t* stage_iters, svt_result* out);

/* Rank r of the current X^k (0 before the first step). */
svt_status svt_get_rank(const svt_ctx* ctx, int* r);

/*
 * Copies X^k = U diag(d) V^T in factored form (X^opt of Algorithm 1 after svt_solve):
 *   U  host, m x capacity_r row-major (first r columns written), or NULL
 *   d  host, capacity_r values sigma_j - tau > 0 (first r written), or NULL
 *   V  host, n x capacity_r row-major (first r columns written), or NULL
 * Columns are the singular vectors of Y^{k-1} for its r largest singular values, in decreasing
 * order.  Errors: SVT_ERR_ARG if capacity_r < r.
 */
svt_status svt_get_factors(svt_ctx* ctx, double* U, double* d, double* V, int capacity_r);

/* Copies the current dual iterate Y on Omega, in row-major (sorted (row, col)) order, to the
 * host array y (nnz values). */
svt_status svt_get_Y(svt_ctx* ctx, double* y);

/* Replaces the current dual iterate by the host array y (nnz values in sorted row-major order).
 * Used to apply one shrink (svt_shrink) to a given sparse matrix supported on Omega. */
svt_status svt_set_Y(svt_ctx* ctx, const double* y);

/*
 * Copies the stored structure of Omega to host arrays (each may be NULL):
 *   row_ptr[m+1], col_idx[nnz]        row-major order, columns increasing within a row
 *   col_ptr[n+1], row_idx[nnz]        column-major order, rows increasing within a column
 *   csc_to_csr[nnz]                   row-major position of each column-major entry
 */
svt_status svt_get_structure(svt_ctx* ctx, int32_t* row_ptr, int32_t* col_idx, int32_t* col_ptr,
                             int32_t* row_idx, int32_t* csc_to_csr);

/*
 * X = D_tau(Y) of the current dual iterate (Sec. 2.1, eq. (2.2)) by the Lanczos partial SVD,
 * without a dual step: computes the factors of D_tau(Y), stores them as the current X, and
 * returns their rank in *r (may be NULL).  The singular values of Y larger than tau are written
 * to the host array sigma (capacity max_rank, may be NULL).  tau <= 0 uses the configured tau.
 */
svt_status svt_shrink(svt_ctx* ctx, double tau, int* r, double* sigma);

/*
 * Kernel-level entry points on the context's Omega (device pointers, row-major dense blocks
 * with b columns, 1 <= b <= 64):
 *   svt_apply_Y   W (m x b, float64) = Y V  for V (n x b, float64)   -- Y times a block
 *   svt_apply_Yt  Z (n x b, float64) = Y^T U for U (m x b, float64)  -- Y transpose times a block
 * Y is the current dual iterate; the arithmetic is that of the context's precision.  These are
 * the two products the Lanczos bidiagonalisation needs (Sec. 2.2 and Sec. 5.1.1).
 * Asynchronous: the kernel is queued on the context stream and the call returns; V/U and W/Z must
 * stay valid until the stream reaches it.  Pointers must be 16-byte aligned and b even.
 */
svt_status svt_apply_Y(svt_ctx* ctx, const double* V, int b, double* W);
svt_status svt_apply_Yt(svt_ctx* ctx, const double* U, int b, double* Z);

/*
 * Fused evaluation of X on Omega and the dual step (Algorithm 1, the residual test and the
 * update of Y; eq. (5.5)) for given device factors Ut (m x r, row-major; Ut = U diag(d)) and
 * V (n x r): for every (i,j) in Omega, x = sum_t Ut[i,t] V[j,t], e = M_ij - x,
 * y_out[p] = y_in[p] + delta e (row-major order p), and *res2 (host) = sum e^2.
 * y_in, y_out: device, nnz float64 each, row-major order (may alias).
 */
svt_status svt_sddmm_update(svt_ctx* ctx, const double* Ut, const double* V, int r, double delta,
                            const double* y_in, double* y_out, double* res2);

/*
 * Random-keys sampler of Omega on the device (Sec. 5.2.1: Omega uniform among all subsets of
 * cardinality nnz): the nnz linear ids i*n + j in [0, m n) with the smallest (key, id), where
 * key(id) is output number id + 1 of SplitMix64 (Steele, Lea & Flood 2014) started at state
 * `seed`.  Writes rows/cols (device, nnz int32 each) sorted by id, i.e. row-major.
 * Allocates its own scratch (O(nnz) device memory) and frees it before returning; synchronises
 * `stream` (cudaStream_t, NULL = default).  Errors: SVT_ERR_ARG, SVT_ERR_OOM, SVT_ERR_CUDA.
 */
svt_status svt_sample_omega(int64_t m, int64_t n, int64_t nnz, uint64_t seed, int32_t* rows, int32_t* cols,
                            void* stream);

/*
 * Snapshot of the solver state (k, r, parameters, Y on Omega, factors of X, warm-start block)
 * into a host buffer.  With buf == NULL, *bytes receives the size needed.  svt_load_state
 * restores a snapshot taken from a context with the same Omega and precision, so that the
 * following iterates are bit-identical to an uninterrupted run.
 */
svt_status svt_save_state(svt_ctx* ctx, void* buf, size_t* bytes);
svt_status svt_load_state(svt_ctx* ctx, const void* buf, size_t bytes);

/*
 * Failure injection for tests (the paper has no counterpart): the number of polls after which a
 * grid-barrier wait in the context's cooperative kernels gives up (0 restores the default 2^22, far
 * beyond any legitimate wait).  With a small value the barrier waits run out, the kernels return,
 * and the call that issued them returns SVT_ERR_TIMEOUT with the context still usable: the barrier
 * word is reset and the next shrink starts from a fresh block.  Synchronises the stream.
 * Errors: SVT_ERR_ARG (NULL ctx, spins < 0).
 */
svt_status svt_set_barrier_spins(svt_ctx* ctx, int spins);

/*
 * Self-test of the library's own float64 reciprocal and reciprocal-square-root helpers (Newton's
 * iteration from the float32 hardware approximations; the paper has no counterpart).  For the n
 * device values x (normal positive doubles) writes, to the device array out (5 n doubles, row i =
 * input i): 1/x with two and with one Newton step, 1/sqrt(x) with two and with one step, and the
 * Cholesky pivot's 1/sqrt(x) (exponent halved exactly, one step).  Synchronises `stream`.
 * Errors: SVT_ERR_ARG, SVT_ERR_CUDA (message in svt_last_error(NULL)).
 */
svt_status svt_selftest_math(int64_t n, const double* x, double* out, void* stream);

/* Device kernels launched by this library so far on ctx (for launch accounting). */
int64_t svt_kernel_launches(const svt_ctx* ctx);

/*
 * Kernel-class profile.  Classes (bit i of the mask = class i):
 *   SVT_PROF_SPMM (Y V), SVT_PROF_SPMM_T (Y^T U), SVT_PROF_GRAM (basis Gram products),
 *   SVT_PROF_BLOCK_UPDATE (P <- (P - Q C) R^-1), SVT_PROF_SMALL (b x b Cholesky steps),
 *   SVT_PROF_JACOBI (projected SVD), SVT_PROF_COMBINE (Ritz vectors), SVT_PROF_SDDMM (fused X on
 *   Omega + dual step), SVT_PROF_ORTH (a whole block orthonormalisation in one cooperative kernel,
 *   which replaces the GRAM / BLOCK_UPDATE / SMALL launches of that block where the device
 *   supports cooperative launches).
 * svt_set_profile selects the classes whose launches are bracketed by CUDA events on the context
 * stream (0 = none) and clears the totals.  svt_get_profile writes, per class, the number of
 * bracketed launch groups, their total device time in milliseconds, the algorithmic bytes they
 * move and the floating-point operations they perform (flops are counted for SPMM, SPMM_T, SDDMM
 * and ORTH, 0 for the other classes; arrays of SVT_PROF_CLASSES entries; any pointer may be NULL).
 * Both synchronise the stream.
 */
enum { SVT_PROF_SPMM = 0, SVT_PROF_SPMM_T, SVT_PROF_GRAM, SVT_PROF_BLOCK_UPDATE, SVT_PROF_SMALL, SVT_PROF_JACOBI,
       SVT_PROF_COMBINE, SVT_PROF_SDDMM, SVT_PROF_ORTH, SVT_PROF_CLASSES };
svt_status svt_set_profile(svt_ctx* ctx, unsigned int class_mask);
svt_status svt_get_profile(svt_ctx* ctx, int64_t* launches, double* ms, double* bytes, double* flops);

/*
 * Cumulative solver counters since svt_create, written to out[0 .. min(n, 11)):
 *   [0] Lanczos cycles, [1] sparse products, [2] projected-SVD calls, [3] Jacobi sweeps in them,
 *   [4] basis columns deflated as numerically dependent, [5] largest orthonormality defect
 *   max |P^T P - I| of an accepted Cholesky pass (before the first-order corrections, which reduce
 *   it to its square), [6] kernel launches, [7] shrinks whose Lanczos stagnated and were accepted
 *   at a relaxed tolerance (30x after 10 cycles, 300x after 25), [8] block orthonormalisations
 *   whose CGS2 + Cholesky QR pass was repeated (a defect above svt_options.orth_repass, or
 *   deflated columns replaced by fresh random directions), [9] largest defect of a first pass
 *   that was repeated for its defect, [10] SVT iterations run as one device-controlled graph
 *   (svt_options.device_loop).
 * Synchronises the stream.
 */
svt_status svt_get_counters(svt_ctx* ctx, double* out, int n);

/*
 * Allocation-free variant of svt_sddmm_update (the paper has no counterpart: this is a deployment
 * convenience).  Some callers cannot call cudaMalloc -- a process whose device memory is already
 * handed to its own pool (a framework's caching allocator, a server with a fixed memory budget)
 * or a latency-critical loop that cannot afford the implicit device synchronisation of
 * cudaMalloc/cudaFree.  This call allocates nothing and needs no context: the caller passes the
 * row-major storage of Omega and all inputs and outputs as device pointers, and the only scratch
 * (one partial sum per 64 rows plus the total) is a file-scope device array of 4096 doubles
 * (32 KB) that every GPU which loads libsvt holds until the process exits.
 *   m, n, nnz           dimensions; 1 <= m <= 262080 (larger m: SVT_ERR_ARG, the scratch holds at
 *                       most 4095 partial sums), n >= 1, 0 <= nnz < 2^31
 *   row_ptr, col_idx    row-major storage of Omega (m + 1 and nnz int32, columns increasing)
 *   M                   nnz sampled values (float64, row-major order)
 *   Ut, V               m x r and n x r float64 factors (Ut = U diag(d)), 0 <= r <= 64
 *   y_in, y_out         nnz float64 each, distinct buffers: y_out = y_in + delta (M - x)
 *   res2                host pointer: sum over Omega of (M - x)^2
 *   stream              cudaStream_t (NULL = default stream); the call synchronises this stream
 *                       (cudaStreamSynchronize) before it returns, to read res2
 * Arithmetic is float64, the kernel of svt_sddmm_update on a float64 context.
 * The first call on each device looks up the device address of the scratch array (once per
 * device, with that device current; again after cudaDeviceReset has replaced the device's
 * context, which the call detects from the current context's id); make that first call before
 * any stream capture.  Every call
 * on a device shares the array and the array keeps the last call's contents; each call writes
 * every entry it reads, so nothing needs clearing, but calls whose device work overlaps (for
 * instance on different streams) race on it.  Errors: SVT_ERR_ARG, SVT_ERR_CUDA, SVT_ERR_NUMERIC;
 * the message is in svt_noalloc_last_error().
 */
svt_status svt_sddmm_update_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                                    const double* M, const double* Ut, const double* V, int r, double delta,
                                    const double* y_in, double* y_out, double* res2, void* stream);
const char* svt_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SVT_H_ */
