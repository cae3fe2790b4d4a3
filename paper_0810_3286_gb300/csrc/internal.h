// Internal launch interface between the C-ABI layer (api.cu) and the kernels.
// Every launcher issues its kernels on `st` and returns the number of kernels launched; they
// never synchronise.  Pointers are device pointers unless the name says otherwise.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace svt {

// ----- generic ------------------------------------------------------------------------------
// out[0..n] = exclusive prefix sum of in[0..n-1], out[n] = total.  Needs scan_scratch_ints(n) ints.
long long scan_scratch_ints(long long n);
int launch_exclusive_scan(const int32_t* in, int32_t* out, long long n, int32_t* scratch, cudaStream_t st);

// ----- Omega storage (sorted segments) ----------------------------------------------------------
// Counts of `major` keys; flags out-of-range pairs (major >= n_major or minor >= n_minor).
int launch_count_major(const int32_t* major, const int32_t* minor, long long nnz, int n_major, int n_minor,
                       int32_t* counts, unsigned int* err, cudaStream_t st);
// Scatter (minor, payload) into segments of `ptr` (cursor must be zeroed).
int launch_scatter_segments(const int32_t* major, const int32_t* minor, const int32_t* payload, long long nnz,
                            int n_major, int n_minor, const int32_t* ptr, int32_t* cursor, int32_t* out_minor,
                            int32_t* out_payload, cudaStream_t st);
// Sort every segment [ptr[s], ptr[s+1]) with length <= seg_cap by minor key (carrying payload),
// in shared memory.  Longer segments are left for launch_sort_long_segment.
int segment_smem_capacity();
int launch_sort_segments(const int32_t* ptr, int n_seg, int32_t* minor, int32_t* payload, cudaStream_t st);
// Sort one long segment in global memory (scratch: 2 * pow2(len) ints).
int launch_sort_long_segment(int32_t* minor, int32_t* payload, int len, int32_t* scratch, cudaStream_t st);
// Longest segment length -> *out (device int).
int launch_max_segment(const int32_t* ptr, int n_seg, int32_t* out, cudaStream_t st);
// Flags adjacent equal minor keys inside a segment (duplicate pairs).
int launch_check_duplicates(const int32_t* ptr, int n_seg, const int32_t* minor, unsigned int* err, cudaStream_t st);
// major index of every position (expand ptr): out[p] = s for ptr[s] <= p < ptr[s+1].
int launch_expand_ptr(const int32_t* ptr, int n_seg, int32_t* out, cudaStream_t st);
// out[i] = in[perm[i]] for float64 input, written as double or float.
int launch_gather_f64(const double* in, const int32_t* perm, long long n, double* out, cudaStream_t st);
int launch_gather_f64_to_f32(const double* in, const int32_t* perm, long long n, float* out, cudaStream_t st);
// inv[perm[i]] = i
int launch_invert_perm(const int32_t* perm, long long n, int32_t* inv, cudaStream_t st);
// *out = sum of squares of x (float64, deterministic two-stage); partial needs 1024 doubles.
int launch_sumsq_f64(const double* x, long long n, double* partial, double* out, cudaStream_t st);

// ----- Omega sampler ---------------------------------------------------------------------------
struct SelectState;  // device-side radix-select state
long long omega_select_state_bytes();
int launch_omega_filter(uint64_t seed, long long N, uint64_t thresh, unsigned long long* cand_key,
                        unsigned long long* cand_id, long long cap, unsigned long long* count, cudaStream_t st);
int launch_omega_select(const unsigned long long* cand_key, const unsigned long long* cand_id,
                        const unsigned long long* count, long long rank, void* state, cudaStream_t st);
long long omega_compact_blocks(long long N);
int launch_omega_compact(uint64_t seed, long long N, long long n_cols, const void* state, int32_t* block_counts,
                         int32_t* block_offsets, int32_t* scan_scratch, int32_t* rows, int32_t* cols,
                         long long m, unsigned int* err, cudaStream_t st);

// ----- per-iteration kernels -------------------------------------------------------------------
// Out (n_out x b, float64) = S X with S given in compressed segments (ptr, idx, val) and X (n_in x b).
// precision 0: float64 values, X and accumulation; 1: float32 values and accumulation, X read from
// the float32 copy Xf when given (b a multiple of 4), else from the float64 X; 2: bfloat16 values,
// float32 copy Xf (required) and float32 accumulation.
// nnz (the total segment length) chooses how many warps share a segment.
int launch_spmm(int precision, const int32_t* ptr, const int32_t* idx, const void* val, const double* X,
                const float* Xf, double* Out, int n_out, int b, cudaStream_t st, long long nnz);

// Batched engine: one launch runs the sparse products (or the fused updates) of up to
// kBatchMaxJobs jobs of different shapes.  The job table travels as a kernel parameter.
static constexpr int kBatchMaxJobs = 32;

struct SpmmJob {                 // host description of one product Out = S X of a job list
  const int32_t* ptr;            // segment pointers (n_out + 1)
  const int32_t* idx;            // entry indices
  const void* val;               // entry values (float64, float32 or bfloat16 by the launch precision)
  const double* X;               // float64 block (precision 0)
  const float* Xf;               // float32 copy of the block (precisions 1 and 2)
  double* Out;                   // n_out x b
  int n_out, b;
  long long nnz;
  int wpr;                       // warps per segment; 0: the rule of launch_spmm
};
struct SpmmJobDev {
  const int32_t* ptr;
  const int32_t* idx;
  const void* val;
  const void* X;
  double* Out;
  int n_out, b, G, WPR, tile0;
};
struct SpmmJobTable {
  int n, tiles;
  SpmmJobDev job[kBatchMaxJobs];
};
// grid: CTAs of the persistent launch (0: 16 per SM).  Returns launches issued (0 on bad input).
int launch_spmm_jobs(int precision, const SpmmJob* jobs, int n, int grid, cudaStream_t st);

// Gram of a tall block against a basis: G ((nq+1) b x b) = [Q_0 .. Q_{nq-1}, P]^T P, where the Q_i
// are n x b blocks spaced `q_stride` doubles apart.  partial: gram_partial_doubles(...) doubles.
long long gram_partial_doubles(int n, int nq, int b);
// With Tcol given, the coefficient rows (the first nq b rows of G) are also written to Tcol
// (leading dimension ldT) as Gprev + G (Gprev may be NULL).
int launch_gram(const double* Q, long long q_stride, int nq, const double* P, int n, int b, double* partial,
                double* G, cudaStream_t st, const double* Gprev = nullptr, double* Tcol = nullptr, int ldT = 0);

// Block orthonormalisation steps (orth.cu).  C is the leading K x b part of a Gram result (K = nq b).
// Fused update + Gram (both kernels of a Gram: partial products and their fixed-order sum into G):
//   mode 0: P <- P - Q C, then G = [Q, P]^T P;  mode 1: P <- (P - Q C) R^-1, then G = P^T P.
int launch_update_gram(int mode, const double* Q, long long q_stride, int nq, const double* C, const double* R,
                       const double* dinv, double* P, int n, int b, double* partial, double* G, cudaStream_t st,
                       const double* Gprev = nullptr, double* Tcol = nullptr, int ldT = 0);
// R = chol(A) with deflation, A the trailing b x b block of G2; dinv = 1/diag(R) (0 if deflated);
// G1 (may be NULL when nq == 0) gives the column norms before the projections.
// counters[2] += deflated columns.
int launch_chol(const double* G1, const double* G2, int nq, int b, double* R, double* dinv,
                unsigned long long* counters, cudaStream_t st);
// P <- P (I - U(G3 - I)); (I + U(G3 - I)) R1 -> Tdiag (ld ldT) and/or Rout (b x b);
// counters[3] = max |G3 - I| (as float64 bits).  Pf (may be NULL): float32 copy of the new P.
int launch_correct(const double* G3, const double* R1, double* Tdiag, int ldT, double* Rout, double* P, int n, int b,
                   unsigned long long* counters, cudaStream_t st, float* Pf = nullptr);

// The whole orthonormalisation above (gram, update + gram, Cholesky, update + gram, correction,
// optionally the second correction) as one cooperative kernel with grid barriers.  bar: a zeroed
// 8-byte barrier word (device).  Tcol / Tdiag / Pf may be NULL.  repass > 0: when the defect
// max |P^T P - I| after the Cholesky pass exceeds it, the whole pass is repeated on its result and
// the coefficients are composed (counters[4] += 1, counters[5] = max first-pass defect).
// spin_limit: polls of a barrier wait before it gives up (SVT_DEVERR_BARRIER).  tc: the first
// pass's coefficients C1 = Q^T P from TF32 tensor-core products (mma.sync), the rest float64.  Uses at most
// min(orth_coop_init(), max_grid) CTAs and at most gram_partial_doubles(n, nq, b) partials.
// Returns 1 when launched, 0 when the device cannot run it (the caller then uses the sequence).
int orth_coop_init();
int launch_orth_coop(double* P, const double* Q, long long q_stride, int nq, int n, int b, double* partial,
                     double* G1, double* G2, double* G3, double* Tcol, double* Tdiag, int ldT, float* Pf,
                     unsigned long long* counters, unsigned int* err, void* bar, int twoc, int max_grid,
                     cudaStream_t st, double repass, unsigned int spin_limit, int tc);

// Jacobi SVD of the K x K matrix T (row-major, leading dimension ldT, block upper triangular with
// b x b blocks, K <= 128): T = Xl diag(theta) Wr^T, theta decreasing; Xl, Wr written K x K
// row-major (only the first nv columns of Wr are formed, the others are zero).  Also res[i] = || S (Xl rows [K-b, K), column i) ||
// for the b x b block S (upper triangular, may be NULL -> res = 0).
// counters[0] += 1, counters[1] += sweeps.
// cluster: CTAs of the launch (0: a cluster of 8 where the device allows it, 1: one CTA).
int launch_small_svd(const double* T, int ldT, int K, const double* S, int b, int nv, double* theta, double* Xl,
                     double* Wr, double* res, double tol, int max_sweeps, unsigned int* err,
                     unsigned long long* counters, cudaStream_t st, int cluster = 0);

// Self-tests of the Newton helpers (out: 5 doubles per input): slots 0..3 rcp (2 steps, 1 step),
// rsqrt (2 steps, 1 step) of jacobi.cu; slot 4 the pivot rsqrt of orth.cu.
int launch_newton_selftest(const double* x, long long n, double* out, cudaStream_t st);
int launch_pivot_selftest(const double* x, long long n, double* out, cudaStream_t st);

// ----- device-side control of the shrink (loop.cu) ---------------------------------------------
// Inputs of the convergence test, written by the host before each launch of the iteration graph.
struct LoopParams {
  double tau, tol;       // threshold; Ritz residual tolerance relative to theta_1
  int s, kmin;           // wanted triplets s_k; min(m, n)
  int max_cycles;        // Lanczos cycles of one pass of the rank policy
  int strict;            // every one of the s triplets must converge, s never grows (the kick)
};
enum { kLoopContinue = 0, kLoopConverged = 1, kLoopGrow = 2, kLoopBudget = 3, kLoopNumeric = 4 };
// Outcome, written by the device after every cycle.
struct LoopState {
  int status;            // kLoop*
  int cycles;            // cycles run in this pass
  int r;                 // rank #{theta_i > tau, i < s_eff} (on convergence)
  int s_eff;             // min(s, K)
  int conv;              // triplets that passed the test
  int relaxed;           // converged at a relaxed tolerance
  double res_fail;       // residual estimate / theta_1 of the first triplet that failed the test
};
// One thread: the convergence test of partial_svd on theta / res (K values), the rank and
// scale[i] = theta_i - tau on convergence, and (set_cond) the `while` condition: continue.
int launch_cycle_decide(const LoopParams* prm, LoopState* st, const double* theta, const double* res, int K,
                        double* scale, cudaGraphConditionalHandle cond, int set_cond, cudaStream_t s);

// Sets the dynamic shared-memory limits of the projected-SVD kernels (call before any stream
// capture); returns 0 on success.
int init_jacobi_attributes();

// Float32-rotation Jacobi with float64 Ritz values for the leading nvec triplets (jacobi.cu); two
// launches: the sweeps (one CTA), then the float64 refinement (nvec CTAs).  wsrc: nvec x K floats
// of scratch.
int launch_small_svd_mixed(const double* T, int ldT, int K, const double* S, int b, double* theta, double* Xl,
                           double* Wr, double* res, int nvec, float* wsrc, double tol, int max_sweeps,
                           unsigned int* err, unsigned long long* counters, cudaStream_t st);

// Out (n x s) = sum over blocks i of B_i (n x b) W[i b .. i b + b, 0 .. s) , columns scaled by
// scale[c] (or 1 when scale is NULL).  W: K x ldW row-major (K = nb * b).  OutF (may be NULL):
// float32 copy of Out with leading dimension ldF >= s.
// s_dev (may be NULL): the number of columns actually formed is min(*s_dev, s), read on the device (s
// is then an upper bound); ldo: row stride of Out (0 = s).
int launch_basis_combine(const double* B, long long b_stride, int nb, int b, int n, const double* W, int ldW, int s,
                         const double* scale, double* Out, cudaStream_t st, float* OutF = nullptr, int ldF = 0,
                         const int* s_dev = nullptr, int ldo = 0);

// T[i, i] = d[i] for i < b (row-major T, leading dimension ldT).
int launch_set_diagonal(double* T, int ldT, const double* d, int b, cudaStream_t st);

// Fill an n x b block with uniform(-1, 1) numbers from SplitMix64 (columns c >= c0 only).
int launch_random_block(double* P, int n, int b, int c0, uint64_t seed, cudaStream_t st);

// Fused X-on-Omega + dual step + residual (precision 0: float64 values, 1: float32 values):
//   x_p = sum_t Ut[i,t] V[j,t];  e = M_p - x_p;  y_out[p] = y_in[p] + delta e;
//   y_out_csc[csr_to_csc[p]] = y_out[p] (if y_out_csc);  res2 = sum e^2 (deterministic).
// Factors: float64 Ut (m x r) and V (n x r) with row stride ld64 (0 = r), or, for precision 1 when
// Utf and Vf32 are given, float32 copies with leading dimension ldf (a multiple of 4, >= r).
// r_dev (may be NULL): the rank is read on the device, r is then an upper bound.
// ys_out / ys_out_csc (both or neither; float32 values only): bfloat16 copies of y_out and of its
// column-major copy (y_out_csc required).
// dual (may be NULL): the two-multiplier form of the matrix Dantzig selector (iteration (iterDS2)):
//   yp_out = [yp_in + delta (e - E)]_+, ym_out = [ym_in + delta (-e - E)]_+, y_out = yp_out - ym_out,
//   res2 = sum [|e| - E]_+^2; y_in is unused.  Needs the float32 factor copies when precision is 1.
struct SddmmDual {
  const void* yp_in;
  const void* ym_in;
  void* yp_out;
  void* ym_out;
  double E;
};
int launch_sddmm_update(int precision, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* csr_to_csc,
                        const void* M, const void* y_in, void* y_out, void* y_out_csc, const double* Ut,
                        const double* V, const float* Utf, const float* Vf32, int ldf, int r, int n_rows,
                        double delta, double* partial, double* res2, unsigned int* err, cudaStream_t st,
                        const SddmmDual* dual = nullptr, void* ys_out = nullptr, void* ys_out_csc = nullptr,
                        const int* r_dev = nullptr, int ld64 = 0);
// bfloat16 copies (round to nearest) of the float32 values y (row-major) and y_csc.
int launch_to_bf16(const float* y, const float* y_csc, void* yb, void* yb_csc, long long nnz, cudaStream_t st);
// y = alpha soft_E(B) (plus the column-major copy), yp = alpha [B - E]_+, ym = alpha [-B - E]_+
// (any of y_csc, yp, ym may be NULL).
int launch_dual_kick(int precision, const void* B, double alpha, double E, void* y, void* y_csc, void* yp, void* ym,
                     const int32_t* csr_to_csc, long long nnz, cudaStream_t st);
int sddmm_partial_doubles();
// The same fused kernel (float64 values, no column-major copy) on `blocks` CTAs of 256 threads,
// one partial sum per CTA in `partial`, the fixed-order total in *res2 (device).
// Fused update of a job list (plain form: no Dantzig multipliers, no bfloat16 copies).  Per job:
// y_out = y_in + delta (M - x) in both orders and res2 = sum (M - x)^2, x = <Ut_i, V_j> on Omega.
struct UpdJob {
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const int32_t* csr_to_csc;
  const void* M;
  const void* y_in;
  void* y_out;
  void* y_out_csc;
  const void* Ut;                // factors: float64 (precision 0) or float32 rows padded to ldf
  const void* V;
  int r, ldf, m;
  double delta;
  double* res2;                  // device scalar
};
struct UpdJobDev {
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const int32_t* csr_to_csc;
  const void* M;
  const void* y_in;
  void* y_out;
  void* y_out_csc;
  const void* Ut;
  const void* V;
  double* res2;
  double delta;
  int r, ldf, m, tile0;
};
struct UpdJobTable {
  int n, tiles;
  UpdJobDev job[kBatchMaxJobs];
};
// partial: one double per tile of 64 rows over all jobs (upd_jobs_partial_doubles bounds it).
int launch_sddmm_update_jobs(int precision, const UpdJob* jobs, int n, double* partial, long long partial_cap,
                             unsigned int* err, int grid, cudaStream_t st);
long long upd_jobs_tiles(const int* m, int n);

int launch_sddmm_update_grid(const int32_t* row_ptr, const int32_t* col_idx, const double* M, const double* y_in,
                             double* y_out, const double* Ut, const double* V, int r, int n_rows, double delta,
                             int blocks, double* partial, double* res2, cudaStream_t st);

// y[p] = alpha * M[p] for the value type of `precision`; also writes the CSC copy via csr_to_csc.
int launch_scale_values(int precision, const void* M, double alpha, void* y, void* y_csc, const int32_t* csr_to_csc,
                        long long nnz, cudaStream_t st);
// Copy float64 values (row-major order) into the value type, plus CSC copy.
int launch_load_values(int precision, const double* src, void* y, void* y_csc, const int32_t* csr_to_csc,
                       long long nnz, cudaStream_t st);
// Store the value type (row-major order) as float64.
int launch_store_values(int precision, const void* y, double* dst, long long nnz, cudaStream_t st);

}  // namespace svt
