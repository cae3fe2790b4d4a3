// C-ABI of libsvt: context, Omega storage build, the rank-adaptive block Lanczos shrink and the
// loop of Algorithm 1 (Sec. 5.1.5).  Host code here only orchestrates: every arithmetic step on
// the matrices runs in the kernels of omega.cu, sparse.cu and dense.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/svt.h"
#include "common.cuh"
#include "internal.h"

using namespace svt;

namespace {

constexpr int kBMax = 32;       // largest Lanczos block
constexpr int kKMax = 128;      // largest projected problem (J b)
constexpr int kGramW = 160;     // widest Gram [Q_0 .. Q_{nq-1}, P] of the orthonormalisation: (nq + 1) b
constexpr int kMaxRankCap = 64; // rank capacity of X^k
// Default Ritz residual tolerances (relative to sigma_1).  Float64 path: its iterates then agree
// with a float64 SVT with exact partial SVDs to ~1e-7 on the final X (the per-iterate bound is
// 1e-5), with ~35 % fewer Lanczos cycles than at 1e-8.  Float32 and bfloat16 values: the products'
// own rounding (~1e-6 of sigma_1) dominates the iterates' error; tightening below 1e-4 changes the
// final X by less than that.
static constexpr double kLanczosTolF64 = 1e-6;
static constexpr double kLanczosTolF32 = 1e-4;
constexpr int kOversample = 4;  // block columns beyond the wanted triplets
constexpr uint64_t kStateMagic = 0x5356545354415445ULL;  // "SVTSTATE"

thread_local std::string g_create_error;

// NVTX range over one host-side phase (visible in Nsight Systems; free when no tool is attached).
// Device phases inside a replayed Lanczos-cycle graph are covered by the enclosing host range.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace

struct svt_ctx {
  int device = 0;
  cudaStream_t st = nullptr;        // the library's own non-blocking stream (capturable)
  cudaStream_t user_st = nullptr;   // the caller's stream (joined at every call)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  struct ProfNode { int cls; double bytes, flops; cudaEvent_t a, b; };
  struct CycleGraph {
    int b, J, ycur, twoc, thick, Jprev, bf16, nk;
    unsigned int prof_mask;
    cudaGraphExec_t exec;
    int64_t launches;
    std::vector<ProfNode> prof;   // event pairs recorded by the graph's own event-record nodes
  };
  std::vector<CycleGraph> graphs;
  // one SVT iteration as one graph: Lanczos cycles under a `while` node driven by the device-side
  // convergence test, then the Ritz vectors and the fused update (svt_options.device_loop)
  struct IterGraph {
    int b, J, nk, ycur, twoc, bf16;
    double delta, dsE;
    cudaGraphExec_t exec;
    int64_t l_pre, l_body, l_post;
  };
  std::vector<IterGraph> igraphs;
  LoopParams* dl_prm = nullptr;     // device: inputs of the convergence test
  LoopState* dl_st = nullptr;       // device: its outcome
  char* dl_pin = nullptr;           // pinned: params staging, state, res2, err word, defect, theta
  bool dl_broken = false;           // the iteration graph could not be built: host loop from then on
  std::string dl_reason;
  int64_t dl_iters = 0;             // iterations run by the iteration graph
  svt_options opt{};
  int64_t m = 0, n = 0, nnz = 0;
  int prec = SVT_FP64;
  size_t vbytes = 8;
  // bfloat16 ladder (precision SVT_BF16, float32 values otherwise): bfloat16 copies of Y (row- and
  // column-major, ping-pong) feed the sparse products while bf16_active
  bool bf16_mode = false, bf16_active = false;
  void* Yb[2] = {nullptr, nullptr};
  void* Ybc[2] = {nullptr, nullptr};
  std::string last_error;
  std::vector<void*> allocations;


  // Omega
  int32_t *row_ptr = nullptr, *col_idx = nullptr, *col_ptr = nullptr, *row_idx = nullptr;
  int32_t *csc_to_csr = nullptr, *csr_to_csc = nullptr;
  void* Mv = nullptr;               // sampled entries, row-major order, value type
  void* Ycsr[2] = {nullptr, nullptr};
  void* Ycsc[2] = {nullptr, nullptr};
  int ycur = 0;
  double normF = 0.0;

  // parameters / state of Algorithm 1
  bool configured = false;
  double tau = 0, delta = 0, eps = 1e-4;
  double noise_sigma = 0.0, noise_eps = 0.0;   // > 0: the noisy-data stopping rule eq. (5.10)
  double ds_E = 0.0;                // > 0: matrix Dantzig selector (iterDS2) with tolerance E
  void* Yp[2] = {nullptr, nullptr}; // its multipliers Y_+ and Y_- (ping-pong, row-major order)
  void* Ym[2] = {nullptr, nullptr};
  int max_rank = 0;
  int64_t k0 = 0, k = 0;
  double norm2 = 0.0;
  int r = 0;                        // rank of X^k
  std::vector<double> d_host;       // sigma - tau of X^k
  double* Ut = nullptr;             // m x kMaxRankCap+1: U diag(sigma - tau)
  double* Uf = nullptr;             // m x cap: U (unscaled)
  double* Vf = nullptr;             // n x cap: V
  double* Vwarm = nullptr;          // n x kKMax: warm start block; right Ritz vectors kept by a thick restart
  double* Uwarm = nullptr;          // m x kKMax: left Ritz vectors kept by a thick restart
  // float32 path only: float32 copies of the dense operands of the per-entry kernels (the sparse
  // products read the current basis block, the fused update the factors), written by the kernels
  // that produce the float64 originals
  float* Ush = nullptr;             // m x kBMax: current U block
  float* Vsh = nullptr;             // n x kBMax: current V block
  float* Utf = nullptr;             // m x ldf: U diag(sigma - tau)
  float* Vff = nullptr;             // n x ldf: V
  int ldf = 0;                      // row length of Utf / Vff: a multiple of 4 >= r
  int ldu = 0;                      // row length of Ut / Uf / Vf: r (host path) or the graph's bound on r
  int warm_cols = 0;
  uint64_t rng_counter = 0;

  // Lanczos workspace
  double *Ub = nullptr, *Vb = nullptr;   // block bases (blocks of rows x b)
  double *T = nullptr, *S = nullptr, *theta = nullptr, *Xl = nullptr, *Wr = nullptr, *res = nullptr;
  float* wsrc = nullptr;   // float32 leading Ritz vectors of the projected SVD (kKMax x kKMax)
  double *G1 = nullptr, *G2 = nullptr, *G3 = nullptr, *gpart = nullptr, *R1 = nullptr, *dinv = nullptr;
  double *Rkeep = nullptr, *scale = nullptr;
  bool two_corrections = false;           // set once an orthonormality defect above 1e-6 was seen
  double orth_repass = 1e-6;              // defect above which a block's orthonormalisation pass is repeated
  int orth_tc = 0;                        // first CGS pass's coefficients from split-TF32 tensor-core products
  unsigned int barrier_spins = kBarrierSpinLimit;
  int coop_grid = 0;                      // > 0: orthonormalise each block in one cooperative kernel
  void* gbar = nullptr;                   // its grid barrier (8 bytes, zeroed)
  double* R2 = nullptr;                   // b x b product of the first correction and R1
  unsigned long long* dcount = nullptr;   // device counters: [0] Jacobi calls [1] Jacobi sweeps
                                          // [2] deflated columns [3] max orthonormality defect (bits)
  double *upd_partial = nullptr, *dscal = nullptr;
  unsigned int* err = nullptr;
  double* h_pin = nullptr;          // pinned host staging (theta, res, scalars)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  // per-kernel-class profile (CUDA events around launches of the classes in prof_mask)
  unsigned int prof_mask = 0;
  std::vector<cudaEvent_t> prof_pool;
  struct ProfRec { int cls; double bytes, flops; cudaEvent_t a, b; bool graph_owned; };
  std::vector<ProfRec> prof_pending;
  double prof_ms[SVT_PROF_CLASSES] = {0};
  double prof_bytes[SVT_PROF_CLASSES] = {0};
  double prof_flops[SVT_PROF_CLASSES] = {0};
  int64_t prof_n[SVT_PROF_CLASSES] = {0};

  // statistics of the last shrink
  int last_cycles = 0, last_spmm = 0, last_s = 0, last_passes = 0;
  double last_sigma1 = 0.0;
  int64_t launches = 0;
  int64_t total_spmm = 0, total_cycles = 0;
  int64_t relaxed_shrinks = 0;      // shrinks accepted at a relaxed Lanczos tolerance (stagnation)
};

// ------------------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------------------
static svt_status fail(svt_ctx* c, svt_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->last_error = buf;
  else g_create_error = buf;
  return s;
}

#define CU(ctx, call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      (void)cudaGetLastError();                                                                \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? SVT_ERR_OOM : SVT_ERR_CUDA,         \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    }                                                                                          \
  } while (0)

#define TRY(expr)                     \
  do {                                \
    svt_status s_ = (expr);           \
    if (s_ != SVT_OK) return s_;      \
  } while (0)

// Device memory of a context: through the caller's allocator hook (svt_options.device_alloc /
// device_free) when one is given, else cudaMalloc / cudaFree.  Memory is released only after the
// context stream has drained.
static void* dev_malloc(svt_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (c->opt.device_alloc) return c->opt.device_alloc(bytes, c->opt.alloc_user);
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return p;
}

static void dev_free(svt_ctx* c, void* p) {
  if (!p) return;
  if (c->opt.device_free) c->opt.device_free(p, c->opt.alloc_user);
  else cudaFree(p);
}

// Frees one allocation that dalloc recorded in the context (so that svt_destroy does not free it
// again).
static void dfree(svt_ctx* c, void* p) {
  if (!p) return;
  auto it = std::find(c->allocations.begin(), c->allocations.end(), p);
  if (it != c->allocations.end()) c->allocations.erase(it);
  dev_free(c, p);
}

static svt_status dalloc(svt_ctx* c, void** p, size_t bytes) {
  *p = dev_malloc(c, bytes);
  if (!*p) return fail(c, SVT_ERR_OOM, "device allocation of %zu bytes failed", bytes);
  c->allocations.push_back(*p);
  return SVT_OK;
}

// Releases the most recent allocation of dalloc (call-local temporaries) after the stream drained.
static void dfree_last(svt_ctx* c) {
  if (c->allocations.empty()) return;
  void* p = c->allocations.back();
  c->allocations.pop_back();
  dev_free(c, p);
}

namespace {
// Temporary device buffers of one call, freed (after the stream drains) when the call returns.
struct TmpBufs {
  svt_ctx* c;
  std::vector<void*> ptrs;
  explicit TmpBufs(svt_ctx* cc) : c(cc) {}
  ~TmpBufs() {
    if (ptrs.empty()) return;
    cudaStreamSynchronize(c->st);
    for (void* p : ptrs) dev_free(c, p);
  }
  template <typename T>
  bool get(T** p, size_t count) {
    void* v = dev_malloc(c, count * sizeof(T));
    *p = (T*)v;
    if (!v) return false;
    ptrs.push_back(v);
    return true;
  }
};
}  // namespace

template <typename T>
static svt_status dalloc_t(svt_ctx* c, T** p, size_t count) {
  void* v = nullptr;
  svt_status s = dalloc(c, &v, count * sizeof(T));
  *p = (T*)v;
  return s;
}

// Launch accounting + launch-error check.
static svt_status launched(svt_ctx* c, int n) {
  c->launches += n;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, SVT_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
  return SVT_OK;
}

static cudaEvent_t prof_event(svt_ctx* c) {
  if (!c->prof_pool.empty()) {
    cudaEvent_t e = c->prof_pool.back();
    c->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { (void)cudaGetLastError(); return nullptr; }
  return e;
}

// Runs `f` (which issues the launches of one kernel class and returns their count); when the
// class is selected by the profile mask, brackets the launches with CUDA events on the context
// stream and records the algorithmic bytes they move and the floating-point operations they do.
template <class F>
static int prof_launch_f(svt_ctx* c, int cls, double bytes, double flops, F&& f) {
  if (!(c->prof_mask & (1u << cls))) return f();
  cudaEvent_t a = prof_event(c), b = prof_event(c);
  if (!a || !b) return f();
  // during stream capture the records must become external event-record nodes of the graph, so
  // that they are real timestamps on every replay
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(c->st, &cs);
  const unsigned flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  cudaEventRecordWithFlags(a, c->st, flags);
  int n = f();
  cudaEventRecordWithFlags(b, c->st, flags);
  c->prof_pending.push_back({cls, bytes, flops, a, b, false});
  return n;
}

template <class F>
static int prof_launch(svt_ctx* c, int cls, double bytes, F&& f) {
  return prof_launch_f(c, cls, bytes, 0.0, f);
}

// Called after the stream has drained: folds the recorded event pairs into the totals.
static void prof_harvest(svt_ctx* c) {
  for (auto& r : c->prof_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.cls] += ms;
      c->prof_bytes[r.cls] += r.bytes;
      c->prof_flops[r.cls] += r.flops;
      c->prof_n[r.cls] += 1;
    } else {
      (void)cudaGetLastError();
    }
    if (!r.graph_owned) {
      c->prof_pool.push_back(r.a);
      c->prof_pool.push_back(r.b);
    }
  }
  c->prof_pending.clear();
}

static svt_status check_err_word(svt_ctx* c, unsigned int e);

static svt_status sync_and_check(svt_ctx* c) {
  unsigned int* herr = reinterpret_cast<unsigned int*>(c->h_pin + 4 * kKMax - 1);
  CU(c, cudaMemcpyAsync(herr, c->err, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->st));
  CU(c, cudaStreamSynchronize(c->st));
  prof_harvest(c);
  return check_err_word(c, *herr);
}

// Reports (and clears) the device error word e, read after a synchronisation.
static svt_status check_err_word(svt_ctx* c, unsigned int e) {
  if (e) {
    CU(c, cudaMemsetAsync(c->err, 0, sizeof e, c->st));
    // A grid barrier that gave up leaves arrivals counted in its word, and the basis it was
    // orthonormalising half done (so other bits are often set in the same window): the word is
    // zeroed first, whatever else is reported, so that the next cooperative launch starts from a
    // clean barrier.  The Lanczos state is rebuilt by the next cycle (a fresh start block).
    if (e & SVT_DEVERR_BARRIER) {
      if (c->gbar) CU(c, cudaMemsetAsync(c->gbar, 0, 8, c->st));
      CU(c, cudaStreamSynchronize(c->st));
      c->warm_cols = 0;
      return fail(c, SVT_ERR_TIMEOUT, "a grid barrier of the cooperative orthonormalisation timed out");
    }
    if (e & SVT_DEVERR_INDEX_RANGE) return fail(c, SVT_ERR_ARG, "index outside [0,m) x [0,n)");
    if (e & SVT_DEVERR_DUPLICATE) return fail(c, SVT_ERR_DUP_INDEX, "duplicate (row, col) pair in Omega");
    if (e & SVT_DEVERR_NONFINITE) return fail(c, SVT_ERR_NUMERIC, "NaN or Inf in a reduction (basis Gram or residual)");
    if (e & SVT_DEVERR_CAPACITY) return fail(c, SVT_ERR_INTERNAL, "device buffer capacity exceeded");
    if (e & SVT_DEVERR_JACOBI) return fail(c, SVT_ERR_NUMERIC, "projected Jacobi SVD did not converge");
    // SVT_DEVERR_CHOL is informational (deflation handled in-kernel)
  }
  return SVT_OK;
}

// Orders the library stream after the caller's stream on entry, and the caller's stream after the
// library stream on exit.
struct StreamJoin {
  svt_ctx* c;
  explicit StreamJoin(svt_ctx* cc) : c(cc) {
    if (c && c->ev_in) {
      cudaEventRecord(c->ev_in, c->user_st);
      cudaStreamWaitEvent(c->st, c->ev_in, 0);
    }
  }
  ~StreamJoin() {
    if (c && c->ev_out) {
      cudaEventRecord(c->ev_out, c->st);
      cudaStreamWaitEvent(c->user_st, c->ev_out, 0);
    }
  }
};

// Device-to-host copy on the library stream, then wait for it.
static svt_status d2h_sync(svt_ctx* c, void* dst, const void* src, size_t bytes) {
  CU(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->st));
  CU(c, cudaStreamSynchronize(c->st));
  return SVT_OK;
}

// Block size for s_need wanted triplets: s_need plus max(4, s_need / 4) spare columns, at least the
// block option, rounded up to a multiple of 8, at most kBMax.  Beyond 28 wanted triplets the block
// stays at 32 and a thick restart keeps several blocks of Ritz pairs (cycle_shape).
static int choose_block(const svt_ctx* c, int s_need) {
  int b = s_need + std::max(kOversample, s_need / 4);
  if (c->opt.block > b) b = c->opt.block;
  b = (b + 7) / 8 * 8;
  if (b > kBMax) b = kBMax;
  if (b < 8) b = 8;
  return b;
}

// Shape of the Lanczos cycles for s wanted triplets: block b, block steps J, and nk, the blocks of
// leading Ritz pairs a thick restart keeps: enough to hold the s wanted ones plus kOversample guard
// columns (one block up to 28 wanted triplets), with at least one new block per cycle (two where K
// allows: J = max(lanczos_steps, nk + 2), K = J b <= kKMax).
static void cycle_shape(const svt_ctx* c, int s, int* b_out, int* J_out, int* nk_out) {
  const int b = choose_block(c, s);
  const int Jcap = kKMax / b;
  int nk = (s + kOversample + b - 1) / b;
  nk = std::max(1, std::min(nk, Jcap - 1));
  int J = std::min(c->opt.lanczos_steps > 0 ? c->opt.lanczos_steps : 3, Jcap);
  J = std::max(J, std::min(nk + 2, Jcap));
  *b_out = b;
  *J_out = std::max(1, J);
  *nk_out = nk;
}

static uint64_t next_seed(svt_ctx* c) {
  uint64_t z = c->opt.seed + (++c->rng_counter) * 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static void* ycur_csr(svt_ctx* c) { return c->Ycsr[c->ycur]; }
static void* ycur_csc(svt_ctx* c) { return c->Ycsc[c->ycur]; }

// Algorithmic bytes of one sparse product Out (n_out x b) = S X (X: n_in x b, float64 blocks):
// index + value stream, segment pointers, each row of X read once, Out written once.
static double spmm_bytes(const svt_ctx* c, int n_out, int n_in, int b) {
  return (double)c->nnz * (4.0 + (double)c->vbytes) + 4.0 * (n_out + 1) + 8.0 * b * ((double)n_in + n_out);
}

// Algorithmic bytes of the fused X-on-Omega + dual step: col_idx, csr_to_csc, M, Y read, Y and its
// column-major copy written, row pointers, the factors read once.
static double sddmm_bytes(const svt_ctx* c, int r) {
  return (double)c->nnz * (8.0 + 4.0 * (double)c->vbytes) + 4.0 * (c->m + 1) + 8.0 * r * ((double)c->m + c->n);
}

// ------------------------------------------------------------------------------------------------
// Block CGS2 + Cholesky QR of P (rows x b) against nq orthonormal blocks Q (stride q_stride).
// Coefficients: P_in = Q (C1 + C2) + P_out (R2 R1); written to Tcol / Tdiag when given.
// ------------------------------------------------------------------------------------------------
static svt_status orthonormalize(svt_ctx* c, double* P, const double* Q, long long q_stride, int nq, int rows, int b,
                                 double* Tcol, double* Tdiag, float* Pf = nullptr) {
  int l = 0;
  if (c->coop_grid > 0) {
    // one cooperative kernel: gram / update / Cholesky / update / correction phases with grid
    // barriers (same arithmetic as the launch sequence below)
    const double bytes = 8.0 * rows * b * (3.0 * (nq + 1) + 2.0 * nq + 3.0);
    // float64 flops the algorithm needs per row: Grams 2 nq b^2 + 2 b (first pass, diagonal of
    // P^T P), 2 nq b^2 + b (b + 1) (second pass, upper triangle), b (b + 1) (after the Cholesky);
    // projections 2 nq b^2 twice; forward substitution b^2; correction b^2.  A second correction
    // adds b (b + 1) + b^2.
    const double bb = (double)b * b, bu = (double)b * (b + 1);
    const double per_row = 8.0 * nq * bb + (nq > 0 ? 2.0 * b : 0.0) + 2.0 * bu + 2.0 * bb +
                           (c->two_corrections ? bu + bb : 0.0);
    const double flops = per_row * (double)rows;
    l += prof_launch_f(c, SVT_PROF_ORTH, bytes, flops, [&] {
      return launch_orth_coop(P, Q, q_stride, nq, rows, b, c->gpart, c->G1, c->G2, c->G3, Tcol, Tdiag, kKMax, Pf,
                              c->dcount, c->err, c->gbar, c->two_corrections ? 1 : 0, c->coop_grid, c->st,
                              c->orth_repass, c->barrier_spins,
                              c->orth_tc);
    });
    if (l == 0) return fail(c, SVT_ERR_CUDA, "cooperative orthonormalisation launch failed: %s",
                            cudaGetErrorString(cudaGetLastError()));
    return launched(c, l);
  }
  const double gram_q = 8.0 * rows * (nq + 1) * b, gram_p = 8.0 * rows * b;
  const double upd_q = 8.0 * rows * (nq + 2) * b, upd_p = 16.0 * rows * b;
  const double* G1 = nullptr;
  if (nq > 0) {
    // C1 = Q^T P; then P <- P - Q C1 fused with the Gram [Q, P]^T P of the projected block
    l += prof_launch(c, SVT_PROF_GRAM, gram_q,
                     [&] { return launch_gram(Q, q_stride, nq, P, rows, b, c->gpart, c->G1, c->st); });
    l += prof_launch(c, SVT_PROF_BLOCK_UPDATE, upd_q + gram_q, [&] {
      return launch_update_gram(0, Q, q_stride, nq, c->G1, nullptr, nullptr, P, rows, b, c->gpart, c->G2, c->st,
                                c->G1, Tcol, kKMax);
    });
    G1 = c->G1;
  } else {
    l += prof_launch(c, SVT_PROF_GRAM, gram_p,
                     [&] { return launch_gram(nullptr, 0, 0, P, rows, b, c->gpart, c->G2, c->st); });
  }
  l += prof_launch(c, SVT_PROF_SMALL, 0.0,
                   [&] { return launch_chol(G1, c->G2, nq, b, c->R1, c->dinv, c->dcount, c->st); });
  // P <- (P - Q C2) R1^-1 fused with the Gram P^T P
  l += prof_launch(c, SVT_PROF_BLOCK_UPDATE, upd_q + gram_p, [&] {
    return launch_update_gram(1, Q, q_stride, nq, c->G2, c->R1, c->dinv, P, rows, b, c->gpart, c->G3, c->st);
  });
  if (!c->two_corrections) {
    l += prof_launch(c, SVT_PROF_BLOCK_UPDATE, upd_p, [&] {
      return launch_correct(c->G3, c->R1, Tdiag, kKMax, nullptr, P, rows, b, c->dcount, c->st, Pf);
    });
  } else {
    // ill-conditioned blocks seen: a second first-order correction (orthonormality O(|E|^4))
    l += prof_launch(c, SVT_PROF_BLOCK_UPDATE, upd_p, [&] {
      return launch_correct(c->G3, c->R1, nullptr, kKMax, c->R2, P, rows, b, c->dcount, c->st);
    });
    l += prof_launch(c, SVT_PROF_GRAM, gram_p,
                     [&] { return launch_gram(nullptr, 0, 0, P, rows, b, c->gpart, c->G3, c->st); });
    l += prof_launch(c, SVT_PROF_BLOCK_UPDATE, upd_p, [&] {
      return launch_correct(c->G3, c->R2, Tdiag, kKMax, nullptr, P, rows, b, nullptr, c->st, Pf);
    });
  }
  return launched(c, l);
}

// Issues one block Golub-Kahan-Lanczos cycle with full reorthogonalisation from the start block in
// Vb[0] (n x b), ending with the projected SVD and the copy of the Ritz values, residual estimates
// and the orthonormality defect to pinned host memory.  Only stream operations: it can be captured.
//
// thick: a thick restart of the previous cycle (same b and J).  Its b leading Ritz pairs become
// block 0 (U_0 = U X[:, 0:b], V_0 = V W[:, 0:b]; Y V_0 = U_0 diag(theta) by the Lanczos relation
// Y V = U T and T = X diag(theta) W^T, so the projection on block 0 is diag(theta)), and the
// recurrence continues from the previous cycle's residual block V_J, which is orthogonal to all
// of V and becomes block 1: the cycle computes blocks 1 .. J-1 only.  The Krylov space is the one
// an explicit restart from V_0 would build (its next block lies in the span of V_J), for two
// sparse products and three orthonormalisations less.  Jprev: block steps of the previous cycle
// (its basis, projected vectors and residual block V_Jprev); the cycle itself may use another J.
//
// The cycle is issued in pieces (cycle_begin, then per block step the sparse product Y V_j,
// cycle_orth_left, the product Y^T U_j, cycle_orth_right, and cycle_end) so that the batched engine
// can interleave the pieces of several jobs and run the sparse products of all of them as one
// launch.
static svt_status cycle_begin(svt_ctx* c, int b, int J, bool thick, int Jprev, int nk, int* j0_out) {
  const int m = (int)c->m, n = (int)c->n;
  const long long su = (long long)m * b, sv = (long long)n * b;
  int j0 = 0;
  (void)J;
  if (!thick) {
    CU(c, cudaMemsetAsync(c->T, 0, sizeof(double) * kKMax * kKMax, c->st));
    TRY(orthonormalize(c, c->Vb, nullptr, 0, 0, n, b, nullptr, nullptr, c->Vsh));
  } else {
    // the nk b leading Ritz pairs become blocks 0 .. nk-1, block by block (Uwarm / Vwarm hold them
    // in the block layout of Ub / Vb), and the residual block V_Jprev becomes block nk
    const int Kp = Jprev * b;
    int l = prof_launch(c, SVT_PROF_COMBINE, 8.0 * ((double)m + n) * (Kp + nk * b), [&] {
      int q = 0;
      for (int j = 0; j < nk; ++j)
        q += launch_basis_combine(c->Ub, su, Jprev, b, m, c->Xl + j * b, Kp, b, nullptr, c->Uwarm + j * su, c->st) +
             launch_basis_combine(c->Vb, sv, Jprev, b, n, c->Wr + j * b, Kp, b, nullptr, c->Vwarm + j * sv, c->st);
      return q;
    });
    TRY(launched(c, l));
    // V_Jprev -> block nk (its float32 copy, written by its orthonormalisation, is still in Vsh);
    // the Ritz vectors -> blocks 0 .. nk-1
    CU(c, cudaMemcpyAsync(c->Vb + nk * sv, c->Vb + Jprev * sv, sizeof(double) * sv, cudaMemcpyDeviceToDevice, c->st));
    CU(c, cudaMemcpyAsync(c->Vb, c->Vwarm, sizeof(double) * nk * sv, cudaMemcpyDeviceToDevice, c->st));
    CU(c, cudaMemcpyAsync(c->Ub, c->Uwarm, sizeof(double) * nk * su, cudaMemcpyDeviceToDevice, c->st));
    CU(c, cudaMemsetAsync(c->T, 0, sizeof(double) * kKMax * kKMax, c->st));
    TRY(launched(c, launch_set_diagonal(c->T, kKMax, c->theta, nk * b, c->st)));
    j0 = nk;
  }
  *j0_out = j0;
  return SVT_OK;
}

// Launch precision of the sparse products: 0 float64, 1 float32, 2 bfloat16 values.
static int spmm_precision(const svt_ctx* c) { return c->bf16_active ? 2 : (c->prec == SVT_FP64 ? 0 : 1); }

// Operands of the sparse product of block step j: U_j = Y V_j (left) or V_{j+1} = Y^T U_j (right,
// column-major copy of the values).
static SpmmJob cycle_spmm_job(svt_ctx* c, int b, int j, bool left) {
  const long long su = (long long)c->m * b, sv = (long long)c->n * b;
  SpmmJob J{};
  if (left) {
    J.ptr = c->row_ptr;
    J.idx = c->col_idx;
    J.val = c->bf16_active ? static_cast<const void*>(c->Yb[c->ycur]) : ycur_csr(c);
    J.X = c->Vb + j * sv;
    J.Xf = c->Vsh;
    J.Out = c->Ub + j * su;
    J.n_out = (int)c->m;
  } else {
    J.ptr = c->col_ptr;
    J.idx = c->row_idx;
    J.val = c->bf16_active ? static_cast<const void*>(c->Ybc[c->ycur]) : ycur_csc(c);
    J.X = c->Ub + j * su;
    J.Xf = c->Ush;
    J.Out = c->Vb + (j + 1) * sv;
    J.n_out = (int)c->n;
  }
  J.b = b;
  J.nnz = c->nnz;
  J.wpr = 0;
  return J;
}

static svt_status cycle_spmm(svt_ctx* c, int b, int j, bool left) {
  const SpmmJob J = cycle_spmm_job(c, b, j, left);
  const int n_in = left ? (int)c->n : (int)c->m;
  const int l = prof_launch_f(c, left ? SVT_PROF_SPMM : SVT_PROF_SPMM_T, spmm_bytes(c, J.n_out, n_in, b),
                              2.0 * c->nnz * b, [&] {
    return launch_spmm(spmm_precision(c), J.ptr, J.idx, J.val, J.X, J.Xf, J.Out, J.n_out, b, c->st, c->nnz);
  });
  return launched(c, l);
}

// U_j against U_0 .. U_{j-1}; its coefficients go to column block j of T.
static svt_status cycle_orth_left(svt_ctx* c, int b, int j) {
  const long long su = (long long)c->m * b;
  return orthonormalize(c, c->Ub + j * su, c->Ub, su, j, (int)c->m, b, c->T + j * b,
                        c->T + (long long)j * b * kKMax + j * b, c->Ush);
}

// V_{j+1} against V_0 .. V_j; the last block's R goes to S (the residual coupling) and its float32
// copy is kept for a thick restart.
static svt_status cycle_orth_right(svt_ctx* c, int b, int j, int J) {
  const long long sv = (long long)c->n * b;
  return orthonormalize(c, c->Vb + (j + 1) * sv, c->Vb, sv, j + 1, (int)c->n, b, nullptr,
                        j == J - 1 ? c->S : nullptr, c->Vsh);
}

static svt_status cycle_end(svt_ctx* c, int b, int J, int nk, bool copy_out) {
  const int K = J * b;
  int l = 0;
  // S is written with leading dimension kKMax; the projected SVD reads it as b x b with leading
  // dimension b, so compact it first.
  CU(c, cudaMemcpy2DAsync(c->Rkeep, b * sizeof(double), c->S, kKMax * sizeof(double), b * sizeof(double), b,
                          cudaMemcpyDeviceToDevice, c->st));
  // one-sided Jacobi stops when every column pair is orthogonal to 1e-11: Ritz vectors and values
  // five orders beyond the float64 path's Lanczos tolerance (1e-6 sigma_1), and the float64
  // kernel then finishes in one float64 sweep after its float32 preconditioning
  const double tol_j = c->opt.lanczos_tol > 0 && c->opt.lanczos_tol < 1e-9
                           ? std::max(1e-15, 2.0 * K * 1.1102230246251565e-16)
                           : 1e-11;
  // Ritz vectors formed in float64: the nk b that a thick restart of this shape keeps (they cover
  // every wanted triplet)
  const int nvec = std::max(1, nk) * b;
  l += prof_launch(c, SVT_PROF_JACOBI, 24.0 * K * K, [&] {
    if (c->prec == SVT_FP64)
      return launch_small_svd(c->T, kKMax, K, c->Rkeep, b, nvec, c->theta, c->Xl, c->Wr, c->res, tol_j, 60, c->err,
                              c->dcount, c->st, c->opt.jacobi_cluster);
    return launch_small_svd_mixed(c->T, kKMax, K, c->Rkeep, b, c->theta, c->Xl, c->Wr, c->res, nvec, c->wsrc, 2e-6,
                                  60, c->err, c->dcount, c->st);
  });
  TRY(launched(c, l));
  if (!copy_out) return SVT_OK;
  CU(c, cudaMemcpyAsync(c->h_pin, c->theta, sizeof(double) * K, cudaMemcpyDeviceToHost, c->st));
  CU(c, cudaMemcpyAsync(c->h_pin + kKMax, c->res, sizeof(double) * K, cudaMemcpyDeviceToHost, c->st));
  CU(c, cudaMemcpyAsync(c->h_pin + 3 * kKMax + 1, c->dcount + 3, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  return SVT_OK;
}

static svt_status issue_cycle(svt_ctx* c, int b, int J, bool thick, int Jprev, int nk, bool copy_out = true) {
  int j0 = 0;
  TRY(cycle_begin(c, b, J, thick, Jprev, nk, &j0));
  for (int j = j0; j < J; ++j) {
    TRY(cycle_spmm(c, b, j, true));
    TRY(cycle_orth_left(c, b, j));
    TRY(cycle_spmm(c, b, j, false));
    TRY(cycle_orth_right(c, b, j, J));
  }
  return cycle_end(c, b, J, nk, copy_out);
}

// Captures issue_cycle for this (b, J, Y buffer, correction mode, restart kind) once and replays it
// afterwards: one graph launch instead of tens of kernel launches per cycle.
static svt_status run_cycle_graph(svt_ctx* c, int b, int J, bool thick, int Jprev, int nk) {
  const int twoc = c->two_corrections ? 1 : 0;
  const int tk = thick ? 1 : 0;
  const int jp = thick ? Jprev : 0;
  const int bf = c->bf16_active ? 1 : 0;
  for (auto& g : c->graphs)
    if (g.b == b && g.J == J && g.ycur == c->ycur && g.twoc == twoc && g.thick == tk && g.Jprev == jp &&
        g.bf16 == bf && g.nk == nk && g.prof_mask == c->prof_mask) {
      CU(c, cudaGraphLaunch(g.exec, c->st));
      c->launches += g.launches;
      // the graph's event-record nodes fire again on every replay: harvest them at the next sync
      for (auto& pn : g.prof) c->prof_pending.push_back({pn.cls, pn.bytes, pn.flops, pn.a, pn.b, true});
      return SVT_OK;
    }
  const int64_t l0 = c->launches;
  const size_t p0 = c->prof_pending.size();
  CU(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
  svt_status s = issue_cycle(c, b, J, thick, Jprev, nk);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->st, &graph);
  const int64_t nl = c->launches - l0;
  c->launches = l0;
  // event pairs recorded during capture belong to the graph (they only fire when it is replayed)
  std::vector<svt_ctx::ProfNode> prof;
  for (size_t i = p0; i < c->prof_pending.size(); ++i) {
    const auto& r = c->prof_pending[i];
    prof.push_back({r.cls, r.bytes, r.flops, r.a, r.b});
  }
  c->prof_pending.resize(p0);
  if (s != SVT_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    (void)cudaGetLastError();
    for (auto& pn : prof) {
      c->prof_pool.push_back(pn.a);
      c->prof_pool.push_back(pn.b);
    }
    if (s != SVT_OK) return s;
    return fail(c, SVT_ERR_CUDA, "stream capture of the Lanczos cycle failed: %s", cudaGetErrorString(e));
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(c, SVT_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
  }
  c->graphs.push_back({b, J, c->ycur, twoc, tk, jp, bf, nk, c->prof_mask, exec, nl, prof});
  CU(c, cudaGraphLaunch(exec, c->st));
  c->launches += nl;
  for (auto& pn : prof) c->prof_pending.push_back({pn.cls, pn.bytes, pn.flops, pn.a, pn.b, true});
  return SVT_OK;
}

// One cycle, then the host reads the Ritz values and residual estimates (theta/res, pinned).
static svt_status lanczos_cycle(svt_ctx* c, int b, int J, bool thick, int Jprev, int nk, const double** theta_h,
                                const double** res_h) {
  NvtxRange nv("svt: Lanczos cycle (SpMM, reorthogonalisation, projected SVD)");
  if (c->opt.use_graphs) {
    TRY(run_cycle_graph(c, b, J, thick, Jprev, nk));
  } else {
    TRY(issue_cycle(c, b, J, thick, Jprev, nk));
  }
  const int nspmm = 2 * (thick ? J - nk : J);
  c->last_spmm += nspmm;
  c->total_spmm += nspmm;
  c->last_cycles += 1;
  c->total_cycles += 1;
  TRY(sync_and_check(c));
  {
    double defect = 0.0;
    std::memcpy(&defect, c->h_pin + 3 * kKMax + 1, sizeof defect);
    if (defect > 1e-6) c->two_corrections = true;
  }
  *theta_h = c->h_pin;
  *res_h = c->h_pin + kKMax;
  return SVT_OK;
}

// Start block of the next cycle: the first `cols` right Ritz vectors V_basis Wr[:, 0:cols] (or the
// warm-start block), random columns after them.
static svt_status set_start_block(svt_ctx* c, int b, int warm) {
  const int n = (int)c->n;
  int l = 0;
  if (warm > 0) {
    // Vwarm is n x warm_cols (row-major, ld = warm_cols); copy the first `warm` columns into Vb[0] (ld b)
    CU(c, cudaMemcpy2DAsync(c->Vb, b * sizeof(double), c->Vwarm, c->warm_cols * sizeof(double), warm * sizeof(double),
                            n, cudaMemcpyDeviceToDevice, c->st));
  }
  if (warm < b) l += launch_random_block(c->Vb, n, b, warm, next_seed(c), c->st);
  return launched(c, l);
}

// Keep the first `cols` right Ritz vectors of the last cycle (basis V_0..V_{J-1}) in Vwarm.
static svt_status keep_ritz(svt_ctx* c, int b, int J, int cols) {
  const int n = (int)c->n;
  const int K = J * b;
  cols = std::min(cols, std::min(K, kBMax));
  int l = prof_launch(c, SVT_PROF_COMBINE, 8.0 * n * (K + cols), [&] {
    return launch_basis_combine(c->Vb, (long long)n * b, J, b, n, c->Wr, K, cols, nullptr, c->Vwarm, c->st);
  });
  c->warm_cols = cols;
  return launched(c, l);
}

// Rank-adaptive partial SVD of the current Y (Sec. 5.1.1).  Computes the leading singular triplets
// until the rank policy stops: s = s_init; converge the first s triplets; while sigma_s > tau,
// s += ell (reusing the converged Ritz vectors as the start block).  On return theta_out holds the
// converged values (host), *s_out the final s, *K_out/J_out/b_out the last cycle's shape.
// strict: the first s_init triplets must all meet the residual tolerance and s never grows (used
// for ||P_Omega M||_2, where the value itself matters).
// One rank-adaptive partial SVD in progress: the state partial_svd carries from one Lanczos cycle
// to the next (the batched engine keeps one per job).
struct ShrinkRun {
  double tau = 0.0, tol = 0.0;
  int kmin = 0, s = 0, passes = 1, b = 0, J = 0, nk = 1, max_cycles = 40;
  bool thick = false;   // the next cycle is a thick restart of the previous one
  int Jprev = 0;        // block steps of the previous cycle
  // cycles of the current pass of the rank policy: each pass is a partial SVD of its own (Sec. 5.1.1
  // asks the partial SVD for s_k triplets, then for s_k + l, ...), with its own cycle budget and
  // stagnation clock
  int cyc = 0;
  bool strict = false;
};

static svt_status shrink_start(svt_ctx* c, ShrinkRun& R, int s_init, double tau, bool strict) {
  R.kmin = (int)std::min(c->m, c->n);
  // float32 values and products carry ~1e-6 of sigma_1 of rounding into the Lanczos relation
  // (length-~100 float32 sums); the float64 path asks for kLanczosTolF64 (much tighter
  // tolerances stall on some 30000 x 30000 shrinks)
  R.tol = c->opt.lanczos_tol > 0 ? c->opt.lanczos_tol : (c->prec == SVT_FP64 ? kLanczosTolF64 : kLanczosTolF32);
  R.tau = tau;
  R.strict = strict;
  R.s = std::min(s_init, R.kmin);
  R.passes = 1;
  cycle_shape(c, R.s, &R.b, &R.J, &R.nk);
  c->last_cycles = 0;
  c->last_spmm = 0;
  TRY(set_start_block(c, R.b, std::min(c->warm_cols, R.b)));
  R.max_cycles = c->opt.max_cycles > 0 ? c->opt.max_cycles : 40;
  R.thick = false;
  R.Jprev = 0;
  R.cyc = 0;
  return SVT_OK;
}

// Applies the rank policy and the convergence test to the Ritz values th and residual estimates
// rs of the cycle just run.  *done: the partial SVD is finished (theta_out, *s_out, ... set);
// otherwise R holds the shape of the next cycle (its start block is issued).
static svt_status shrink_advance(svt_ctx* c, ShrinkRun& R, const double* th, const double* rs, bool* done,
                                 std::vector<double>& theta_out, int* s_out, int* passes_out, int* b_out, int* J_out) {
  *done = false;
  if (!std::isfinite(th[0]) || !std::isfinite(rs[0]))
    return fail(c, SVT_ERR_NUMERIC, "non-finite Ritz value or residual estimate");
  // stagnation: a cluster of Ritz values that the working precision cannot separate further
  // keeps its residuals above tol; after 10 cycles of one shrink the tolerance is relaxed 30x,
  // after 25 cycles 300x (recorded in the relaxed_shrinks counter)
  const double tol_c = R.cyc >= 25 ? 300.0 * R.tol : (R.cyc >= 10 ? 30.0 * R.tol : R.tol);
  R.thick = false;
  R.Jprev = R.J;
  const int b = R.b;
  const int K = R.J * b;
  const int s_eff = std::min(R.s, K);
  // Ritz values are lower bounds of the singular values (interlacing of U^T Y V), so
  // theta_s > tau already proves sigma_s > tau: the rank policy grows s without waiting for
  // convergence.  Otherwise every Ritz triplet above tau must be converged to `tol`, and the
  // first Ritz value at or below tau must be resolved (residual <= 1e-3 theta_1: the Krylov
  // space has found the singular value it stands for; an unresolved Ritz value with a large
  // residual bounds no particular singular value) and bounded away from tau
  // (theta + residual <= tau).
  const double tau = R.tau;
  const bool grow = !R.strict && th[s_eff - 1] > tau && R.s < R.kmin;
  int conv = 0;
  bool all_conv = !grow;
  for (int i = 0; i < s_eff && all_conv; ++i) {
    const bool above = R.strict || th[i] > tau;
    const bool ok = rs[i] <= tol_c * th[0] || (!above && rs[i] <= 1e-3 * th[0] && th[i] + rs[i] <= tau);
    if (!ok) all_conv = false;
    else ++conv;
    if (!above) break;
  }
  if (all_conv || grow) {
    if (grow) {
      if (R.s + c->opt.ell > kMaxRankCap + 1) {
        theta_out.assign(th, th + s_eff);
        *s_out = R.s;
        return fail(c, SVT_ERR_RANK_LIMIT, "more than %d singular values exceed tau", kMaxRankCap);
      }
      R.s = std::min(R.s + c->opt.ell, R.kmin);
      ++R.passes;
      int nb = 0;
      cycle_shape(c, R.s, &nb, &R.J, &R.nk);
      TRY(keep_ritz(c, b, R.Jprev, std::min(b, nb)));
      R.b = nb;
      TRY(set_start_block(c, R.b, std::min(c->warm_cols, R.b)));
      R.cyc = 0;
      return SVT_OK;
    }
    theta_out.assign(th, th + s_eff);
    *s_out = s_eff;
    *passes_out = R.passes;
    if (R.cyc >= 10) c->relaxed_shrinks += 1;
    *b_out = b;
    *J_out = R.J;
    *done = true;
    return SVT_OK;
  }
  if (R.cyc + 1 >= R.max_cycles)
    return fail(c, SVT_ERR_NUMERIC, "Lanczos did not converge in %d cycles (converged %d of %d, res %.3e)",
                R.max_cycles, conv, s_eff, rs[std::min(conv, s_eff - 1)] / th[0]);
  // not converged, same block: continue from the leading Ritz pairs (nk blocks) and the residual
  // block, extending the space by restart_steps - nk blocks
  int Jr = std::min(c->opt.restart_steps > 0 ? c->opt.restart_steps : R.J, kKMax / b);
  Jr = std::max(Jr, std::min(R.nk + 1, kKMax / b));
  if (Jr >= R.nk + 1) {
    R.thick = true;
    R.J = Jr;
  } else {
    TRY(keep_ritz(c, b, R.J, b));
    TRY(set_start_block(c, b, b));
  }
  ++R.cyc;
  return SVT_OK;
}

static svt_status partial_svd(svt_ctx* c, int s_init, double tau, std::vector<double>& theta_out, int* s_out,
                              int* passes_out, int* b_out, int* J_out, bool strict = false) {
  ShrinkRun R;
  TRY(shrink_start(c, R, s_init, tau, strict));
  for (;;) {
    const double *th, *rs;
    TRY(lanczos_cycle(c, R.b, R.J, R.thick, R.Jprev, R.nk, &th, &rs));
    bool done = false;
    TRY(shrink_advance(c, R, th, rs, &done, theta_out, s_out, passes_out, b_out, J_out));
    if (done) return SVT_OK;
  }
}

// X = D_tau(Y): factors of the triplets with sigma > tau from the last cycle.
// The factors of D_tau(Y) from the converged Ritz triplets th of the last cycle (shape b, J).
static svt_status shrink_finish(svt_ctx* c, double tau, const std::vector<double>& th, int s, int passes, int b,
                                int J, int* r_out) {
  int r = 0;
  while (r < (int)th.size() && th[r] > tau) ++r;
  if (r > c->max_rank) return fail(c, SVT_ERR_RANK_LIMIT, "rank %d exceeds max_rank %d", r, c->max_rank);
  const int m = (int)c->m, n = (int)c->n;
  const int K = J * b;
  c->d_host.assign(r, 0.0);
  for (int i = 0; i < r; ++i) c->d_host[i] = th[i] - tau;
  c->last_s = s;
  c->last_passes = passes;
  c->last_sigma1 = th.empty() ? 0.0 : th[0];
  int l = 0;
  if (r > 0) {
    std::memcpy(c->h_pin + 2 * kKMax, c->d_host.data(), sizeof(double) * r);
    CU(c, cudaMemcpyAsync(c->scale, c->h_pin + 2 * kKMax, sizeof(double) * r, cudaMemcpyHostToDevice, c->st));
    // float32 path: the factors of the fused update are also written as float32 rows padded to a
    // multiple of four values (16-byte gathers)
    c->ldf = (r + 3) & ~3;
    l += prof_launch(c, SVT_PROF_COMBINE, 8.0 * (2.0 * m * (K + r) + n * (K + r)), [&] {
      return launch_basis_combine(c->Ub, (long long)m * b, J, b, m, c->Xl, K, r, nullptr, c->Uf, c->st) +
             launch_basis_combine(c->Ub, (long long)m * b, J, b, m, c->Xl, K, r, c->scale, c->Ut, c->st, c->Utf,
                                  c->ldf) +
             launch_basis_combine(c->Vb, (long long)n * b, J, b, n, c->Wr, K, r, nullptr, c->Vf, c->st, c->Vff,
                                  c->ldf);
    });
  }
  c->ldu = r;
  TRY(launched(c, l));
  // warm start of the next shrink: the leading right Ritz vectors
  TRY(keep_ritz(c, b, J, std::min(b, std::max(r + c->opt.ell + 1, 8))));
  c->r = r;
  *r_out = r;
  return SVT_OK;
}

static svt_status shrink_current(svt_ctx* c, double tau, int s_init, int* r_out) {
  NvtxRange nv("svt: shrink D_tau (rank-adaptive partial SVD, Ritz vectors)");
  std::vector<double> th;
  int s = 0, passes = 0, b = 0, J = 0;
  TRY(partial_svd(c, s_init, tau, th, &s, &passes, &b, &J));
  return shrink_finish(c, tau, th, s, passes, b, J, r_out);
}

// D_tau(Y) by a randomized range finder (Sec. 6, the first of the two alternatives the paper names):
// Y ~ Q Q^T Y with Q an orthonormal basis of Y Omega refined by power steps, and D_tau(Q Q^T Y) from the
// SVD of the small factor.  Every product is the library's sparse product, every basis goes through
// the block orthonormalisation, and the small SVD is the projected-SVD kernel:
//   Omega (n x l, warm columns then SplitMix64 columns) -> orthonormalised (same span(Y Omega); it
//   also writes the float32 copy the float32 products read);  Q = orth(Y Omega);  power steps
//   Q = orth(Y orth(Y^T Q));  Z = Y^T Q = P R (orthonormalisation with R written to T);
//   R = Xl diag(theta) Wr^T (projected SVD)  =>  Q^T Y = Z^T = Wr diag(theta) (P Xl)^T, so
//   U = Q Wr and V = P Xl are the singular vectors of Q Q^T Y with values theta.
// The rank policy of Sec. 5.1.1 (s_k = r_{k-1} + 1, s_k += l while theta_{s_k} > tau) repeats the
// pass with the previous pass's right vectors as warm columns.
static svt_status shrink_randomized(svt_ctx* c, double tau, int s_init, int* r_out) {
  NvtxRange nv("svt: shrink D_tau (randomized range finder)");
  const int m = (int)c->m, n = (int)c->n;
  const int kmin = (int)std::min(c->m, c->n);
  const int p = c->opt.rsvd_oversample;
  const int q = c->opt.rsvd_power;
  double* Q = c->Ub;                 // m x l
  double* Om = c->Vb;                // n x l
  double* P = nullptr;               // n x l (block 1 of Vb, placed once l is known)
  int s = std::min(s_init, kmin);
  int passes = 0;
  c->last_cycles = 0;
  c->last_spmm = 0;
  for (;;) {
    if (s + p > kBMax && s < kmin)
      return fail(c, SVT_ERR_RANK_LIMIT, "randomized shrink: s_k + oversampling = %d exceeds %d test columns", s + p,
                  kBMax);
    const int l = std::min(kBMax, (s + p + 7) / 8 * 8);
    P = c->Vb + (long long)n * l;
    const int c0 = std::min(c->warm_cols, l);
    if (c0 > 0)
      CU(c, cudaMemcpy2DAsync(Om, l * sizeof(double), c->Vwarm, c->warm_cols * sizeof(double), c0 * sizeof(double), n,
                              cudaMemcpyDeviceToDevice, c->st));
    const uint64_t seed = c->opt.rsvd_seed + 1000ull * (uint64_t)(c->k + 1) + (uint64_t)passes;
    if (c0 < l) TRY(launched(c, launch_random_block(Om, n, l, c0, seed, c->st)));
    ++passes;
    auto prod = [&](bool transpose, const double* X, const float* Xf, double* Out) -> svt_status {
      const int n_out = transpose ? n : m;
      int l2 = prof_launch_f(c, transpose ? SVT_PROF_SPMM_T : SVT_PROF_SPMM,
                             spmm_bytes(c, n_out, transpose ? m : n, l), 2.0 * c->nnz * l, [&] {
        return transpose ? launch_spmm(c->prec, c->col_ptr, c->row_idx, ycur_csc(c), X, Xf, Out, n, l, c->st, c->nnz)
                         : launch_spmm(c->prec, c->row_ptr, c->col_idx, ycur_csr(c), X, Xf, Out, m, l, c->st, c->nnz);
      });
      c->last_spmm += 1;
      c->total_spmm += 1;
      return launched(c, l2);
    };
    TRY(orthonormalize(c, Om, nullptr, 0, 0, n, l, nullptr, nullptr, c->Vsh));
    TRY(prod(false, Om, c->Vsh, Q));
    TRY(orthonormalize(c, Q, nullptr, 0, 0, m, l, nullptr, nullptr, c->Ush));
    for (int it = 0; it < q; ++it) {
      TRY(prod(true, Q, c->Ush, P));
      TRY(orthonormalize(c, P, nullptr, 0, 0, n, l, nullptr, nullptr, c->Vsh));
      TRY(prod(false, P, c->Vsh, Q));
      TRY(orthonormalize(c, Q, nullptr, 0, 0, m, l, nullptr, nullptr, c->Ush));
    }
    TRY(prod(true, Q, c->Ush, P));
    CU(c, cudaMemsetAsync(c->T, 0, sizeof(double) * kKMax * kKMax, c->st));
    TRY(orthonormalize(c, P, nullptr, 0, 0, n, l, nullptr, c->T, c->Vsh));
    const double tol_j = std::max(1e-15, 2.0 * l * 1.1102230246251565e-16);
    int lj = prof_launch(c, SVT_PROF_JACOBI, 24.0 * l * l, [&] {
      if (c->prec == SVT_FP64)
        return launch_small_svd(c->T, kKMax, l, nullptr, l, l, c->theta, c->Xl, c->Wr, c->res, tol_j, 60, c->err,
                                c->dcount, c->st, c->opt.jacobi_cluster);
      return launch_small_svd_mixed(c->T, kKMax, l, nullptr, l, c->theta, c->Xl, c->Wr, c->res, l, c->wsrc, 2e-6, 60,
                                    c->err, c->dcount, c->st);
    });
    TRY(launched(c, lj));
    CU(c, cudaMemcpyAsync(c->h_pin, c->theta, sizeof(double) * l, cudaMemcpyDeviceToHost, c->st));
    c->last_cycles += 1;
    c->total_cycles += 1;
    TRY(sync_and_check(c));
    const double* th = c->h_pin;
    if (!std::isfinite(th[0])) return fail(c, SVT_ERR_NUMERIC, "non-finite singular value estimate");
    // right singular vectors of this pass, V = P Xl (all l): the warm columns of the next pass or shrink
    int lc = prof_launch(c, SVT_PROF_COMBINE, 8.0 * (double)n * 2 * l, [&] {
      return launch_basis_combine(P, (long long)n * l, 1, l, n, c->Xl, l, l, nullptr, c->Vwarm, c->st);
    });
    TRY(launched(c, lc));
    c->warm_cols = l;
    const int s_eff = std::min(s, l);
    if (s_eff < kmin && th[s_eff - 1] > tau) {
      s = std::min(s + c->opt.ell, kmin);
      continue;
    }
    int r = 0;
    while (r < l && th[r] > tau) ++r;
    if (r > c->max_rank) return fail(c, SVT_ERR_RANK_LIMIT, "rank %d exceeds max_rank %d", r, c->max_rank);
    c->d_host.assign(r, 0.0);
    for (int i = 0; i < r; ++i) c->d_host[i] = th[i] - tau;
    c->last_s = s_eff;
    c->last_passes = passes;
    c->last_sigma1 = th[0];
    if (r > 0) {
      std::memcpy(c->h_pin + 2 * kKMax, c->d_host.data(), sizeof(double) * r);
      CU(c, cudaMemcpyAsync(c->scale, c->h_pin + 2 * kKMax, sizeof(double) * r, cudaMemcpyHostToDevice, c->st));
      c->ldf = (r + 3) & ~3;
      int l3 = prof_launch(c, SVT_PROF_COMBINE, 8.0 * (2.0 * m * (l + r) + n * (l + r)), [&] {
        return launch_basis_combine(Q, (long long)m * l, 1, l, m, c->Wr, l, r, nullptr, c->Uf, c->st) +
               launch_basis_combine(Q, (long long)m * l, 1, l, m, c->Wr, l, r, c->scale, c->Ut, c->st, c->Utf,
                                    c->ldf) +
               launch_basis_combine(P, (long long)n * l, 1, l, n, c->Xl, l, r, nullptr, c->Vf, c->st, c->Vff,
                                    c->ldf);
      });
      TRY(launched(c, l3));
    }
    c->ldu = r;
    c->r = r;
    *r_out = r;
    return SVT_OK;
  }
}

static svt_status shrink_dispatch(svt_ctx* c, double tau, int s_init, int* r_out) {
  if (c->opt.shrink_engine == SVT_SHRINK_RANDOMIZED) return shrink_randomized(c, tau, s_init, r_out);
  return shrink_current(c, tau, s_init, r_out);
}

// ------------------------------------------------------------------------------------------------
// C-ABI
// ------------------------------------------------------------------------------------------------
extern "C" void svt_default_options(svt_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof *opt);
  opt->precision = SVT_FP64;
  opt->block = 0;
  opt->ell = 5;
  opt->k_max = 1000;
  opt->lanczos_steps = 3;
  opt->max_cycles = 40;
  opt->lanczos_tol = 0.0;
  opt->indices_on_device = 0;
  opt->use_graphs = 1;
  opt->seed = 0x5eed5eedULL;
  opt->stream = nullptr;
  opt->fused_orth = 1;
  opt->restart_steps = 0;
  opt->bf16_switch = 1e-2;
  opt->orth_grid = 0;
  opt->orth_repass = 0.0;
  opt->device_alloc = nullptr;
  opt->device_free = nullptr;
  opt->alloc_user = nullptr;
  opt->shrink_engine = SVT_SHRINK_LANCZOS;
  opt->rsvd_oversample = 8;
  opt->rsvd_power = 1;
  opt->rsvd_seed = 0;
  opt->device_loop = 1;
  opt->orth_tf32 = 0;
  opt->jacobi_cluster = 0;
}

extern "C" const char* svt_last_error(const svt_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

extern "C" int64_t svt_kernel_launches(const svt_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" void svt_destroy(svt_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  for (auto& g : c->graphs) {
    cudaGraphExecDestroy(g.exec);
    for (auto& pn : g.prof) {
      cudaEventDestroy(pn.a);
      cudaEventDestroy(pn.b);
    }
  }
  c->graphs.clear();
  for (auto& g : c->igraphs) cudaGraphExecDestroy(g.exec);
  c->igraphs.clear();
  for (void* p : c->allocations) dev_free(c, p);
  if (c->h_pin) cudaFreeHost(c->h_pin);
  if (c->dl_pin) cudaFreeHost(c->dl_pin);
  for (auto& r : c->prof_pending) {
    if (r.graph_owned) continue;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->st) cudaStreamDestroy(c->st);
  delete c;
}

static svt_status build_structure(svt_ctx* c, const int32_t* rows_d, const int32_t* cols_d, const double* M_d) {
  const int m = (int)c->m, n = (int)c->n;
  const long long nnz = c->nnz;
  int32_t *counts, *cursor, *scan_scratch, *src, *rows_csr, *maxseg;
  const long long nmax = std::max<long long>(m, n) + 1;
  TmpBufs tmp(c);
  if (!tmp.get(&counts, nmax) || !tmp.get(&cursor, nmax) || !tmp.get(&scan_scratch, scan_scratch_ints(nmax)) ||
      !tmp.get(&src, nnz) || !tmp.get(&rows_csr, nnz) || !tmp.get(&maxseg, 1))
    return fail(c, SVT_ERR_OOM, "device allocation of build scratch failed");
  int32_t* host_ptr = nullptr;
  int l = 0;
  // ---- CSR: major = row, minor = col, payload = input position
  CU(c, cudaMemsetAsync(counts, 0, sizeof(int32_t) * nmax, c->st));
  CU(c, cudaMemsetAsync(cursor, 0, sizeof(int32_t) * nmax, c->st));
  l += launch_count_major(rows_d, cols_d, nnz, m, n, counts, c->err, c->st);
  l += launch_exclusive_scan(counts, c->row_ptr, m, scan_scratch, c->st);
  l += launch_scatter_segments(rows_d, cols_d, nullptr, nnz, m, n, c->row_ptr, cursor, c->col_idx, src, c->st);
  l += launch_sort_segments(c->row_ptr, m, c->col_idx, src, c->st);
  l += launch_max_segment(c->row_ptr, m, maxseg, c->st);
  TRY(launched(c, l)); l = 0;
  TRY(sync_and_check(c));
  int32_t mx = 0;
  TRY(d2h_sync(c, &mx, maxseg, sizeof mx));
  if (mx > segment_smem_capacity()) {
    host_ptr = new (std::nothrow) int32_t[m + 1];
    if (!host_ptr) return fail(c, SVT_ERR_OOM, "host allocation failed");
    if (d2h_sync(c, host_ptr, c->row_ptr, sizeof(int32_t) * (m + 1)) != SVT_OK) {
      delete[] host_ptr;
      return SVT_ERR_CUDA;
    }
    int32_t* scratch = nullptr;
    int L = 1;
    while (L < mx) L <<= 1;
    if (!tmp.get(&scratch, 2LL * L)) { delete[] host_ptr; return fail(c, SVT_ERR_OOM, "sort scratch"); }
    for (int i = 0; i < m; ++i) {
      int len = host_ptr[i + 1] - host_ptr[i];
      if (len > segment_smem_capacity())
        l += launch_sort_long_segment(c->col_idx + host_ptr[i], src + host_ptr[i], len, scratch, c->st);
    }
    delete[] host_ptr;
    host_ptr = nullptr;
    TRY(launched(c, l)); l = 0;
  }
  l += launch_check_duplicates(c->row_ptr, m, c->col_idx, c->err, c->st);
  // values in row-major order
  if (c->prec == SVT_FP64) l += launch_gather_f64(M_d, src, nnz, (double*)c->Mv, c->st);
  else l += launch_gather_f64_to_f32(M_d, src, nnz, (float*)c->Mv, c->st);
  l += launch_expand_ptr(c->row_ptr, m, rows_csr, c->st);
  // ---- CSC: major = col, minor = row, payload = row-major position
  CU(c, cudaMemsetAsync(counts, 0, sizeof(int32_t) * nmax, c->st));
  CU(c, cudaMemsetAsync(cursor, 0, sizeof(int32_t) * nmax, c->st));
  l += launch_count_major(c->col_idx, rows_csr, nnz, n, m, counts, c->err, c->st);
  l += launch_exclusive_scan(counts, c->col_ptr, n, scan_scratch, c->st);
  // payload: identity positions 0..nnz-1 (nullptr => p)
  l += launch_scatter_segments(c->col_idx, rows_csr, nullptr, nnz, n, m, c->col_ptr, cursor, c->row_idx,
                               c->csc_to_csr, c->st);
  l += launch_sort_segments(c->col_ptr, n, c->row_idx, c->csc_to_csr, c->st);
  l += launch_max_segment(c->col_ptr, n, maxseg, c->st);
  TRY(launched(c, l)); l = 0;
  TRY(sync_and_check(c));
  TRY(d2h_sync(c, &mx, maxseg, sizeof mx));
  if (mx > segment_smem_capacity()) {
    host_ptr = new (std::nothrow) int32_t[n + 1];
    if (!host_ptr) return fail(c, SVT_ERR_OOM, "host allocation failed");
    if (d2h_sync(c, host_ptr, c->col_ptr, sizeof(int32_t) * (n + 1)) != SVT_OK) {
      delete[] host_ptr;
      return SVT_ERR_CUDA;
    }
    int32_t* scratch = nullptr;
    int L = 1;
    while (L < mx) L <<= 1;
    if (!tmp.get(&scratch, 2LL * L)) { delete[] host_ptr; return fail(c, SVT_ERR_OOM, "sort scratch"); }
    for (int j = 0; j < n; ++j) {
      int len = host_ptr[j + 1] - host_ptr[j];
      if (len > segment_smem_capacity())
        l += launch_sort_long_segment(c->row_idx + host_ptr[j], c->csc_to_csr + host_ptr[j], len, scratch, c->st);
    }
    delete[] host_ptr;
    TRY(launched(c, l)); l = 0;
  }
  l += launch_invert_perm(c->csc_to_csr, nnz, c->csr_to_csc, c->st);
  // ||P_Omega M||_F (float64, from the input values)
  l += launch_sumsq_f64(M_d, nnz, c->upd_partial, c->dscal, c->st);
  TRY(launched(c, l));
  TRY(sync_and_check(c));
  double ss = 0.0;
  TRY(d2h_sync(c, &ss, c->dscal, sizeof ss));
  if (!std::isfinite(ss)) return fail(c, SVT_ERR_ARG, "M_omega holds a NaN or Inf value");
  c->normF = std::sqrt(ss);
  return SVT_OK;
}

// Allocations, input staging and the Omega storage build of svt_create.  Local temporaries are
// released when this returns, before svt_create destroys a failed context.
static svt_status create_body(svt_ctx* c, const int32_t* rows, const int32_t* cols, const double* M_omega) {
  NvtxRange nv("svt_create (Omega storage: CSR, CSC, permutations)");
  const int64_t m = c->m, n = c->n, nnz = c->nnz;
  StreamJoin join(c);
  TRY(dalloc_t(c, &c->err, 4));
  CU(c, cudaMemsetAsync(c->err, 0, 4, c->st));
  TRY(dalloc_t(c, &c->row_ptr, m + 1));
  TRY(dalloc_t(c, &c->col_idx, nnz));
  TRY(dalloc_t(c, &c->col_ptr, n + 1));
  TRY(dalloc_t(c, &c->row_idx, nnz));
  TRY(dalloc_t(c, &c->csc_to_csr, nnz));
  TRY(dalloc_t(c, &c->csr_to_csc, nnz));
  TRY(dalloc(c, &c->Mv, nnz * c->vbytes));
  for (int i = 0; i < 2; ++i) {
    TRY(dalloc(c, &c->Ycsr[i], nnz * c->vbytes));
    TRY(dalloc(c, &c->Ycsc[i], nnz * c->vbytes));
  }
  const int cap = kMaxRankCap + 1;
  TRY(dalloc_t(c, &c->Ut, (size_t)m * cap));
  TRY(dalloc_t(c, &c->Uf, (size_t)m * cap));
  TRY(dalloc_t(c, &c->Vf, (size_t)n * cap));
  TRY(dalloc_t(c, &c->Vwarm, (size_t)n * kKMax));
  TRY(dalloc_t(c, &c->Uwarm, (size_t)m * kKMax));
  if (c->bf16_mode) {
    for (int i = 0; i < 2; ++i) {
      TRY(dalloc(c, &c->Yb[i], nnz * 2));
      TRY(dalloc(c, &c->Ybc[i], nnz * 2));
    }
  }
  if (c->prec == SVT_FP32) {
    const size_t capf = (size_t)((cap + 3) & ~3);
    TRY(dalloc_t(c, &c->Ush, (size_t)m * kBMax));
    TRY(dalloc_t(c, &c->Vsh, (size_t)n * kBMax));
    TRY(dalloc_t(c, &c->Utf, (size_t)m * capf));
    TRY(dalloc_t(c, &c->Vff, (size_t)n * capf));
  }
  TRY(dalloc_t(c, &c->Ub, (size_t)m * (kKMax + kBMax)));
  TRY(dalloc_t(c, &c->Vb, (size_t)n * (kKMax + kBMax)));
  TRY(dalloc_t(c, &c->T, (size_t)kKMax * kKMax));
  TRY(dalloc_t(c, &c->S, (size_t)kKMax * kBMax));
  TRY(dalloc_t(c, &c->theta, kKMax));
  TRY(dalloc_t(c, &c->Xl, (size_t)kKMax * kKMax));
  TRY(dalloc_t(c, &c->Wr, (size_t)kKMax * kKMax));
  TRY(dalloc_t(c, &c->res, kKMax));
  TRY(dalloc_t(c, &c->wsrc, (size_t)kKMax * kKMax));
  TRY(dalloc_t(c, &c->G1, kGramW * kBMax));
  TRY(dalloc_t(c, &c->G2, kGramW * kBMax));
  TRY(dalloc_t(c, &c->G3, kGramW * kBMax));
  TRY(dalloc_t(c, &c->R1, kBMax * kBMax));
  TRY(dalloc_t(c, &c->R2, kBMax * kBMax));
  TRY(dalloc_t(c, &c->dinv, kBMax));
  TRY(dalloc_t(c, &c->dcount, 8));
  TRY(dalloc(c, &c->gbar, 8));
  CU(c, cudaMemsetAsync(c->gbar, 0, 8, c->st));
  CU(c, cudaMemsetAsync(c->dcount, 0, 8 * sizeof(unsigned long long), c->st));
  // (nq + 1) b <= kGramW columns against b <= 32: at most kGramW x 32 entries per row chunk
  TRY(dalloc_t(c, &c->gpart, (size_t)gram_partial_doubles((int)std::max(m, n), kGramW / kBMax - 1, kBMax)));
  TRY(dalloc_t(c, &c->Rkeep, kBMax * kBMax));
  TRY(dalloc_t(c, &c->scale, kKMax));
  TRY(dalloc_t(c, &c->dl_prm, 1));
  TRY(dalloc_t(c, &c->dl_st, 1));
  CU(c, cudaMallocHost((void**)&c->dl_pin, 2048));
  TRY(dalloc_t(c, &c->upd_partial, std::max(sddmm_partial_doubles(), 1024)));
  TRY(dalloc_t(c, &c->dscal, 16));
  CU(c, cudaMallocHost((void**)&c->h_pin, sizeof(double) * 4 * kKMax));
  CU(c, cudaEventCreate(&c->ev0));
  CU(c, cudaEventCreate(&c->ev1));
  // inputs on the device
  const int32_t *rows_d = rows, *cols_d = cols;
  const double* M_d = M_omega;
  TmpBufs staged(c);
  if (!c->opt.indices_on_device) {
    int32_t *r2, *c2;
    double* m2;
    if (!staged.get(&r2, nnz) || !staged.get(&c2, nnz) || !staged.get(&m2, nnz))
      return fail(c, SVT_ERR_OOM, "device allocation of the input copy failed");
    CU(c, cudaMemcpyAsync(r2, rows, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, c->st));
    CU(c, cudaMemcpyAsync(c2, cols, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, c->st));
    CU(c, cudaMemcpyAsync(m2, M_omega, sizeof(double) * nnz, cudaMemcpyHostToDevice, c->st));
    rows_d = r2; cols_d = c2; M_d = m2;
  }
  TRY(build_structure(c, rows_d, cols_d, M_d));
  // Y^0 = 0 until configured
  CU(c, cudaMemsetAsync(c->Ycsr[0], 0, nnz * c->vbytes, c->st));
  CU(c, cudaMemsetAsync(c->Ycsc[0], 0, nnz * c->vbytes, c->st));
  return sync_and_check(c);
}

// Device bytes of a context: the persistent buffers of create_body plus the scratch of the
// structure build (input staging, counting sort, segment sorts), plus a fixed allowance for
// allocation rounding, the captured graphs and the pinned staging.
extern "C" size_t svt_estimate_device_bytes(int64_t m, int64_t n, int64_t nnz, const svt_options* opt) {
  if (m < 1 || n < 1 || nnz < 0) return 0;
  svt_options o;
  svt_default_options(&o);
  if (opt) o = *opt;
  const bool bf16 = o.precision == SVT_BF16;
  const size_t vb = o.precision == SVT_FP64 ? 8 : 4;
  const size_t M = (size_t)m, N = (size_t)n, Z = (size_t)nnz, cap = kMaxRankCap + 1;
  size_t b = 0;
  b += 4 * (M + 1) + 4 * (N + 1) + 4 * 4 * Z;                 // row_ptr, col_ptr, col_idx, row_idx, perms
  b += 5 * Z * vb;                                           // M, two Y copies in both orders
  b += 8 * (2 * M + N) * cap + 8 * (M + N) * kKMax;          // factors, warm-start / kept Ritz blocks
  if (bf16) b += 4 * 2 * Z;                                  // bfloat16 copies of Y
  if (o.precision != SVT_FP64) b += 4 * (M + N) * kBMax + 4 * (M + N) * ((cap + 3) & ~3);
  b += 8 * (M + N) * (kKMax + kBMax);                        // Lanczos bases
  b += 8 * (3 * kKMax * kKMax + kKMax * kBMax + 3 * kGramW * kBMax + 3 * kBMax * kBMax + 256 + 4096);
  b += 4 * kKMax * kKMax;                                    // float32 Ritz vectors of the projected SVD
  b += 8 * (size_t)gram_partial_doubles((int)std::max(m, n), kGramW / kBMax - 1, kBMax);
  // scratch of the structure build, peak (host inputs staged as int32, int32, float64)
  const size_t nmax = std::max(M, N) + 1;
  size_t pow2 = 1;
  while (pow2 < nmax) pow2 <<= 1;
  b += 16 * Z + 8 * Z + 8 * nmax + 8 * pow2 + 4 * (size_t)scan_scratch_ints((long long)nmax);
  return b + (4u << 20);
}

extern "C" svt_status svt_create(int64_t m, int64_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
                                 const double* M_omega, const svt_options* opt, svt_ctx** out) {
  if (!out) return fail(nullptr, SVT_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (m < 1 || n < 1 || m >= (1LL << 31) || n >= (1LL << 31))
    return fail(nullptr, SVT_ERR_ARG, "dimensions must satisfy 1 <= m, n < 2^31");
  if (nnz < 1 || nnz >= (1LL << 31) || nnz > m * n) return fail(nullptr, SVT_ERR_ARG, "need 1 <= nnz <= m*n, nnz < 2^31");
  if (!rows || !cols || !M_omega) return fail(nullptr, SVT_ERR_ARG, "rows, cols and M_omega must be non-NULL");
  svt_options o;
  svt_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != SVT_FP64 && o.precision != SVT_FP32 && o.precision != SVT_BF16)
    return fail(nullptr, SVT_ERR_ARG, "unknown precision");
  if (o.precision == SVT_BF16 && !(o.bf16_switch >= 0.0)) return fail(nullptr, SVT_ERR_ARG, "bf16_switch must be >= 0");
  if (o.orth_grid < 0) return fail(nullptr, SVT_ERR_ARG, "orth_grid must be >= 0");
  if (!(o.orth_repass == o.orth_repass)) return fail(nullptr, SVT_ERR_ARG, "orth_repass is NaN");
  if (o.jacobi_cluster != 0 && o.jacobi_cluster != 1) return fail(nullptr, SVT_ERR_ARG, "jacobi_cluster must be 0 or 1");
  if ((o.device_alloc == nullptr) != (o.device_free == nullptr))
    return fail(nullptr, SVT_ERR_ARG, "device_alloc and device_free must be given together");
  if (o.shrink_engine != SVT_SHRINK_LANCZOS && o.shrink_engine != SVT_SHRINK_RANDOMIZED)
    return fail(nullptr, SVT_ERR_ARG, "unknown shrink engine");
  if (o.shrink_engine == SVT_SHRINK_RANDOMIZED &&
      (std::min(m, n) < 32 || o.rsvd_oversample < 1 || o.rsvd_oversample > 24 || o.rsvd_power < 0 ||
       o.rsvd_power > 8))
    return fail(nullptr, SVT_ERR_ARG,
                "randomized shrink needs min(m, n) >= 32, 1 <= rsvd_oversample <= 24, 0 <= rsvd_power <= 8");
  if (o.ell < 1) o.ell = 5;
  if (o.k_max < 1) o.k_max = 1000;
  if (o.lanczos_steps < 1) o.lanczos_steps = 3;
  if (o.max_cycles < 1) o.max_cycles = 40;
  svt_ctx* c = new (std::nothrow) svt_ctx();
  if (!c) return fail(nullptr, SVT_ERR_OOM, "host allocation failed");
  c->opt = o;
  c->m = m; c->n = n; c->nnz = nnz;
  c->bf16_mode = o.precision == SVT_BF16;
  c->prec = c->bf16_mode ? SVT_FP32 : o.precision;   // float32 values; the bfloat16 copies are extra
  c->vbytes = c->prec == SVT_FP64 ? 8 : 4;
  c->user_st = (cudaStream_t)o.stream;
  c->orth_repass = o.orth_repass == 0.0 ? 1e-6 : (o.orth_repass < 0.0 ? 0.0 : o.orth_repass);
  // tensor-core first pass: by default for FP32 / BF16 values only; it needs the repeated pass
  c->orth_tc = (o.orth_tf32 > 0 || (o.orth_tf32 == 0 && c->prec != SVT_FP64)) && c->orth_repass > 0.0 ? 1 : 0;
  svt_status s = SVT_OK;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    s = fail(c, SVT_ERR_CUDA, "no CUDA device");
  } else if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
             cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    s = fail(c, SVT_ERR_CUDA, "stream/event creation failed");
  } else if (init_jacobi_attributes() != 0) {
    s = fail(c, SVT_ERR_CUDA, "setting the shared-memory limit of the projected-SVD kernels failed");
  } else {
    // the partial-Gram buffer holds at most 2 * 152 row chunks (gram_partial_doubles)
    c->coop_grid = o.fused_orth ? std::min(orth_coop_init(), 2 * 152) : 0;
    if (c->coop_grid > 0 && o.orth_grid > 0) c->coop_grid = std::min(c->coop_grid, o.orth_grid);
    s = create_body(c, rows, cols, M_omega);
  }
  if (s != SVT_OK) {
    (void)cudaGetLastError();
    g_create_error = c->last_error;
    svt_destroy(c);
    return s;
  }
  *out = c;
  return SVT_OK;
}

extern "C" svt_status svt_configure(svt_ctx* c, double tau, double delta, double eps, int max_rank, int64_t k0) {
  if (!c) return SVT_ERR_ARG;
  NvtxRange nv("svt_configure (kick: ||P_Omega M||_2, k0, Y^0)");
  StreamJoin join(c);
  if (max_rank < 1 || max_rank > kMaxRankCap)
    return fail(c, SVT_ERR_ARG, "max_rank must be in [1, %d]", kMaxRankCap);
  const double mn = (double)c->m * (double)c->n;
  c->tau = tau > 0 ? tau : 5.0 * std::sqrt(mn);
  c->delta = delta > 0 ? delta : 1.2 * mn / (double)c->nnz;
  c->eps = eps > 0 ? eps : 1e-4;
  c->max_rank = max_rank;
  if (!std::isfinite(c->tau) || !std::isfinite(c->delta)) return fail(c, SVT_ERR_ARG, "tau/delta not finite");
  // ||P_Omega M||_2: leading singular value of Y = P_Omega M (Lanczos, s = 1); for the Dantzig
  // selector the operand of the first shrinks is k delta soft_E(B) instead (see svt_set_dantzig)
  c->ycur = 0;
  c->warm_cols = 0;
  if (c->ds_E > 0.0)
    TRY(launched(c, launch_dual_kick(c->prec, c->Mv, 1.0, c->ds_E, c->Ycsr[0], c->Ycsc[0], nullptr, nullptr,
                                     c->csr_to_csc, c->nnz, c->st)));
  else
    TRY(launched(c, launch_scale_values(c->prec, c->Mv, 1.0, c->Ycsr[0], c->Ycsc[0], c->csr_to_csc, c->nnz, c->st)));
  std::vector<double> th;
  int s = 0, passes = 0, b = 0, J = 0;
  // huge tau so that the rank policy stops after the first converged triplet
  TRY(partial_svd(c, 1, INFINITY, th, &s, &passes, &b, &J, /*strict=*/true));
  c->norm2 = th.empty() ? 0.0 : th[0];
  if (!(c->norm2 > 0.0))
    return fail(c, SVT_ERR_NUMERIC, c->ds_E > 0.0 ? "soft_E(B) is zero: X = 0 already meets |B - X| <= E"
                                                  : "||P_Omega M||_2 is zero");
  TRY(keep_ritz(c, b, J, std::min(b, 8)));
  // the randomized engine's first shrink starts from random test columns only
  if (c->opt.shrink_engine == SVT_SHRINK_RANDOMIZED) c->warm_cols = 0;
  if (k0 >= 0) c->k0 = k0;
  else c->k0 = (int64_t)std::ceil(c->tau / (c->delta * c->norm2));
  if (c->ds_E > 0.0)
    TRY(launched(c, launch_dual_kick(c->prec, c->Mv, (double)c->k0 * c->delta, c->ds_E, c->Ycsr[0], c->Ycsc[0],
                                     c->Yp[0], c->Ym[0], c->csr_to_csc, c->nnz, c->st)));
  else
    TRY(launched(c, launch_scale_values(c->prec, c->Mv, (double)c->k0 * c->delta, c->Ycsr[0], c->Ycsc[0],
                                        c->csr_to_csc, c->nnz, c->st)));
  c->bf16_active = false;
  if (c->bf16_mode && !(c->ds_E > 0.0)) {
    // the kick's ||P_Omega M||_2 above was taken on the float32 values; the iterations start on
    // the bfloat16 copies
    TRY(launched(c, launch_to_bf16((const float*)c->Ycsr[0], (const float*)c->Ycsc[0], c->Yb[0], c->Ybc[0], c->nnz,
                                   c->st)));
    c->bf16_active = true;
  }
  c->r = 0;
  c->k = 0;
  c->d_host.clear();
  c->configured = true;
  return sync_and_check(c);
}

extern "C" svt_status svt_set_dantzig(svt_ctx* c, double E) {
  if (!c) return SVT_ERR_ARG;
  if (!std::isfinite(E)) return fail(c, SVT_ERR_ARG, "E must be finite");
  StreamJoin join(c);
  if (E > 0.0) {
    for (int i = 0; i < 2; ++i) {
      if (!c->Yp[i]) TRY(dalloc(c, &c->Yp[i], c->nnz * c->vbytes));
      if (!c->Ym[i]) TRY(dalloc(c, &c->Ym[i], c->nnz * c->vbytes));
    }
  }
  c->ds_E = E > 0.0 ? E : 0.0;
  c->configured = false;   // the multipliers exist only after the next svt_configure / svt_solve
  return SVT_OK;
}

extern "C" svt_status svt_set_noise_stop(svt_ctx* c, double sigma, double eps_noise) {
  if (!c) return SVT_ERR_ARG;
  if (!(eps_noise >= 0.0) || !std::isfinite(eps_noise) || !std::isfinite(sigma))
    return fail(c, SVT_ERR_ARG, "eps_noise must be finite and >= 0, sigma finite");
  c->noise_sigma = sigma > 0.0 ? sigma : 0.0;
  c->noise_eps = eps_noise;
  return SVT_OK;
}

// ------------------------------------------------------------------------------------------------
// One SVT iteration as one graph (Algorithm 1's loop body with the shrink's Lanczos cycles, rank
// policy and convergence test on the device; Sec. 5.1.1, Sec. 5.1.5)
// ------------------------------------------------------------------------------------------------
// Pinned staging of the device loop (dl_pin): params, state, res2, error word, defect, theta.
constexpr size_t kPinPrm = 0, kPinSt = 64, kPinRes2 = 128, kPinErr = 136, kPinDefect = 144, kPinTheta = 152;

static bool device_loop_ok(const svt_ctx* c) {
  return c->opt.device_loop && !c->dl_broken && c->opt.use_graphs && c->prof_mask == 0 &&
         c->opt.shrink_engine == SVT_SHRINK_LANCZOS;
}

// Bound on r_k that the graph's Ritz-vector and update kernels are shaped for (r <= max_rank <= 64).
static int iter_rank_bound(int b, int nk) { return std::min(nk * b, kMaxRankCap); }

// Captures: the first Lanczos cycle of the shrink (start block already in Vb[0]) and the device
// test; a `while` node whose body is a thick restart and the test again (the test sets the node's
// condition: repeat while neither converged, grown nor out of budget); then the Ritz vectors of the
// r_k converged triplets (r_k read on the device), the warm start of the next shrink (b right
// Ritz vectors), the fused X-on-Omega + dual step + residual, and the copies of the outcome to
// pinned memory.  Stream operations only.
static svt_status capture_iter_graph(svt_ctx* c, int b, int J, int nk, svt_ctx::IterGraph* out) {
  const int m = (int)c->m, n = (int)c->n;
  const int K = J * b;
  const int rb = iter_rank_bound(b, nk);
  const int ldf = (rb + 3) & ~3;
  const int nxt = 1 - c->ycur;
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  cudaGraph_t g = nullptr;
  CU(c, cudaGraphCreate(&g, 0));
  struct GraphGuard {
    cudaGraph_t g;
    ~GraphGuard() { if (g) cudaGraphDestroy(g); }
  } guard{g};
  cudaGraphConditionalHandle cond;
  CU(c, cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault));
  auto end_capture = [&](cudaGraph_t* gg, svt_status s) -> svt_status {
    cudaGraph_t got = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->st, &got);
    if (s != SVT_OK) return s;
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(c, SVT_ERR_CUDA, "capture of the iteration graph failed: %s", cudaGetErrorString(e));
    }
    *gg = got;
    return SVT_OK;
  };
  // segment 1: first cycle + test
  const int64_t l0 = c->launches;
  CU(c, cudaStreamBeginCaptureToGraph(c->st, g, nullptr, nullptr, 0, mode));
  svt_status s = SVT_OK;
  if (cudaMemsetAsync(&c->dl_st->cycles, 0, sizeof(int), c->st) != cudaSuccess)
    s = fail(c, SVT_ERR_CUDA, "memset of the loop state failed");
  if (s == SVT_OK) s = issue_cycle(c, b, J, false, 0, nk, false);
  if (s == SVT_OK)
    s = launched(c, launch_cycle_decide(c->dl_prm, c->dl_st, c->theta, c->res, K, c->scale, cond, 1, c->st));
  std::vector<cudaGraphNode_t> deps;
  if (s == SVT_OK) {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(c->st, &cs, nullptr, nullptr, &d, nullptr, &nd) != cudaSuccess)
      s = fail(c, SVT_ERR_CUDA, "cudaStreamGetCaptureInfo failed");
    else
      deps.assign(d, d + nd);
  }
  TRY(end_capture(&g, s));
  const int64_t l_pre = c->launches - l0;
  // the while node
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  CU(c, cudaGraphAddNode(&cnode, g, deps.data(), nullptr, deps.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const int64_t l1 = c->launches;
  CU(c, cudaStreamBeginCaptureToGraph(c->st, body, nullptr, nullptr, 0, mode));
  s = issue_cycle(c, b, J, true, J, nk, false);
  if (s == SVT_OK)
    s = launched(c, launch_cycle_decide(c->dl_prm, c->dl_st, c->theta, c->res, K, c->scale, cond, 1, c->st));
  TRY(end_capture(&body, s));
  const int64_t l_body = c->launches - l1;
  // segment 3: Ritz vectors, warm start, fused update, outcome
  const int64_t l2 = c->launches;
  CU(c, cudaStreamBeginCaptureToGraph(c->st, g, &cnode, nullptr, 1, mode));
  const int* rdev = &c->dl_st->r;
  int l = 0;
  l += launch_basis_combine(c->Ub, (long long)m * b, J, b, m, c->Xl, K, rb, nullptr, c->Uf, c->st, nullptr, 0, rdev,
                            rb);
  l += launch_basis_combine(c->Ub, (long long)m * b, J, b, m, c->Xl, K, rb, c->scale, c->Ut, c->st, c->Utf, ldf, rdev,
                            rb);
  l += launch_basis_combine(c->Vb, (long long)n * b, J, b, n, c->Wr, K, rb, nullptr, c->Vf, c->st, c->Vff, ldf, rdev,
                            rb);
  l += launch_basis_combine(c->Vb, (long long)n * b, J, b, n, c->Wr, K, b, nullptr, c->Vwarm, c->st);
  SddmmDual dual{c->Yp[c->ycur], c->Ym[c->ycur], c->Yp[nxt], c->Ym[nxt], c->ds_E};
  l += launch_sddmm_update(c->prec, c->row_ptr, c->col_idx, c->csr_to_csc, c->Mv, ycur_csr(c), c->Ycsr[nxt],
                           c->Ycsc[nxt], c->Ut, c->Vf, c->Utf, c->Vff, ldf, rb, (int)c->m, c->delta, c->upd_partial,
                           c->dscal, c->err, c->st, c->ds_E > 0.0 ? &dual : nullptr,
                           c->bf16_active ? c->Yb[nxt] : nullptr, c->bf16_active ? c->Ybc[nxt] : nullptr, rdev, rb);
  s = launched(c, l);
  auto cp_d2h = [&](size_t off, const void* src, size_t bytes) {
    if (s == SVT_OK && cudaMemcpyAsync(c->dl_pin + off, src, bytes, cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
      s = fail(c, SVT_ERR_CUDA, "copy of the iteration outcome failed");
  };
  cp_d2h(kPinSt, c->dl_st, sizeof(LoopState));
  cp_d2h(kPinRes2, c->dscal, sizeof(double));
  cp_d2h(kPinErr, c->err, sizeof(unsigned int));
  cp_d2h(kPinDefect, c->dcount + 3, sizeof(double));
  cp_d2h(kPinTheta, c->theta, sizeof(double) * K);
  TRY(end_capture(&g, s));
  const int64_t l_post = c->launches - l2;
  c->launches = l0;
  cudaGraphExec_t exec = nullptr;
  CU(c, cudaGraphInstantiate(&exec, g, 0));
  *out = svt_ctx::IterGraph{b, J, nk, c->ycur, c->two_corrections ? 1 : 0, c->bf16_active ? 1 : 0, c->delta,
                            c->ds_E, exec, l_pre, l_body, l_post};
  return SVT_OK;
}

// The tail of an iteration shared by both paths: residual of eq. (5.5) (or the noisy rule), the
// record, and the stop test (commit Y' unless stopped).
static svt_status finish_step(svt_ctx* c, int r, double res2, float ms, svt_step_info* info) {
  const int nxt = 1 - c->ycur;
  const double res = std::sqrt(res2) / c->normF;
  c->k += 1;
  if (info) {
    info->k = c->k;
    info->r = r;
    info->s = c->last_s;
    info->passes = c->last_passes;
    info->lanczos_cycles = c->last_cycles;
    info->spmm_calls = c->last_spmm;
    info->residual = res;
    info->sigma1 = c->last_sigma1;
    info->ms = ms;
  }
  if (!std::isfinite(res)) return fail(c, SVT_ERR_NUMERIC, "residual is not finite");
  if (c->noise_sigma > 0.0 && !(c->ds_E > 0.0)) {
    // eq. (5.10): ||P_Omega(X^k - B)||_F^2 <= (1 + eps) m sigma^2 with m = |Omega|
    if (res2 <= (1.0 + c->noise_eps) * (double)c->nnz * c->noise_sigma * c->noise_sigma) return SVT_STOPPED;
  } else if (res <= c->eps) {
    return SVT_STOPPED;
  }
  // bfloat16 ladder: from here on the sparse products read the float32 values
  if (c->bf16_active && res < c->opt.bf16_switch) c->bf16_active = false;
  c->ycur = nxt;
  return SVT_OK;
}

// Host path: the shrink decided on the host cycle by cycle, then the fused update.
static svt_status step_host(svt_ctx* c, svt_step_info* info, int s_init) {
  int r = 0;
  TRY(shrink_dispatch(c, c->tau, s_init, &r));
  const int nxt = 1 - c->ycur;
  NvtxRange nv_upd("svt: fused X on Omega + dual step + residual");
  SddmmDual dual{c->Yp[c->ycur], c->Ym[c->ycur], c->Yp[nxt], c->Ym[nxt], c->ds_E};
  const double upd_bytes = sddmm_bytes(c, r) + (c->ds_E > 0.0 ? 4.0 * c->nnz * c->vbytes - c->nnz * c->vbytes : 0.0);
  TRY(launched(c, prof_launch_f(c, SVT_PROF_SDDMM, upd_bytes, (2.0 * r + 4.0) * c->nnz, [&] {
    return launch_sddmm_update(c->prec, c->row_ptr, c->col_idx, c->csr_to_csc, c->Mv, ycur_csr(c), c->Ycsr[nxt],
                               c->Ycsc[nxt], c->Ut, c->Vf, c->Utf, c->Vff, c->ldf, r, (int)c->m, c->delta,
                               c->upd_partial, c->dscal, c->err, c->st, c->ds_E > 0.0 ? &dual : nullptr,
                               c->bf16_active ? c->Yb[nxt] : nullptr, c->bf16_active ? c->Ybc[nxt] : nullptr);
  })));
  CU(c, cudaMemcpyAsync(c->h_pin + 3 * kKMax, c->dscal, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CU(c, cudaEventRecord(c->ev1, c->st));
  TRY(sync_and_check(c));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  return finish_step(c, r, c->h_pin[3 * kKMax], ms, info);
}

// Device path: one graph launch and one synchronisation per iteration.  When the rank policy grows
// s (theta_s > tau) the iteration is finished on the host path from s + l (the graph's update is
// discarded: Y' is only committed by finish_step).
static svt_status step_device(svt_ctx* c, svt_step_info* info) {
  const int kmin = (int)std::min(c->m, c->n);
  const int s = std::min(c->r + 1, kmin);
  int b = 0, J = 0, nk = 1;
  cycle_shape(c, s, &b, &J, &nk);
  int Jr = std::min(c->opt.restart_steps > 0 ? c->opt.restart_steps : J, kKMax / b);
  Jr = std::max(Jr, std::min(nk + 1, kKMax / b));
  if (Jr != J) return step_host(c, info, s);   // restarts of another length: the host loop
  const double tol = c->opt.lanczos_tol > 0 ? c->opt.lanczos_tol : (c->prec == SVT_FP64 ? kLanczosTolF64 : kLanczosTolF32);
  c->last_cycles = 0;
  c->last_spmm = 0;
  TRY(set_start_block(c, b, std::min(c->warm_cols, b)));
  LoopParams* hp = reinterpret_cast<LoopParams*>(c->dl_pin + kPinPrm);
  *hp = LoopParams{c->tau, tol, s, kmin, c->opt.max_cycles > 0 ? c->opt.max_cycles : 40, 0};
  CU(c, cudaMemcpyAsync(c->dl_prm, hp, sizeof(LoopParams), cudaMemcpyHostToDevice, c->st));
  const int twoc = c->two_corrections ? 1 : 0, bf = c->bf16_active ? 1 : 0;
  svt_ctx::IterGraph* g = nullptr;
  for (auto& ig : c->igraphs)
    if (ig.b == b && ig.J == J && ig.nk == nk && ig.ycur == c->ycur && ig.twoc == twoc && ig.bf16 == bf &&
        ig.delta == c->delta && ig.dsE == c->ds_E) {
      g = &ig;
      break;
    }
  if (!g) {
    svt_ctx::IterGraph ng{};
    const int64_t l_before = c->launches;
    if (capture_iter_graph(c, b, J, nk, &ng) != SVT_OK) {
      // the device cannot run the iteration graph (conditional nodes unsupported): the host loop
      (void)cudaGetLastError();
      c->launches = l_before;
      c->dl_broken = true;
      c->dl_reason = c->last_error;
      c->last_error.clear();
      return step_host(c, info, s);
    }
    c->igraphs.push_back(ng);
    g = &c->igraphs.back();
  }
  CU(c, cudaGraphLaunch(g->exec, c->st));
  CU(c, cudaEventRecord(c->ev1, c->st));
  CU(c, cudaStreamSynchronize(c->st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  LoopState ls;
  std::memcpy(&ls, c->dl_pin + kPinSt, sizeof ls);
  unsigned int e = 0;
  std::memcpy(&e, c->dl_pin + kPinErr, sizeof e);
  double defect = 0.0, res2 = 0.0;
  std::memcpy(&defect, c->dl_pin + kPinDefect, sizeof defect);
  std::memcpy(&res2, c->dl_pin + kPinRes2, sizeof res2);
  const double* th = reinterpret_cast<const double*>(c->dl_pin + kPinTheta);
  c->launches += g->l_pre + (int64_t)std::max(0, ls.cycles - 1) * g->l_body + g->l_post;
  c->last_cycles = ls.cycles;
  c->last_spmm = 2 * J + 2 * std::max(0, ls.cycles - 1) * (J - nk);
  c->total_cycles += ls.cycles;
  c->total_spmm += c->last_spmm;
  if (defect > 1e-6) c->two_corrections = true;
  TRY(check_err_word(c, e));
  switch (ls.status) {
    case kLoopConverged: break;
    case kLoopGrow: {
      // grow s on the host from the Ritz vectors the graph kept (b columns in Vwarm)
      c->warm_cols = b;
      const int cyc = c->last_cycles, spmm = c->last_spmm;
      svt_status st2 = step_host(c, info, std::min(s + c->opt.ell, kmin));
      if (info) {
        info->lanczos_cycles += cyc;
        info->spmm_calls += spmm;
        info->passes += 1;
      }
      return st2;
    }
    case kLoopBudget:
      return fail(c, SVT_ERR_NUMERIC, "Lanczos did not converge in %d cycles (converged %d of %d, res %.3e)",
                  ls.cycles, ls.conv, ls.s_eff, ls.res_fail);
    default:
      return fail(c, SVT_ERR_NUMERIC, "non-finite Ritz value or residual estimate");
  }
  const int r = ls.r;
  if (r > c->max_rank) return fail(c, SVT_ERR_RANK_LIMIT, "rank %d exceeds max_rank %d", r, c->max_rank);
  c->d_host.assign(r, 0.0);
  for (int i = 0; i < r; ++i) c->d_host[i] = th[i] - c->tau;
  c->r = r;
  c->ldu = iter_rank_bound(b, nk);
  c->ldf = (c->ldu + 3) & ~3;
  c->warm_cols = b;
  c->last_s = ls.s_eff;
  c->last_passes = 1;
  c->last_sigma1 = th[0];
  c->relaxed_shrinks += ls.relaxed;
  c->dl_iters += 1;
  return finish_step(c, r, res2, ms, info);
}

extern "C" svt_status svt_step(svt_ctx* c, svt_step_info* info) {
  if (!c) return SVT_ERR_ARG;
  NvtxRange nv("svt_step");
  StreamJoin join(c);
  if (!c->configured) return fail(c, SVT_ERR_ARG, "svt_configure (or svt_solve) must come first");
  CU(c, cudaEventRecord(c->ev0, c->st));
  if (device_loop_ok(c)) return step_device(c, info);
  return step_host(c, info, c->r + 1);
}

extern "C" svt_status svt_solve(svt_ctx* c, double tau, double delta, double eps, int max_rank, svt_result* out) {
  if (!c) return SVT_ERR_ARG;
  NvtxRange nv("svt_solve");
  StreamJoin join(c);
  cudaEvent_t e0, e1;
  CU(c, cudaEventCreate(&e0));
  CU(c, cudaEventCreate(&e1));
  CU(c, cudaEventRecord(e0, c->st));
  const int64_t spmm0 = c->total_spmm, cyc0 = c->total_cycles;
  svt_status s = svt_configure(c, tau, delta, eps, max_rank, -1);
  svt_step_info info{};
  info.residual = INFINITY;
  bool converged = false;
  if (s == SVT_OK) {
    for (int it = 0; it < c->opt.k_max; ++it) {
      s = svt_step(c, &info);
      if (s == SVT_STOPPED) { converged = true; s = SVT_OK; break; }
      if (s != SVT_OK) break;
    }
    if (s == SVT_OK && !converged) s = fail(c, SVT_ERR_NOT_CONVERGED, "k_max iterations reached");
  }
  cudaEventRecord(e1, c->st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (out) {
    out->iterations = c->k;
    out->k0 = c->k0;
    out->rank = c->r;
    out->converged = converged ? 1 : 0;
    out->residual = info.residual;
    out->norm2_M = c->norm2;
    out->normF_M = c->normF;
    out->ms = ms;
    out->spmm_calls = c->total_spmm - spmm0;
    out->lanczos_cycles = c->total_cycles - cyc0;
  }
  return s;
}

extern "C" svt_status svt_set_tau(svt_ctx* c, double tau) {
  if (!c) return SVT_ERR_ARG;
  if (!(tau > 0.0) || !std::isfinite(tau)) return fail(c, SVT_ERR_ARG, "tau must be positive and finite");
  if (!c->configured) return fail(c, SVT_ERR_ARG, "svt_configure (or svt_solve) must come first");
  c->tau = tau;
  c->k = 0;
  return SVT_OK;
}

// ------------------------------------------------------------------------------------------------
// Batched engine: Algorithm 1 for several independent completion problems at once, in lockstep.
// Every SVT iteration of the batch runs the shrinks of all unfinished jobs together, one Lanczos
// cycle of every still-shrinking job at a time; inside a cycle the sparse products of all jobs at
// the same block step are one persistent launch over the job list (launch_spmm_jobs), and the
// fused updates of all jobs are one launch (launch_sddmm_update_jobs).  Orthonormalisations,
// projected SVDs and Ritz vectors stay per job.  Each job's decisions (rank policy, convergence,
// thick restarts, stop rule) are those of its solo run; with the fixed tile rule its sparse
// products are computed exactly as solo, so every iterate equals the solo iterate (the residual
// sums differ in grouping only).  One host synchronisation per lockstep cycle and one per
// iteration serve the whole batch.
// ------------------------------------------------------------------------------------------------
namespace {

// Warps per segment chosen by the tuner, per (precision, block, direction, mean segment length
// class), for the whole process.
struct TuneKey {
  int prec, b, left, len_class;
  bool operator==(const TuneKey& o) const {
    return prec == o.prec && b == o.b && left == o.left && len_class == o.len_class;
  }
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, int>> g_tune;

int len_class(long long nnz, int n_out) {
  const double mean = n_out > 0 ? (double)nnz / n_out : 0.0;
  int k = 0;
  while (k < 30 && (double)(1LL << (k + 1)) <= mean) ++k;
  return k;
}

}  // namespace

// Times the candidate tile shapes (warps per segment 1, 2, 4, 8) of one product on the batch
// stream and returns the fastest.  Runs real products (into the job's own output block, which the
// batched launch overwrites), three timed launches per candidate after one untimed.
static int tune_spmm(svt_ctx* c, const SpmmJob& J0, int prec, cudaStream_t st) {
  cudaEvent_t a = nullptr, z = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&z) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    (void)cudaGetLastError();
    return 0;
  }
  int best = 0;
  float best_ms = 0.f;
  for (int w = 1; w <= 8; w <<= 1) {
    SpmmJob J = J0;
    J.wpr = w;
    launch_spmm_jobs(prec, &J, 1, 0, st);
    cudaEventRecord(a, st);
    for (int rep = 0; rep < 3; ++rep) launch_spmm_jobs(prec, &J, 1, 0, st);
    cudaEventRecord(z, st);
    if (cudaEventSynchronize(z) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, z);
    if (best == 0 || ms < best_ms) {
      best = w;
      best_ms = ms;
    }
    c->launches += 4;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(z);
  (void)cudaGetLastError();
  return best;
}

static int tuned_wpr(svt_ctx* c, const SpmmJob& J, int prec, bool left, cudaStream_t st) {
  const TuneKey key{prec, J.b, left ? 1 : 0, len_class(J.nnz, J.n_out)};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto& e : g_tune)
      if (e.first == key) return e.second;
  }
  const int w = tune_spmm(c, J, prec, st);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.push_back({key, w});
  return w;
}

extern "C" void svt_batch_default_options(svt_batch_options* opt) {
  if (!opt) return;
  opt->spmm_grid = 0;
  opt->update_grid = 0;
  opt->autotune = 0;
  opt->concurrent = 1;
}

// Restores every job's stream and cooperative grid, and releases the batch's own stream and
// events, when the batch returns.
struct BatchStreams {
  std::vector<svt_ctx*> jobs;
  std::vector<cudaStream_t> saved;
  std::vector<int> saved_grid;
  std::vector<cudaEvent_t> ev;
  cudaStream_t own = nullptr;
  ~BatchStreams() {
    if (own) cudaStreamSynchronize(own);
    for (size_t i = 0; i < jobs.size(); ++i) {
      cudaStreamSynchronize(jobs[i]->st);
      jobs[i]->st = saved[i];
      jobs[i]->coop_grid = saved_grid[i];
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (own) cudaStreamDestroy(own);
  }
};

extern "C" svt_status svt_batch_solve(svt_ctx* const* jobs, int n, const double* tau, const double* delta,
                                      double eps, int max_rank, const svt_batch_options* opt, svt_result* results,
                                      svt_status* status) {
  if (!jobs || n < 1 || n > kBatchMaxJobs || !results || !status) return SVT_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!jobs[i]) return SVT_ERR_ARG;
    for (int k = 0; k < i; ++k)
      if (jobs[k] == jobs[i]) return fail(jobs[i], SVT_ERR_ARG, "a context appears twice in the batch");
  }
  svt_batch_options bo;
  svt_batch_default_options(&bo);
  if (opt) bo = *opt;
  svt_ctx* c0 = jobs[0];
  for (int i = 0; i < n; ++i) {
    svt_ctx* c = jobs[i];
    if (c->prec != c0->prec || c->bf16_mode)
      return fail(c, SVT_ERR_ARG, "a batch needs one value precision (FP64 or FP32) for all jobs");
    if (c->ds_E > 0.0 || c->noise_sigma > 0.0 || c->opt.shrink_engine != SVT_SHRINK_LANCZOS)
      return fail(c, SVT_ERR_ARG, "batched jobs run the plain iteration with the Lanczos shrink");
    if (c->coop_grid <= 0) return fail(c, SVT_ERR_ARG, "batched jobs need the cooperative orthonormalisation");
  }
  NvtxRange nv("svt_batch_solve");
  // earlier work of every job is finished first
  for (int i = 0; i < n; ++i) {
    CU(jobs[i], cudaStreamSynchronize(jobs[i]->user_st));
    CU(jobs[i], cudaStreamSynchronize(jobs[i]->st));
  }
  BatchStreams guard;
  for (int i = 0; i < n; ++i) {
    guard.jobs.push_back(jobs[i]);
    guard.saved.push_back(jobs[i]->st);
    guard.saved_grid.push_back(jobs[i]->coop_grid);
  }
  // concurrent: the batched launches run on a stream of the batch's own, every job's own work on
  // its library stream (events order the two), and each job's cooperative orthonormalisation gets
  // max(16, 2 SMs / n) CTAs so that the jobs' kernels overlap on the GPU; otherwise everything runs
  // on the first job's stream with the solo launch shapes (every iterate equals the solo one)
  const bool conc = bo.concurrent != 0 && n > 1;
  cudaStream_t bst = c0->st;
  if (conc) {
    CU(c0, cudaStreamCreateWithFlags(&guard.own, cudaStreamNonBlocking));
    bst = guard.own;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int i = 0; i < n; ++i) {
      jobs[i]->coop_grid = std::min(jobs[i]->coop_grid, std::max(16, 2 * sms / n));
      cudaEvent_t e = nullptr;
      CU(c0, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      guard.ev.push_back(e);
    }
    cudaEvent_t e = nullptr;
    CU(c0, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    guard.ev.push_back(e);   // the batch stream's event, last
  } else {
    for (int i = 0; i < n; ++i) jobs[i]->st = bst;
  }
  // the batch stream waits for the listed jobs' streams; then the jobs' streams wait for it
  auto batch_after_jobs = [&](const std::vector<int>& L) -> svt_status {
    if (!conc) return SVT_OK;
    for (int i : L) {
      CU(c0, cudaEventRecord(guard.ev[i], jobs[i]->st));
      CU(c0, cudaStreamWaitEvent(bst, guard.ev[i], 0));
    }
    return SVT_OK;
  };
  auto jobs_after_batch = [&](const std::vector<int>& L) -> svt_status {
    if (!conc) return SVT_OK;
    CU(c0, cudaEventRecord(guard.ev[n], bst));
    for (int i : L) CU(c0, cudaStreamWaitEvent(jobs[i]->st, guard.ev[n], 0));
    return SVT_OK;
  };
  const int prec = c0->prec == SVT_FP64 ? 0 : 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(c0, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(c0, SVT_ERR_CUDA, "cudaEventCreate failed");
  }
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } evg{e0, e1};
  CU(c0, cudaEventRecord(e0, bst));
  if (conc)
    for (int i = 0; i < n; ++i) CU(c0, cudaStreamWaitEvent(jobs[i]->st, e0, 0));
  std::vector<int> alive;
  std::vector<int64_t> spmm0(n), cyc0(n);
  for (int i = 0; i < n; ++i) {
    svt_ctx* c = jobs[i];
    results[i] = svt_result{};
    spmm0[i] = c->total_spmm;
    cyc0[i] = c->total_cycles;
    status[i] = svt_configure(c, tau ? tau[i] : 0.0, delta ? delta[i] : 0.0, eps, max_rank, -1);
    if (status[i] == SVT_OK) alive.push_back(i);
  }
  // tile partials of the batched update: one per 64 rows of every job
  std::vector<int> mrows(n);
  for (int i = 0; i < n; ++i) mrows[i] = (int)jobs[i]->m;
  const long long cap = upd_jobs_tiles(mrows.data(), n);
  double* partial = nullptr;
  TRY(dalloc_t(c0, &partial, (size_t)cap + 1));
  struct PartialGuard {
    svt_ctx* c;
    double* p;
    ~PartialGuard() { dfree(c, p); }
  } pg{c0, partial};
  unsigned int* berr = reinterpret_cast<unsigned int*>(partial + cap);
  CU(c0, cudaMemsetAsync(berr, 0, sizeof(unsigned int), bst));
  int64_t batch_launches = 0;
  auto drop = [&](std::vector<int>& v, int i) { v.erase(std::find(v.begin(), v.end(), i)); };
  // a launch failure leaves the batch's streams unusable: every unfinished job reports it
  auto abort_all = [&](svt_status st) {
    for (int i : alive) status[i] = st;
    return st;
  };

  // every return inside the loop is a failure of the batch's launches or streams (a job's own
  // failure is recorded in status[] and the job leaves); the jobs still running then report it
  auto run = [&]() -> svt_status {
    while (!alive.empty()) {
      // ---- shrink of every unfinished job: lockstep Lanczos cycles ----
      std::vector<ShrinkRun> R(n);
      std::vector<std::vector<double>> th(n);
      std::vector<int> sh_s(n), sh_passes(n), sh_b(n), sh_J(n), j0(n);
      std::vector<int> shrinking;
      for (int i : std::vector<int>(alive)) {
        svt_ctx* c = jobs[i];
        const int kmin = (int)std::min(c->m, c->n);
        const svt_status st = shrink_start(c, R[i], std::min(c->r + 1, kmin), c->tau, false);
        if (st != SVT_OK) {
          status[i] = st;
          drop(alive, i);
        } else {
          shrinking.push_back(i);
        }
      }
      while (!shrinking.empty()) {
        int Jmax = 0;
        for (int i : std::vector<int>(shrinking)) {
          const svt_status st = cycle_begin(jobs[i], R[i].b, R[i].J, R[i].thick, R[i].Jprev, R[i].nk, &j0[i]);
          if (st != SVT_OK) {
            status[i] = st;
            drop(shrinking, i);
            drop(alive, i);
            continue;
          }
          Jmax = std::max(Jmax, R[i].J);
        }
        for (int j = 0; j < Jmax; ++j) {
          std::vector<int> L;
          for (int i : shrinking)
            if (j >= j0[i] && j < R[i].J) L.push_back(i);
          if (L.empty()) continue;
          for (int side = 0; side < 2; ++side) {
            const bool left = side == 0;
            std::vector<SpmmJob> sj;
            for (int i : L) {
              SpmmJob J = cycle_spmm_job(jobs[i], R[i].b, j, left);
              if (bo.autotune) J.wpr = tuned_wpr(jobs[i], J, prec, left, bst);
              sj.push_back(J);
            }
            TRY(batch_after_jobs(L));
            if (launch_spmm_jobs(prec, sj.data(), (int)sj.size(), bo.spmm_grid, bst) != 1)
              return abort_all(fail(c0, SVT_ERR_CUDA, "batched sparse product launch failed: %s",
                                    cudaGetErrorString(cudaGetLastError())));
            ++batch_launches;
            TRY(jobs_after_batch(L));
            for (int i : L) {
              const int nspmm = 1;
              jobs[i]->last_spmm += nspmm;
              jobs[i]->total_spmm += nspmm;
              const svt_status st = left ? cycle_orth_left(jobs[i], R[i].b, j)
                                         : cycle_orth_right(jobs[i], R[i].b, j, R[i].J);
              if (st != SVT_OK) return abort_all(st);
            }
          }
        }
        for (int i : shrinking) {
          svt_ctx* c = jobs[i];
          const svt_status se = cycle_end(c, R[i].b, R[i].J, R[i].nk, true);
          if (se != SVT_OK) return abort_all(se);
          c->last_cycles += 1;
          c->total_cycles += 1;
          unsigned int* herr = reinterpret_cast<unsigned int*>(c->h_pin + 4 * kKMax - 1);
          CU(c, cudaMemcpyAsync(herr, c->err, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->st));
        }
        if (conc) {
          for (int i : shrinking) CU(jobs[i], cudaStreamSynchronize(jobs[i]->st));
        } else {
          CU(c0, cudaStreamSynchronize(bst));
        }
        for (int i : std::vector<int>(shrinking)) {
          svt_ctx* c = jobs[i];
          prof_harvest(c);
          svt_status st = check_err_word(c, *reinterpret_cast<unsigned int*>(c->h_pin + 4 * kKMax - 1));
          if (st == SVT_OK) {
            double defect = 0.0;
            std::memcpy(&defect, c->h_pin + 3 * kKMax + 1, sizeof defect);
            if (defect > 1e-6) c->two_corrections = true;
            bool done = false;
            st = shrink_advance(c, R[i], c->h_pin, c->h_pin + kKMax, &done, th[i], &sh_s[i], &sh_passes[i], &sh_b[i],
                                &sh_J[i]);
            if (st == SVT_OK && !done) continue;
            if (st == SVT_OK) {
              int r = 0;
              st = shrink_finish(c, c->tau, th[i], sh_s[i], sh_passes[i], sh_b[i], sh_J[i], &r);
            }
          }
          drop(shrinking, i);
          if (st != SVT_OK) {
            status[i] = st;
            drop(alive, i);
          }
        }
      }
      if (alive.empty()) break;
      // ---- fused update of every unfinished job: one launch ----
      std::vector<UpdJob> uj;
      for (int i : alive) {
        svt_ctx* c = jobs[i];
        const int nxt = 1 - c->ycur;
        UpdJob u{};
        u.row_ptr = c->row_ptr;
        u.col_idx = c->col_idx;
        u.csr_to_csc = c->csr_to_csc;
        u.M = c->Mv;
        u.y_in = ycur_csr(c);
        u.y_out = c->Ycsr[nxt];
        u.y_out_csc = c->Ycsc[nxt];
        if (prec == 0) {
          u.Ut = c->Ut;
          u.V = c->Vf;
          u.ldf = c->r;
        } else {
          u.Ut = c->Utf;
          u.V = c->Vff;
          u.ldf = c->ldf;
        }
        u.r = c->r;
        u.m = (int)c->m;
        u.delta = c->delta;
        u.res2 = c->dscal;
        uj.push_back(u);
      }
      TRY(batch_after_jobs(alive));
      if (launch_sddmm_update_jobs(prec, uj.data(), (int)uj.size(), partial, cap, berr, bo.update_grid, bst) != 2)
        return abort_all(fail(c0, SVT_ERR_CUDA, "batched update launch failed: %s",
                              cudaGetErrorString(cudaGetLastError())));
      batch_launches += 2;
      for (int i : alive)
        CU(jobs[i], cudaMemcpyAsync(jobs[i]->h_pin + 3 * kKMax, jobs[i]->dscal, sizeof(double), cudaMemcpyDeviceToHost,
                                    bst));
      CU(c0, cudaEventRecord(e1, bst));
      CU(c0, cudaEventSynchronize(e1));
      TRY(jobs_after_batch(alive));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      for (int i : std::vector<int>(alive)) {
        svt_ctx* c = jobs[i];
        const svt_status st = finish_step(c, c->r, c->h_pin[3 * kKMax], ms, nullptr);
        svt_result& res = results[i];
        res.iterations = c->k;
        res.k0 = c->k0;
        res.rank = c->r;
        res.residual = std::sqrt(c->h_pin[3 * kKMax]) / c->normF;
        res.norm2_M = c->norm2;
        res.normF_M = c->normF;
        res.ms = ms;
        res.spmm_calls = c->total_spmm - spmm0[i];
        res.lanczos_cycles = c->total_cycles - cyc0[i];
        if (st == SVT_STOPPED) {
          res.converged = 1;
          status[i] = SVT_OK;
          drop(alive, i);
        } else if (st != SVT_OK) {
          status[i] = st;
          drop(alive, i);
        } else if (c->k >= c->opt.k_max) {
          status[i] = fail(c, SVT_ERR_NOT_CONVERGED, "k_max iterations reached");
          drop(alive, i);
        }
      }
    }
    return SVT_OK;
  };
  const svt_status fatal = run();
  if (fatal != SVT_OK) return abort_all(fatal);
  c0->launches += batch_launches;
  for (int i = 0; i < n; ++i)
    if (status[i] != SVT_OK) return status[i] == SVT_ERR_NOT_CONVERGED ? SVT_ERR_NOT_CONVERGED : status[i];
  return SVT_OK;
}

extern "C" svt_status svt_solve_continuation(svt_ctx* c, const double* taus, int n_tau, double delta, double eps,
                                             int max_rank, int64_t* stage_iters, svt_result* out) {
  if (!c) return SVT_ERR_ARG;
  if (!taus || n_tau < 1) return fail(c, SVT_ERR_ARG, "need n_tau >= 1 values of tau");
  for (int i = 0; i < n_tau; ++i)
    if (!(taus[i] > 0.0) || !std::isfinite(taus[i])) return fail(c, SVT_ERR_ARG, "every tau must be positive");
  NvtxRange nv("svt_solve_continuation");
  StreamJoin join(c);
  cudaEvent_t e0, e1;
  CU(c, cudaEventCreate(&e0));
  CU(c, cudaEventCreate(&e1));
  CU(c, cudaEventRecord(e0, c->st));
  const int64_t spmm0 = c->total_spmm, cyc0 = c->total_cycles;
  svt_status s = svt_configure(c, taus[0], delta, eps, max_rank, -1);
  svt_step_info info{};
  info.residual = INFINITY;
  bool converged = false;
  int64_t total = 0;
  for (int i = 0; i < n_tau && s == SVT_OK; ++i) {
    if (i > 0) s = svt_set_tau(c, taus[i]);
    converged = false;
    int64_t it = 0;
    while (s == SVT_OK && it < c->opt.k_max) {
      ++it;
      s = svt_step(c, &info);
      if (s == SVT_STOPPED) { converged = true; s = SVT_OK; break; }
    }
    if (stage_iters) stage_iters[i] = it;
    total += it;
    if (s == SVT_OK && !converged) s = fail(c, SVT_ERR_NOT_CONVERGED, "k_max iterations reached in stage %d", i);
  }
  cudaEventRecord(e1, c->st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (out) {
    out->iterations = total;
    out->k0 = c->k0;
    out->rank = c->r;
    out->converged = converged ? 1 : 0;
    out->residual = info.residual;
    out->norm2_M = c->norm2;
    out->normF_M = c->normF;
    out->ms = ms;
    out->spmm_calls = c->total_spmm - spmm0;
    out->lanczos_cycles = c->total_cycles - cyc0;
  }
  return s;
}

extern "C" svt_status svt_get_rank(const svt_ctx* c, int* r) {
  if (!c || !r) return SVT_ERR_ARG;
  *r = c->r;
  return SVT_OK;
}

extern "C" svt_status svt_get_factors(svt_ctx* c, double* U, double* d, double* V, int capacity_r) {
  if (!c) return SVT_ERR_ARG;
  StreamJoin join(c);
  if (capacity_r < c->r) return fail(c, SVT_ERR_ARG, "capacity_r %d < rank %d", capacity_r, c->r);
  const int r = c->r;
  if (r == 0) return SVT_OK;
  const size_t pitch = sizeof(double) * std::max(c->ldu, r);
  if (U)
    CU(c, cudaMemcpy2DAsync(U, sizeof(double) * capacity_r, c->Uf, pitch, sizeof(double) * r, c->m,
                            cudaMemcpyDeviceToHost, c->st));
  if (V)
    CU(c, cudaMemcpy2DAsync(V, sizeof(double) * capacity_r, c->Vf, pitch, sizeof(double) * r, c->n,
                            cudaMemcpyDeviceToHost, c->st));
  CU(c, cudaStreamSynchronize(c->st));
  if (d) std::memcpy(d, c->d_host.data(), sizeof(double) * r);
  return SVT_OK;
}

extern "C" svt_status svt_get_Y(svt_ctx* c, double* y) {
  if (!c || !y) return SVT_ERR_ARG;
  StreamJoin join(c);
  double* tmp = nullptr;
  TRY(dalloc_t(c, &tmp, c->nnz));
  TRY(launched(c, launch_store_values(c->prec, ycur_csr(c), tmp, c->nnz, c->st)));
  CU(c, cudaMemcpyAsync(y, tmp, sizeof(double) * c->nnz, cudaMemcpyDeviceToHost, c->st));
  CU(c, cudaStreamSynchronize(c->st));
  dfree_last(c);
  return SVT_OK;
}

extern "C" svt_status svt_set_Y(svt_ctx* c, const double* y) {
  if (!c || !y) return SVT_ERR_ARG;
  StreamJoin join(c);
  double* tmp = nullptr;
  TRY(dalloc_t(c, &tmp, c->nnz));
  CU(c, cudaMemcpyAsync(tmp, y, sizeof(double) * c->nnz, cudaMemcpyHostToDevice, c->st));
  TRY(launched(c, launch_load_values(c->prec, tmp, ycur_csr(c), ycur_csc(c), c->csr_to_csc, c->nnz, c->st)));
  CU(c, cudaStreamSynchronize(c->st));
  dfree_last(c);
  return SVT_OK;
}

extern "C" svt_status svt_get_structure(svt_ctx* c, int32_t* row_ptr, int32_t* col_idx, int32_t* col_ptr,
                                        int32_t* row_idx, int32_t* csc_to_csr) {
  if (!c) return SVT_ERR_ARG;
  StreamJoin join(c);
  if (row_ptr) CU(c, cudaMemcpyAsync(row_ptr, c->row_ptr, 4 * (c->m + 1), cudaMemcpyDeviceToHost, c->st));
  if (col_idx) CU(c, cudaMemcpyAsync(col_idx, c->col_idx, 4 * c->nnz, cudaMemcpyDeviceToHost, c->st));
  if (col_ptr) CU(c, cudaMemcpyAsync(col_ptr, c->col_ptr, 4 * (c->n + 1), cudaMemcpyDeviceToHost, c->st));
  if (row_idx) CU(c, cudaMemcpyAsync(row_idx, c->row_idx, 4 * c->nnz, cudaMemcpyDeviceToHost, c->st));
  if (csc_to_csr) CU(c, cudaMemcpyAsync(csc_to_csr, c->csc_to_csr, 4 * c->nnz, cudaMemcpyDeviceToHost, c->st));
  CU(c, cudaStreamSynchronize(c->st));
  return SVT_OK;
}

extern "C" svt_status svt_shrink(svt_ctx* c, double tau, int* r_out, double* sigma) {
  if (!c) return SVT_ERR_ARG;
  StreamJoin join(c);
  if (tau <= 0) tau = c->tau;
  if (!(tau > 0)) return fail(c, SVT_ERR_ARG, "tau must be positive (or configured)");
  if (c->max_rank < 1) c->max_rank = kMaxRankCap;
  int r = 0;
  TRY(shrink_dispatch(c, tau, c->r + 1, &r));
  TRY(sync_and_check(c));
  if (r_out) *r_out = r;
  if (sigma)
    for (int i = 0; i < r; ++i) sigma[i] = c->d_host[i] + tau;
  return SVT_OK;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

extern "C" svt_status svt_apply_Y(svt_ctx* c, const double* V, int b, double* W) {
  if (!c || !V || !W) return SVT_ERR_ARG;
  StreamJoin join(c);
  if (b < 2 || b > 64 || (b & 1)) return fail(c, SVT_ERR_ARG, "b must be even, 2 <= b <= 64");
  if (!aligned16(V) || !aligned16(W)) return fail(c, SVT_ERR_ARG, "V and W must be 16-byte aligned");
  return launched(c, prof_launch(c, SVT_PROF_SPMM, spmm_bytes(c, (int)c->m, (int)c->n, b), [&] {
    return launch_spmm(c->prec, c->row_ptr, c->col_idx, ycur_csr(c), V, nullptr, W, (int)c->m, b, c->st, c->nnz);
  }));
}

extern "C" svt_status svt_apply_Yt(svt_ctx* c, const double* U, int b, double* Z) {
  if (!c || !U || !Z) return SVT_ERR_ARG;
  StreamJoin join(c);
  if (b < 2 || b > 64 || (b & 1)) return fail(c, SVT_ERR_ARG, "b must be even, 2 <= b <= 64");
  if (!aligned16(U) || !aligned16(Z)) return fail(c, SVT_ERR_ARG, "U and Z must be 16-byte aligned");
  return launched(c, prof_launch(c, SVT_PROF_SPMM_T, spmm_bytes(c, (int)c->n, (int)c->m, b), [&] {
    return launch_spmm(c->prec, c->col_ptr, c->row_idx, ycur_csc(c), U, nullptr, Z, (int)c->n, b, c->st, c->nnz);
  }));
}

extern "C" svt_status svt_sddmm_update(svt_ctx* c, const double* Ut, const double* V, int r, double delta,
                                       const double* y_in, double* y_out, double* res2) {
  if (!c || !y_in || !y_out || !res2) return SVT_ERR_ARG;
  StreamJoin join(c);
  if (r < 0 || r > 64 || (r > 0 && (!Ut || !V))) return fail(c, SVT_ERR_ARG, "need 0 <= r <= 64 and factors");
  // the kernel works in the context's value type: stage float64 in/out through the Y buffers
  const int nxt = 1 - c->ycur;
  TRY(launched(c, launch_load_values(c->prec, y_in, c->Ycsr[nxt], nullptr, nullptr, c->nnz, c->st)));
  TRY(launched(c, launch_sddmm_update(c->prec, c->row_ptr, c->col_idx, c->csr_to_csc, c->Mv, c->Ycsr[nxt],
                                      c->Ycsc[nxt], nullptr, Ut, V, nullptr, nullptr, 0, r, (int)c->m, delta,
                                      c->upd_partial, c->dscal, c->err, c->st)));
  TRY(launched(c, launch_store_values(c->prec, c->Ycsc[nxt], y_out, c->nnz, c->st)));
  CU(c, cudaMemcpyAsync(res2, c->dscal, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  return sync_and_check(c);
}

// ------------------------------------------------------------------------------------------------
// Omega sampler
// ------------------------------------------------------------------------------------------------
extern "C" svt_status svt_sample_omega(int64_t m, int64_t n, int64_t nnz, uint64_t seed, int32_t* rows,
                                       int32_t* cols, void* stream) {
  if (m < 1 || n < 1 || m >= (1LL << 31) || n >= (1LL << 31)) return fail(nullptr, SVT_ERR_ARG, "bad dimensions");
  const long long N = m * n;
  if (nnz < 0 || nnz > N || nnz >= (1LL << 31)) return fail(nullptr, SVT_ERR_ARG, "need 0 <= nnz <= m*n");
  if (nnz > 0 && (!rows || !cols)) return fail(nullptr, SVT_ERR_ARG, "rows/cols are NULL");
  if (nnz == 0) return SVT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<void*> bufs;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    for (void* p : bufs) cudaFree(p);
  };
  auto mal = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) { (void)cudaGetLastError(); return false; }
    bufs.push_back(*p);
    return true;
  };
  double margin = 8.0;
  for (int attempt = 0; attempt < 6; ++attempt, margin *= 2.0) {
    const double want = (double)nnz + margin * std::sqrt((double)nnz) + 64.0;
    uint64_t thresh;
    long long cap;
    if (want >= (double)N) {
      thresh = ~0ULL;
      cap = N;
    } else {
      double frac = want / (double)N;
      thresh = (uint64_t)(frac * 18446744073709551616.0);
      cap = (long long)(want + margin * std::sqrt(want) + 64.0);
      if (cap > N) cap = N;
    }
    unsigned long long *ck = nullptr, *cid = nullptr, *cnt = nullptr;
    void* state = nullptr;
    if (!mal((void**)&ck, sizeof(unsigned long long) * cap) || !mal((void**)&cid, sizeof(unsigned long long) * cap) ||
        !mal((void**)&cnt, sizeof(unsigned long long)) || !mal(&state, (size_t)omega_select_state_bytes())) {
      cleanup();
      return fail(nullptr, SVT_ERR_OOM, "device allocation failed in svt_sample_omega");
    }
    launch_omega_filter(seed, N, thresh, ck, cid, cap, cnt, st);
    unsigned long long count = 0;
    if (cudaMemcpyAsync(&count, cnt, sizeof count, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      (void)cudaGetLastError();
      cleanup();
      return fail(nullptr, SVT_ERR_CUDA, "svt_sample_omega: filter failed");
    }
    if ((long long)count < nnz || (long long)count > cap) {
      // too few candidates (threshold too low) or overflow: retry with a wider margin
      cleanup();
      bufs.clear();
      if ((long long)count > cap) margin = std::max(1.0, margin / 4.0);
      continue;
    }
    launch_omega_select(ck, cid, cnt, nnz, state, st);
    const long long nb = omega_compact_blocks(N);
    int32_t *bc = nullptr, *bo = nullptr, *scr = nullptr;
    unsigned int* err = nullptr;
    if (!mal((void**)&bc, sizeof(int32_t) * nb) || !mal((void**)&bo, sizeof(int32_t) * (nb + 1)) ||
        !mal((void**)&scr, sizeof(int32_t) * scan_scratch_ints(nb)) || !mal((void**)&err, sizeof(unsigned int))) {
      cleanup();
      return fail(nullptr, SVT_ERR_OOM, "device allocation failed in svt_sample_omega");
    }
    cudaMemsetAsync(err, 0, sizeof(unsigned int), st);
    launch_omega_compact(seed, N, n, state, bc, bo, scr, rows, cols, nnz, err, st);
    unsigned int e = 0;
    int32_t total = 0;
    cudaMemcpyAsync(&e, err, sizeof e, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&total, bo + nb, sizeof total, cudaMemcpyDeviceToHost, st);
    cudaError_t ce = cudaStreamSynchronize(st);
    if (ce == cudaSuccess) ce = cudaGetLastError();
    cleanup();
    if (ce != cudaSuccess) return fail(nullptr, SVT_ERR_CUDA, "svt_sample_omega: %s", cudaGetErrorString(ce));
    if (e || total != nnz) return fail(nullptr, SVT_ERR_INTERNAL, "svt_sample_omega: selected %d of %lld", total,
                                       (long long)nnz);
    return SVT_OK;
  }
  return fail(nullptr, SVT_ERR_INTERNAL, "svt_sample_omega: threshold search failed");
}

// ------------------------------------------------------------------------------------------------
// Checkpoint / resume
// ------------------------------------------------------------------------------------------------
struct StateHeader {
  uint64_t magic;
  int64_t m, n, nnz;
  int32_t prec, r, warm_cols, configured;
  int64_t k0, k;
  double tau, delta, eps, norm2;
  int32_t max_rank, flags;   // flags bit 0: two orthonormality corrections
  uint64_t rng_counter;
  double noise_sigma, noise_eps, ds_E;   // stopping rule eq. (5.10); Dantzig selector tolerance
};

static size_t state_bytes(const svt_ctx* c) {
  return sizeof(StateHeader) + c->nnz * c->vbytes + sizeof(double) * (size_t)c->r * (1 + c->m + c->m + c->n) +
         sizeof(double) * (size_t)c->n * c->warm_cols + (c->ds_E > 0.0 ? 2 * c->nnz * c->vbytes : 0);
}

extern "C" svt_status svt_save_state(svt_ctx* c, void* buf, size_t* bytes) {
  if (!c || !bytes) return SVT_ERR_ARG;
  StreamJoin join(c);
  const size_t need = state_bytes(c);
  if (!buf) { *bytes = need; return SVT_OK; }
  if (*bytes < need) return fail(c, SVT_ERR_ARG, "buffer too small (%zu < %zu)", *bytes, need);
  StateHeader h{};
  h.magic = kStateMagic; h.m = c->m; h.n = c->n; h.nnz = c->nnz; h.prec = c->prec; h.r = c->r;
  h.warm_cols = c->warm_cols; h.configured = c->configured; h.k0 = c->k0; h.k = c->k; h.tau = c->tau;
  h.delta = c->delta; h.eps = c->eps; h.norm2 = c->norm2; h.max_rank = c->max_rank; h.rng_counter = c->rng_counter;
  h.flags = (c->two_corrections ? 1 : 0) | (c->bf16_active ? 2 : 0);
  h.noise_sigma = c->noise_sigma; h.noise_eps = c->noise_eps; h.ds_E = c->ds_E;
  char* p = (char*)buf;
  std::memcpy(p, &h, sizeof h); p += sizeof h;
  CU(c, cudaMemcpyAsync(p, ycur_csr(c), c->nnz * c->vbytes, cudaMemcpyDeviceToHost, c->st)); p += c->nnz * c->vbytes;
  std::memcpy(p, c->d_host.data(), sizeof(double) * c->r); p += sizeof(double) * c->r;
  {
    // factors packed with r columns per row (the device keeps them with row stride ldu >= r)
    const size_t rb = sizeof(double) * c->r, pitch = sizeof(double) * std::max(c->ldu, c->r);
    if (c->r > 0) {
      CU(c, cudaMemcpy2DAsync(p, rb, c->Ut, pitch, rb, c->m, cudaMemcpyDeviceToHost, c->st)); p += rb * c->m;
      CU(c, cudaMemcpy2DAsync(p, rb, c->Uf, pitch, rb, c->m, cudaMemcpyDeviceToHost, c->st)); p += rb * c->m;
      CU(c, cudaMemcpy2DAsync(p, rb, c->Vf, pitch, rb, c->n, cudaMemcpyDeviceToHost, c->st)); p += rb * c->n;
    }
  }
  CU(c, cudaMemcpyAsync(p, c->Vwarm, sizeof(double) * c->n * c->warm_cols, cudaMemcpyDeviceToHost, c->st));
  p += sizeof(double) * c->n * c->warm_cols;
  if (c->ds_E > 0.0) {
    CU(c, cudaMemcpyAsync(p, c->Yp[c->ycur], c->nnz * c->vbytes, cudaMemcpyDeviceToHost, c->st)); p += c->nnz * c->vbytes;
    CU(c, cudaMemcpyAsync(p, c->Ym[c->ycur], c->nnz * c->vbytes, cudaMemcpyDeviceToHost, c->st));
  }
  CU(c, cudaStreamSynchronize(c->st));
  *bytes = need;
  return SVT_OK;
}

extern "C" svt_status svt_load_state(svt_ctx* c, const void* buf, size_t bytes) {
  if (!c || !buf) return SVT_ERR_ARG;
  StreamJoin join(c);
  if (bytes < sizeof(StateHeader)) return fail(c, SVT_ERR_ARG, "state buffer too small");
  StateHeader h;
  std::memcpy(&h, buf, sizeof h);
  if (h.magic != kStateMagic || h.m != c->m || h.n != c->n || h.nnz != c->nnz || h.prec != c->prec)
    return fail(c, SVT_ERR_ARG, "state does not match this context");
  if (h.r < 0 || h.r > kMaxRankCap || h.warm_cols < 0 || h.warm_cols > kBMax)
    return fail(c, SVT_ERR_ARG, "corrupt state");
  c->r = h.r; c->warm_cols = h.warm_cols; c->configured = h.configured != 0; c->k0 = h.k0; c->k = h.k;
  c->tau = h.tau; c->delta = h.delta; c->eps = h.eps; c->norm2 = h.norm2; c->max_rank = h.max_rank;
  c->rng_counter = h.rng_counter;
  c->two_corrections = (h.flags & 1) != 0;
  if ((h.flags & 2) && !c->bf16_mode) return fail(c, SVT_ERR_ARG, "state of a bfloat16 context");
  if (!std::isfinite(h.ds_E) || !std::isfinite(h.noise_sigma) || !std::isfinite(h.noise_eps))
    return fail(c, SVT_ERR_ARG, "corrupt state");
  if (h.ds_E > 0.0) TRY(svt_set_dantzig(c, h.ds_E));
  else c->ds_E = 0.0;
  c->configured = h.configured != 0;
  c->noise_sigma = h.noise_sigma; c->noise_eps = h.noise_eps;
  if (bytes < state_bytes(c)) return fail(c, SVT_ERR_ARG, "state buffer too small");
  const char* p = (const char*)buf + sizeof h;
  CU(c, cudaMemcpyAsync(ycur_csr(c), p, c->nnz * c->vbytes, cudaMemcpyHostToDevice, c->st)); p += c->nnz * c->vbytes;
  c->d_host.assign((const double*)p, (const double*)p + c->r); p += sizeof(double) * c->r;
  CU(c, cudaMemcpyAsync(c->Ut, p, sizeof(double) * c->m * c->r, cudaMemcpyHostToDevice, c->st)); p += sizeof(double) * c->m * c->r;
  CU(c, cudaMemcpyAsync(c->Uf, p, sizeof(double) * c->m * c->r, cudaMemcpyHostToDevice, c->st)); p += sizeof(double) * c->m * c->r;
  CU(c, cudaMemcpyAsync(c->Vf, p, sizeof(double) * c->n * c->r, cudaMemcpyHostToDevice, c->st)); p += sizeof(double) * c->n * c->r;
  c->ldu = c->r;
  CU(c, cudaMemcpyAsync(c->Vwarm, p, sizeof(double) * c->n * c->warm_cols, cudaMemcpyHostToDevice, c->st));
  p += sizeof(double) * c->n * c->warm_cols;
  if (c->ds_E > 0.0) {
    CU(c, cudaMemcpyAsync(c->Yp[c->ycur], p, c->nnz * c->vbytes, cudaMemcpyHostToDevice, c->st)); p += c->nnz * c->vbytes;
    CU(c, cudaMemcpyAsync(c->Ym[c->ycur], p, c->nnz * c->vbytes, cudaMemcpyHostToDevice, c->st));
  }
  c->bf16_active = (h.flags & 2) != 0;
  // rebuild the column-major copy of Y from the row-major values
  if (c->prec == SVT_FP64)
    TRY(launched(c, launch_gather_f64((const double*)ycur_csr(c), c->csc_to_csr, c->nnz, (double*)ycur_csc(c), c->st)));
  else {
    double* tmp = nullptr;
    TRY(dalloc_t(c, &tmp, c->nnz));
    TRY(launched(c, launch_store_values(c->prec, ycur_csr(c), tmp, c->nnz, c->st)));
    TRY(launched(c, launch_gather_f64_to_f32(tmp, c->csc_to_csr, c->nnz, (float*)ycur_csc(c), c->st)));
    CU(c, cudaStreamSynchronize(c->st));
    dfree_last(c);
    if (c->bf16_active)
      TRY(launched(c, launch_to_bf16((const float*)ycur_csr(c), (const float*)ycur_csc(c), c->Yb[c->ycur],
                                     c->Ybc[c->ycur], c->nnz, c->st)));
  }
  return sync_and_check(c);
}

// ------------------------------------------------------------------------------------------------
// Self-test of the Newton helpers
// ------------------------------------------------------------------------------------------------
extern "C" svt_status svt_selftest_math(int64_t n, const double* x, double* out, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return fail(nullptr, SVT_ERR_ARG, "svt_selftest_math: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  launch_newton_selftest(x, n, out, st);
  launch_pivot_selftest(x, n, out, st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(nullptr, SVT_ERR_CUDA, "svt_selftest_math: %s", cudaGetErrorString(e));
  return SVT_OK;
}

// ------------------------------------------------------------------------------------------------
// Failure injection
// ------------------------------------------------------------------------------------------------
static void drop_graphs(svt_ctx* c) {
  for (auto& g : c->graphs) {
    cudaGraphExecDestroy(g.exec);
    for (auto& pn : g.prof) {
      cudaEventDestroy(pn.a);
      cudaEventDestroy(pn.b);
    }
  }
  c->graphs.clear();
  for (auto& g : c->igraphs) cudaGraphExecDestroy(g.exec);
  c->igraphs.clear();
}

extern "C" svt_status svt_set_barrier_spins(svt_ctx* c, int spins) {
  if (!c) return SVT_ERR_ARG;
  if (spins < 0) return fail(c, SVT_ERR_ARG, "spins must be >= 0");
  StreamJoin join(c);
  CU(c, cudaStreamSynchronize(c->st));
  prof_harvest(c);
  // the limit is an argument of the captured kernels: later cycles are captured again
  drop_graphs(c);
  c->barrier_spins = spins > 0 ? (unsigned int)spins : kBarrierSpinLimit;
  return SVT_OK;
}

// ------------------------------------------------------------------------------------------------
// Profile
// ------------------------------------------------------------------------------------------------
extern "C" svt_status svt_set_profile(svt_ctx* c, unsigned int class_mask) {
  if (!c) return SVT_ERR_ARG;
  StreamJoin join(c);
  CU(c, cudaStreamSynchronize(c->st));
  prof_harvest(c);
  c->prof_mask = class_mask;
  for (int i = 0; i < SVT_PROF_CLASSES; ++i) {
    c->prof_ms[i] = 0.0;
    c->prof_bytes[i] = 0.0;
    c->prof_flops[i] = 0.0;
    c->prof_n[i] = 0;
  }
  return SVT_OK;
}

extern "C" svt_status svt_get_profile(svt_ctx* c, int64_t* launches, double* ms, double* bytes, double* flops) {
  if (!c) return SVT_ERR_ARG;
  StreamJoin join(c);
  CU(c, cudaStreamSynchronize(c->st));
  prof_harvest(c);
  for (int i = 0; i < SVT_PROF_CLASSES; ++i) {
    if (launches) launches[i] = c->prof_n[i];
    if (ms) ms[i] = c->prof_ms[i];
    if (bytes) bytes[i] = c->prof_bytes[i];
    if (flops) flops[i] = c->prof_flops[i];
  }
  return SVT_OK;
}

extern "C" svt_status svt_get_counters(svt_ctx* c, double* out, int n) {
  if (!c || !out || n < 0) return SVT_ERR_ARG;
  unsigned long long dc[8] = {0};
  StreamJoin join(c);
  TRY(d2h_sync(c, dc, c->dcount, sizeof dc));
  double maxdef = 0.0, maxdef1 = 0.0;
  std::memcpy(&maxdef, &dc[3], sizeof maxdef);
  std::memcpy(&maxdef1, &dc[5], sizeof maxdef1);
  const double v[11] = {(double)c->total_cycles, (double)c->total_spmm, (double)dc[0], (double)dc[1], (double)dc[2],
                        maxdef, (double)c->launches, (double)c->relaxed_shrinks, (double)dc[4], maxdef1,
                        (double)c->dl_iters};
  for (int i = 0; i < n && i < 11; ++i) out[i] = v[i];
  return SVT_OK;
}
