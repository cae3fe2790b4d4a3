// Block orthonormalisation of the Lanczos partial SVD (Sec. 5.1.1: the Lanczos bidiagonalisation
// needs an orthonormal basis; here every new n x b block is made orthogonal to all previous ones
// by classical Gram-Schmidt applied twice, then orthonormalised).
//
// GB300 executes float64 with a dependent-operation latency of ~64 cycles (divide and square
// root ~650), so the sequence avoids long float64 dependency chains on a single SM:
//   1. C1 = Q^T P                      (Gram, all SMs)
//   2. P <- P - Q C1, [C2; A] = [Q, P]^T P   (one fused kernel: update + Gram of the same rows)
//      R1 = chol(A)                    (one warp; reciprocal square root of each pivot seeded from
//                                       its bits through a float32 rsqrt, one float64 Newton step;
//                                       columns that lost all but 1e-12 of their norm to the
//                                       projections are deflated to zero)
//   3. P <- (P - Q C2) R1^-1, E = P^T P - I  (fused; per-row forward substitution, no inverse)
//      P <- P (I - U(E)),  R2 = I + U(E)   with U(E) the upper triangle of E, halved diagonal: the
//                                       Cholesky factor of I + E to first order, so P^T P = I up to
//                                       O(|E|^2) (|E| is at rounding level after step 2 unless P was
//                                       ill conditioned; the host then adds a second step 3, giving
//                                       O(|E|^4))
// The coefficients satisfy P_in = Q (C1 + C2) + P_out R2 R1 exactly for the factors used; C1 + C2
// and R2 R1 are the entries of the projected block bidiagonal matrix.  Of each P^T P only what is
// used is formed: its diagonal in step 1 (the deflation reference), its upper triangle in steps 2
// and 3 (the Cholesky factor and U(E) read nothing else).
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace svt {

static constexpr int ORTH_T = 256;
static constexpr int OB_MAXB = 32;
static constexpr int OB_MAXK = 128;   // nq b <= 128 previous basis columns
static constexpr double DEFLATE_REL2 = 1e-24;  // squared norm ratio below which a column is dependent

// group of lanes per row: smallest power of two >= b
static inline int row_group(int b) {
  int g = 1;
  while (g < b) g <<= 1;
  return g;
}

// ------------------------------------------------------------------------------------------------
// Gram products G = [Q_0 .. Q_{nq-1}, P]^T P, split over row chunks: every CTA owns a contiguous
// chunk of rows and writes the partial Gram of its rows; a second kernel sums the partials in a
// fixed order (deterministic).  float64 adds run at ~2 per clock per SM on GB300, so the sums are
// spread over many CTAs too.
// ------------------------------------------------------------------------------------------------
static constexpr int GRAM_SUB = 8;        // rows staged in shared memory at a time
static constexpr int GRAM_MAXW = 160;     // (nq + 1) b <= 160
static constexpr int GRAM_MAXE = GRAM_MAXW * 32;
static constexpr int GRAM_EPT = GRAM_MAXE / ORTH_T;  // entries per thread (20)

static int gram_rows_per_cta(int n) {
  int rows = (n + 2 * 152 - 1) / (2 * 152);
  rows = (rows + GRAM_SUB - 1) / GRAM_SUB * GRAM_SUB;
  return rows < GRAM_SUB ? GRAM_SUB : rows;
}

// Upper bound on the row chunks of any launch with n' <= n rows: each chunk has >= GRAM_SUB rows
// and >= ceil(n' / 304) rows, so there are at most min(ceil(n / GRAM_SUB), 304) chunks.
long long gram_partial_doubles(int n, int nq, int b) {
  long long nblk = (n + GRAM_SUB - 1) / GRAM_SUB;
  if (nblk > 2 * 152) nblk = 2 * 152;
  return nblk * (long long)(nq + 1) * b * b;
}

// Entry layout of a Gram G = [Q_0 .. Q_{nq-1}, P]^T P: the nq b x b blocks Q_k^T P row-major,
// then of P^T P only what is used: its diagonal (the squared column norms before the projection,
// `first` pass) or its upper triangle (i <= j) folded into b / 2 rows of b + 1 entries: row r
// holds (r, r .. b-1) followed by (b-1-r, b-1-r .. b-1), so both directions of the index map are
// a division by b + 1 and a comparison (b is even).
__host__ __device__ __forceinline__ int gram_entries(int nq, int b, bool first) {
  return nq * b * b + (first ? b : b * (b + 1) / 2);
}
__host__ __device__ __forceinline__ int upper_index(int i, int j, int b) {
  return i < b / 2 ? i * (b + 1) + (j - i) : (b - 1 - i) * (b + 1) + (j + 1);
}
// (i, j) of entry t of the folded upper triangle of a b x b matrix
__device__ __forceinline__ void upper_ij(int t, int b, int& i, int& j) {
  const int r = t / (b + 1), q = t - r * (b + 1);
  if (q < b - r) {
    i = r;
    j = r + q;
  } else {
    i = b - 1 - r;
    j = q - 1;
  }
}

// Partial Gram of rows [r0, r1) into partial[blockIdx.x * E ...), E = gram_entries(nq, b, first).
// Called by all threads.
__device__ void gram_chunk(const double* __restrict__ Q, long long q_stride, int nq, const double* __restrict__ P,
                           int b, int r0, int r1, double* __restrict__ partial, bool first) {
  __shared__ double tile[GRAM_SUB][GRAM_MAXW];
  const int W = (nq + 1) * b;
  const int E = gram_entries(nq, b, first);
  const int EQ = nq * b * b;
  double acc[GRAM_EPT];
#pragma unroll
  for (int k = 0; k < GRAM_EPT; ++k) acc[k] = 0.0;
  for (int rs = r0; rs < r1; rs += GRAM_SUB) {
    const int nr = min(GRAM_SUB, r1 - rs);
    for (int t = threadIdx.x; t < GRAM_SUB * W; t += blockDim.x) {
      int rr = t / W, c = t - rr * W;
      double v = 0.0;
      if (rr < nr) {
        int blk = c / b, cc = c - blk * b;
        const double* src = blk < nq ? Q + blk * q_stride : P;
        v = src[(long long)(rs + rr) * b + cc];
      }
      tile[rr][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GRAM_EPT; ++k) {
      int e = threadIdx.x + k * ORTH_T;
      if (e < E) {
        int c, d;
        if (e < EQ) {
          c = e / b;
          d = e - c * b;
        } else if (first) {
          c = nq * b + (e - EQ);
          d = e - EQ;
        } else {
          upper_ij(e - EQ, b, c, d);
          c += nq * b;
        }
        double s = acc[k];
        for (int rr = 0; rr < nr; ++rr) s = fma(tile[rr][c], tile[rr][nq * b + d], s);
        acc[k] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < GRAM_EPT; ++k) {
    int e = threadIdx.x + k * ORTH_T;
    if (e < E) partial[(long long)blockIdx.x * E + e] = acc[k];
  }
}

// First-pass Gram on the tensor cores: C1 = Q^T P from split TF32 products (each operand x =
// x_hi + x_lo with x_hi its TF32 rounding and x_lo the TF32 rounding of the remainder; x y ~
// x_hi y_hi + x_hi y_lo + x_lo y_hi, the lo x lo term dropped), float32 accumulation within the
// CTA's rows, float64 across CTAs: about float32 accuracy (~2^-22 of |Q||P| per entry) where one
// TF32 product (~2^-11) leaves the second pass's coefficients too large for blocks with little
// new direction.  The diagonal of P^T P (the deflation reference) is float64.  Same partial layout
// as gram_chunk(first = true).  C1 only decides what the first projection P <- P - Q C1 removes;
// the projection and the second pass are float64, so the Lanczos coefficients stay exact for the
// C1 used.  mma.sync m16n8k8 (row.col, tf32): per 8-row step, the warp's output tiles of 16 basis
// columns x 8 columns of P; A[m][k] = Q[row k][m], B[k][n] = P[row k][n], from the staged rows.
__device__ __forceinline__ void split_tf32(double x, unsigned int& hi, unsigned int& lo) {
  const float f = (float)x;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(f));
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(f - __uint_as_float(hi)));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned int (&a)[4], unsigned int b0,
                                         unsigned int b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int B>
__device__ void gram_chunk_tc(const double* __restrict__ Q, long long q_stride, int nq, const double* __restrict__ P,
                              int r0, int r1, double* __restrict__ partial) {
  constexpr int b = B;
  __shared__ double tile[GRAM_SUB][GRAM_MAXW];
  const int W = (nq + 1) * b;
  const int K = nq * b;
  const int E = gram_entries(nq, b, true);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int mt_n = (K + 15) / 16, nt_n = b / 8, ntiles = mt_n * nt_n;
  // output tiles per warp: at most (128 / 16) x (B / 8) tiles over the CTA's 8 warps
  constexpr int TPW = B / 8;
  static_assert(OB_MAXK / 16 * (B / 8) <= TPW * (ORTH_T / 32), "tiles per warp");
  float acc[TPW][4];
#pragma unroll
  for (int q = 0; q < TPW; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
  double dg = 0.0;   // thread d < b: squared norm of column d of P over the chunk
  for (int rs = r0; rs < r1; rs += GRAM_SUB) {
    const int nr = min(GRAM_SUB, r1 - rs);
    for (int e = threadIdx.x; e < GRAM_SUB * W; e += blockDim.x) {
      const int rr = e / W, c = e - rr * W;
      double v = 0.0;
      if (rr < nr) {
        const int blk = c / b, cc = c - blk * b;
        const double* src = blk < nq ? Q + blk * q_stride : P;
        v = src[(long long)(rs + rr) * b + cc];
      }
      tile[rr][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TPW; ++q) {
      const int tl = warp + q * nw;   // warp-uniform
      if (tl < ntiles) {
        const int m0 = (tl / nt_n) * 16, n0 = (tl % nt_n) * 8;
        const int ma = m0 + g, mb = m0 + g + 8;
        unsigned int ah[4], al[4], bh0, bl0, bh1, bl1;
        split_tf32(ma < K ? tile[t][ma] : 0.0, ah[0], al[0]);
        split_tf32(mb < K ? tile[t][mb] : 0.0, ah[1], al[1]);
        split_tf32(ma < K ? tile[t + 4][ma] : 0.0, ah[2], al[2]);
        split_tf32(mb < K ? tile[t + 4][mb] : 0.0, ah[3], al[3]);
        split_tf32(tile[t][K + n0 + g], bh0, bl0);
        split_tf32(tile[t + 4][K + n0 + g], bh1, bl1);
        // small terms first
        mma_tf32(acc[q], al, bh0, bh1);
        mma_tf32(acc[q], ah, bl0, bl1);
        mma_tf32(acc[q], ah, bh0, bh1);
      }
    }
    if (threadIdx.x < b)
      for (int rr = 0; rr < nr; ++rr) dg += tile[rr][K + threadIdx.x] * tile[rr][K + threadIdx.x];
    __syncthreads();
  }
  double* out = partial + (long long)blockIdx.x * E;
#pragma unroll
  for (int q = 0; q < TPW; ++q) {
    const int tl = warp + q * nw;
    if (tl < ntiles) {
      const int m0 = (tl / nt_n) * 16, n0 = (tl % nt_n) * 8;
      const int ma = m0 + g, mb = m0 + g + 8, n = n0 + 2 * t;
      if (ma < K) {
        out[ma * b + n] = (double)acc[q][0];
        out[ma * b + n + 1] = (double)acc[q][1];
      }
      if (mb < K) {
        out[mb * b + n] = (double)acc[q][2];
        out[mb * b + n + 1] = (double)acc[q][3];
      }
    }
  }
  if (threadIdx.x < b) out[K * b + threadIdx.x] = dg;   // the diagonal follows the K x b coefficients
}

__global__ void __launch_bounds__(ORTH_T)
k_gram_partial(const double* __restrict__ Q, long long q_stride, int nq, const double* __restrict__ P, int n, int b,
               int rows_per_cta, double* __restrict__ partial) {
  const int r0 = blockIdx.x * rows_per_cta;
  gram_chunk(Q, q_stride, nq, P, b, r0, min(n, r0 + rows_per_cta), partial, nq > 0);
}

// CTA x owns 32 entries; its four warps sum the partials k = w, w + 4, ... and combine in a fixed
// order.  The loads of a thread are issued in batches of eight before they are added, so a thread
// waits for one memory latency per batch instead of one per partial.  With Tcol given, the entries
// e < ncoef (the projection coefficients, ncoef = K b) are also written as Tcol = Gprev + G (the
// coefficients of the two projection passes), leading dimension ldT.
__global__ void __launch_bounds__(128) k_gram_reduce(const double* __restrict__ partial, int nblk, int E,
                                                     double* __restrict__ G, const double* __restrict__ Gprev,
                                                     double* __restrict__ Tcol, int ldT, int ncoef, int b) {
  __shared__ double part[4][32];
  const int el = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + el;
  double s = 0.0;
  if (e < E) {
    int k = w;
    for (; k + 28 < nblk; k += 32) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = partial[(long long)(k + 4 * u) * E + e];
      s += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    }
    for (; k < nblk; k += 4) s += partial[(long long)k * E + e];
  }
  part[w][el] = s;
  __syncthreads();
  if (w == 0 && e < E) {
    const double g = (part[0][el] + part[1][el]) + (part[2][el] + part[3][el]);
    G[e] = g;
    if (Tcol && e < ncoef) {
      const int i = e / b, j = e - i * b;
      Tcol[i * ldT + j] = (Gprev ? Gprev[e] : 0.0) + g;
    }
  }
}

static int gram_reduce_launch(const double* partial, int nblk, int E, double* G, cudaStream_t st,
                              const double* Gprev = nullptr, double* Tcol = nullptr, int ldT = 0, int ncoef = 0,
                              int b = 1) {
  k_gram_reduce<<<(E + 31) / 32, 128, 0, st>>>(partial, nblk, E, G, Gprev, Tcol, ldT, ncoef, b);
  return 1;
}

int launch_gram(const double* Q, long long q_stride, int nq, const double* P, int n, int b, double* partial, double* G,
                cudaStream_t st, const double* Gprev, double* Tcol, int ldT) {
  const int rows = gram_rows_per_cta(n);
  const int nblk = (n + rows - 1) / rows;
  k_gram_partial<<<nblk, ORTH_T, 0, st>>>(Q, q_stride, nq, P, n, b, rows, partial);
  return 1 + gram_reduce_launch(partial, nblk, gram_entries(nq, b, nq > 0), G, st, Gprev, Tcol, ldT, nq * b * b, b);
}

// ------------------------------------------------------------------------------------------------
// Fused update + partial Gram: every CTA updates the rows of its chunk, then (after a barrier, so
// its own writes are visible) forms the partial Gram of the same rows.
//   mode 0: P <- P - Q C,             partial of [Q, P]^T P   (second projection pass follows)
//   mode 1: P <- (P - Q C) R^-1,      partial of P^T P        (correction pass follows)
// ------------------------------------------------------------------------------------------------
// Rows [r0, r1) of P, g lanes per row (lane d owns column d < b):
//   mode 0: P <- P - Q C;   mode 1: P <- (P - Q C) R^-1 with dinv = 1 / diag(R)
// C (nq b x b), sR = R diag(dinv) (the columns of R scaled by the reciprocal pivots, b x b) and
// dinv (b) in shared memory.  Called by all threads of the CTA.
__device__ void update_rows(int mode, const double* __restrict__ Q, long long q_stride, int nq,
                            const double* __restrict__ sC, const double* __restrict__ sR,
                            const double* __restrict__ sD, double* __restrict__ P, int b, int g, int r0, int r1,
                            int tid0 = 0, int nthr = ORTH_T) {
  // threads [tid0, tid0 + nthr) take part (mode 0 only may leave warps out: mode 1 shuffles
  // within row groups); tid0 and nthr are multiples of 32
  const int tid = threadIdx.x - tid0;
  if (tid < 0 || tid >= nthr) return;
  const int rows_per_iter = nthr / g;
  const int rl = tid / g, d = tid - rl * g;
  const int gbase = (threadIdx.x & 31) & ~(g - 1);
  const int wrow = (tid & ~31) / g;   // first row of this warp within an iteration
  for (int ib = r0; ib < r1; ib += rows_per_iter) {
    if (ib + wrow >= r1) break;      // no row of this warp is left (warp-uniform)
    const int i = ib + rl;
    const bool live = i < r1 && d < b;
    double v = 0.0;
    if (live) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      for (int blk = 0; blk < nq; ++blk) {
        const double* qrow = Q + blk * q_stride + (long long)i * b;
        const double* ccol = sC + blk * b * b + d;
        int c = 0;
        for (; c + 3 < b; c += 4) {
          a0 = fma(qrow[c], ccol[c * b], a0);
          a1 = fma(qrow[c + 1], ccol[(c + 1) * b], a1);
          a2 = fma(qrow[c + 2], ccol[(c + 2) * b], a2);
          a3 = fma(qrow[c + 3], ccol[(c + 3) * b], a3);
        }
        for (; c < b; ++c) a0 = fma(qrow[c], ccol[c * b], a0);
      }
      v = P[(long long)i * b + d] - ((a0 + a1) + (a2 + a3));
    }
    if (mode == 1) {
      // forward substitution out_d = (v_d - sum_{e<d} out_e R[e][d]) dinv[d], written as
      // w = v dinv, w_d -= out_e (R[e][d] dinv[d]): one float64 operation per step, and lane e
      // holds out_e once the steps before it are done
      double w = d < b ? v * sD[d] : 0.0;
      for (int e = 0; e < b; ++e) {
        const double ob = __shfl_sync(0xffffffffu, w, gbase + e);
        if (d > e && d < b) w -= ob * sR[e * b + d];
      }
      v = w;
    }
    if (live) P[(long long)i * b + d] = v;
  }
}

__global__ void __launch_bounds__(ORTH_T)
k_update_gram(int mode, const double* __restrict__ Q, long long q_stride, int nq, const double* __restrict__ C,
              const double* __restrict__ R, const double* __restrict__ dinv, double* __restrict__ P, int n, int b,
              int g, int rows_per_cta, double* __restrict__ partial) {
  extern __shared__ double sm_upd[];   // C (K x b), then R diag(1 / diag(R)) (b x b), 1 / diag(R)
  double* sC = sm_upd;
  double* sR = sC + nq * b * b;
  double* sD = sR + b * b;
  const int K = nq * b;
  for (int t = threadIdx.x; t < K * b; t += blockDim.x) sC[t] = C[t];
  if (mode == 1) {
    // R diag(dinv): the columns of R scaled by the reciprocal pivots
    for (int t = threadIdx.x; t < b * b; t += blockDim.x) sR[t] = R[t] * dinv[t % b];
    for (int t = threadIdx.x; t < b; t += blockDim.x) sD[t] = dinv[t];
  }
  __syncthreads();
  const int r0 = blockIdx.x * rows_per_cta;
  const int r1 = min(n, r0 + rows_per_cta);
  update_rows(mode, Q, q_stride, nq, sC, sR, sD, P, b, g, r0, r1);
  __syncthreads();
  gram_chunk(Q, q_stride, mode == 0 ? nq : 0, P, b, r0, r1, partial, false);
}

int launch_update_gram(int mode, const double* Q, long long q_stride, int nq, const double* C, const double* R,
                       const double* dinv, double* P, int n, int b, double* partial, double* G, cudaStream_t st,
                       const double* Gprev, double* Tcol, int ldT) {
  const int g = row_group(b);
  const int rows = gram_rows_per_cta(n);
  const int nblk = (n + rows - 1) / rows;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_update_gram, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((OB_MAXK * OB_MAXB + OB_MAXB * OB_MAXB + OB_MAXB) * sizeof(double)));
  });
  const size_t smem = (size_t)(nq * b * b + b * b + b) * sizeof(double);
  k_update_gram<<<nblk, ORTH_T, smem, st>>>(mode, Q, q_stride, nq, C, R, dinv, P, n, b, g, rows, partial);
  const int nqg = mode == 0 ? nq : 0;
  const int E = gram_entries(nqg, b, false);
  return 1 + gram_reduce_launch(partial, nblk, E, G, st, Gprev, Tcol, ldT, nqg * b * b, b);
}

// ------------------------------------------------------------------------------------------------
// Cholesky with deflation of the b x b block A of G2 (one warp; B = compile-time block size so
// every loop has exact bounds).  A float64 operation of one warp occupies the SM sub-partition's
// float64 pipe for ~64 cycles whatever the number of active lanes, so the factorisation is timed
// by its count of warp-wide float64 instructions:
//   * for B <= 16 the warp is split into H = 32 / B lane groups; lane (h, c) = h B + c owns
//     column c of the rows i = h, h + H, ... (upper triangle), so a rank-1 update of the trailing
//     block costs ceil(rows / H) instructions instead of one per row;
//   * the pivot's reciprocal square root is seeded from the double's bits (exponent halved
//     exactly, 23 mantissa bits to a float32 rsqrt), refined by one Newton step in float64
//     (relative error ~1e-13, three float64 instructions); deflation is decided by integer
//     comparison of the bit patterns against 1e-24 times the column's squared norm before the
//     projections (precomputed for all columns at once).
// Columns that lost all but 1e-12 of their norm (or whose pivot is not a normal positive double
// above 2^-1021) are deflated: R's row is zero and 1 / R_jj = 0.
// ------------------------------------------------------------------------------------------------
// Reciprocal square root of a normal positive double (biased exponent 2 .. 2046) to ~1e-13: the
// seed halves the exponent exactly and takes a float32 rsqrt of the mantissa, then one step of
// Newton's iteration for 1/sqrt(d), y <- y + y (1 - d y^2) / 2, squares its relative error.
__device__ __forceinline__ double rsqrt_pivot(double d) {
  const unsigned int hi = (unsigned int)__double2hiint(d), lo = (unsigned int)__double2loint(d);
  const int E = (int)((hi >> 20) & 0x7FFu);
  const int p = 1 - (E & 1);                      // unbiased exponent odd: mantissa scaled into [2, 4)
  const int k = (E - 1023 - p) >> 1;              // d = m 4^k, m in [1, 4)
  const float m = __int_as_float((int)(((unsigned int)(127 + p) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29)));
  const unsigned int f = (unsigned int)__float_as_int(rsqrtf(m));   // in (0.5, 1]
  const int fe = (int)((f >> 23) & 0xFFu);
  const double y0 = __hiloint2double((int)(((unsigned int)(fe - 127 + 1023 - k) << 20) | ((f & 0x7FFFFFu) >> 3)),
                                     (int)((f & 7u) << 29));
  const double h = __hiloint2double((int)(hi - 0x100000u), (int)lo);   // d / 2, exact
  const double t = h * y0;
  const double u = fma(-t, y0, 0.5);              // (1 - d y0^2) / 2
  return fma(y0, u, y0);
}

// Self-test of rsqrt_pivot: out[5 i + 4] = rsqrt_pivot(x_i) (x_i a normal positive double).
__global__ void k_pivot_selftest(const double* __restrict__ x, long long n, double* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[5 * i + 4] = rsqrt_pivot(x[i]);
}

int launch_pivot_selftest(const double* x, long long n, double* out, cudaStream_t st) {
  if (n <= 0) return 0;
  const int blocks = (int)svt_min_ll(svt_ceil_div(n, 256), 152LL * 4);
  k_pivot_selftest<<<blocks, 256, 0, st>>>(x, n, out);
  return 1;
}

// One warp (lanes 0..31 of the calling warp).  G1 / G2 may have been written by other CTAs of the
// same kernel: they are read through L2.
template <int B>
__device__ __forceinline__ void chol_warp(const double* __restrict__ G1, const double* __restrict__ G2, int nq,
                                          double* __restrict__ R, double* __restrict__ dinv,
                                          unsigned long long* __restrict__ counters,
                                          const double* __restrict__ Asm = nullptr) {
  constexpr int H = B <= 16 ? 32 / B : 1;       // lane groups
  constexpr int NR = (B + H - 1) / H;           // rows per lane
  const int lane = threadIdx.x & 31;
  const int h = lane / B, c = lane - h * B;     // for B = 24 lanes 24..31 get h = 1: idle
  const bool col = h < H;
  const int K = nq * B;
  double a[NR];
#pragma unroll
  for (int s = 0; s < NR; ++s) {
    const int i = s * H + h;
    // the Gram to factor: from G2, or (Asm != NULL) the B x B row-major copy in shared memory
    a[s] = (col && i < B && i <= c) ? (Asm ? Asm[i * B + c] : __ldcg(G2 + K * B + upper_index(i, c, B))) : 0.0;
  }
  // the column's squared norm before the projections (diagonal layout of the first pass)
  const double ref = col ? ((G1 && nq > 0) ? __ldcg(G1 + K * B + c) : __ldcg(G2 + K * B + upper_index(c, c, B)))
                         : 0.0;
  const long long thr = __double_as_longlong(DEFLATE_REL2 * ref);
  int deflated = 0;
#pragma unroll
  for (int j = 0; j < B; ++j) {
    const int hj = j % H, sj = j / H;
    const double d = __shfl_sync(0xffffffffu, a[sj], hj * B + j);
    const long long tj = __shfl_sync(0xffffffffu, thr, j);
    const long long db = __double_as_longlong(d);
    const bool ok = db > tj && db >= 0x0020000000000000LL && db < 0x7FF0000000000000LL;
    const double y = ok ? rsqrt_pivot(d) : 0.0;
    deflated += ok ? 0 : 1;
    // row j of R: R_jc = A_jc y, held by the lanes of group hj in slot sj; broadcast per column
    const double rown = a[sj] * y;
    double rj = __shfl_sync(0xffffffffu, rown, (hj * B + c) & 31);
    if (!col || c < j) rj = 0.0;
    if (h == 0) R[j * B + c] = rj;
    if (lane == 0) dinv[j] = y;
    __syncwarp();
    // trailing update A_ic -= R_ji R_jc for j < i <= c (R_ji read back from R)
#pragma unroll
    for (int s = sj; s < NR; ++s) {
      const int i = s * H + h;
      if (col && i > j && i <= c) a[s] = fma(-R[j * B + i], rj, a[s]);
    }
  }
  if (lane == 0 && deflated && counters) atomicAdd(&counters[2], (unsigned long long)deflated);
}

template <int B>
__global__ void __launch_bounds__(32)
k_chol(const double* __restrict__ G1, const double* __restrict__ G2, int nq, double* __restrict__ R,
       double* __restrict__ dinv, unsigned long long* __restrict__ counters) {
  chol_warp<B>(G1, G2, nq, R, dinv, counters);
}

// ------------------------------------------------------------------------------------------------
// P <- P (I - U(E)) with E = G3 - I; (I + U(E)) R1 (upper triangular) goes to Tdiag and/or Rout,
// and max |E| over non-deflated columns to counters[3].
// ------------------------------------------------------------------------------------------------
// sU = U(E) (upper triangle of E, halved diagonal; b x b row-major), from G3 (upper-triangle
// layout) read through L2.  All threads.
__device__ __forceinline__ void correct_load_U(const double* __restrict__ G3, int b, double* __restrict__ sU) {
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    int i = e / b, j = e - i * b;
    double v = 0.0;
    if (j >= i) {
      const double x = __ldcg(G3 + upper_index(i, j, b)) - (i == j ? 1.0 : 0.0);
      v = (j > i) ? x : 0.5 * x;
    }
    sU[e] = v;
  }
}

// (I + U(E)) R1 -> Tdiag / Rout / sRout (any may be NULL).  All threads of one CTA; sU, sR1 in
// shared memory.
__device__ void correct_coefs(const double* __restrict__ sU, const double* __restrict__ sR1, int b,
                              double* __restrict__ Tdiag, int ldT, double* __restrict__ Rout,
                              double* __restrict__ sRout) {
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    int i = e / b, j = e - i * b;
    double v = 0.0;
    if (i <= j) {
      v = sR1[i * b + j];
      for (int k = i; k <= j; ++k) v += sU[i * b + k] * sR1[k * b + j];
    }
    if (Tdiag) Tdiag[i * ldT + j] = v;
    if (Rout) Rout[e] = v;
    if (sRout) sRout[e] = v;
  }
}

// max |E| over the non-deflated columns -> counters[3] (as the bits of a non-negative double, so
// atomicMax orders them), from U(E) in shared memory: E_ij = U_ij above the diagonal, E_ii =
// 2 U_ii; a deflated column has G3_ii = 0, i.e. U_ii = -1/2, and a column counts as live when
// U_ii > -1/4.  Integer operations on the bit patterns (the float64 pipe is the scarce one); NaN
// entries are ignored.  One warp (all 32 lanes).
__device__ void correct_defect(const double* __restrict__ sU, int b, unsigned long long* __restrict__ counters) {
  constexpr long long kAbs = 0x7FFFFFFFFFFFFFFFLL, kInf = 0x7FF0000000000000LL, kQuarter = 0x3FD0000000000000LL;
  const int lane = threadIdx.x & 31;
  long long off = 0, dia = 0;
  for (int e = lane; e < b * b; e += 32) {
    const int i = e / b, j = e - i * b;
    if (j < i) continue;
    const long long xi = __double_as_longlong(sU[i * b + i]), xj = __double_as_longlong(sU[j * b + j]);
    const bool li = (xi >= 0 && xi <= kInf) || (xi & kAbs) < kQuarter;
    const bool lj = (xj >= 0 && xj <= kInf) || (xj & kAbs) < kQuarter;
    const long long x = __double_as_longlong(sU[e]) & kAbs;
    if (li && lj && x <= kInf) {
      if (i == j) dia = max(dia, x);
      else off = max(off, x);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    off = max(off, __shfl_xor_sync(0xffffffffu, off, o));
    dia = max(dia, __shfl_xor_sync(0xffffffffu, dia, o));
  }
  if (lane == 0) {
    const double mx = fmax(__longlong_as_double(off), 2.0 * __longlong_as_double(dia));
    atomicMax(&counters[3], (unsigned long long)__double_as_longlong(mx));
  }
}

// Rows ib0, ib0 + step, ... (< n) of P <- P (I - U), g lanes per row; Pf: float32 copy.  The trip
// count is uniform within a warp (a warp stops once none of its rows is left); row values are
// exchanged with shuffles so that no lane reads an element another lane has already overwritten.
__device__ void correct_rows(const double* __restrict__ sU, double* __restrict__ P, int b, int g, int ib0,
                             int ib_end, int step, float* __restrict__ Pf) {
  const int rl = threadIdx.x / g, d = threadIdx.x - rl * g;
  const int gbase = (threadIdx.x & 31) & ~(g - 1);
  const int wrow = (threadIdx.x & ~31) / g;   // first row of this warp within an iteration
  for (int ib = ib0; ib < ib_end; ib += step) {
    if (ib + wrow >= ib_end) break;            // no row of this warp is left (warp-uniform)
    const int i = ib + rl;
    const bool live = i < ib_end && d < b;
    const double p = live ? P[(long long)i * b + d] : 0.0;
    double a0 = p, a1 = 0.0;
    for (int k = 0; k < b; ++k) {
      const double pk = __shfl_sync(0xffffffffu, p, gbase + k);
      if (k <= d) {
        if (k & 1) a0 -= pk * sU[k * b + d];
        else a1 -= pk * sU[k * b + d];
      }
    }
    if (live) {
      const double v = a0 + a1;
      P[(long long)i * b + d] = v;
      if (Pf) Pf[(long long)i * b + d] = (float)v;
    }
  }
}

__global__ void __launch_bounds__(ORTH_T)
k_correct(const double* __restrict__ G3, const double* __restrict__ R1, double* __restrict__ Tdiag, int ldT,
          double* __restrict__ Rout, double* __restrict__ P, int n, int b, int g,
          unsigned long long* __restrict__ counters, float* __restrict__ Pf) {
  __shared__ double sU[OB_MAXB * OB_MAXB];   // U(E)
  __shared__ double sR[OB_MAXB * OB_MAXB];
  correct_load_U(G3, b, sU);
  if (blockIdx.x == 0)   // only block 0 forms the product with R1
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) sR[e] = R1[e];
  __syncthreads();
  if (blockIdx.x == 0) correct_coefs(sU, sR, b, Tdiag, ldT, Rout, nullptr);
  if (blockIdx.x == 0 && counters && threadIdx.x < 32) correct_defect(sU, b, counters);
  const int rows_per_block = ORTH_T / g;
  correct_rows(sU, P, b, g, blockIdx.x * rows_per_block, n, gridDim.x * rows_per_block, Pf);
}

int launch_chol(const double* G1, const double* G2, int nq, int b, double* R, double* dinv,
                unsigned long long* counters, cudaStream_t st) {
  switch (b) {
    case 8: k_chol<8><<<1, 32, 0, st>>>(G1, G2, nq, R, dinv, counters); return 1;
    case 16: k_chol<16><<<1, 32, 0, st>>>(G1, G2, nq, R, dinv, counters); return 1;
    case 24: k_chol<24><<<1, 32, 0, st>>>(G1, G2, nq, R, dinv, counters); return 1;
    case 32: k_chol<32><<<1, 32, 0, st>>>(G1, G2, nq, R, dinv, counters); return 1;
    default: return 0;  // block sizes are multiples of 8 up to 32 (checked by the caller)
  }
}

int launch_correct(const double* G3, const double* R1, double* Tdiag, int ldT, double* Rout, double* P, int n, int b,
                   unsigned long long* counters, cudaStream_t st, float* Pf) {
  const int g = row_group(b);
  const int rows_per_block = ORTH_T / g;
  int blocks = (int)svt_min_ll(svt_ceil_div(n, rows_per_block), 152LL * 8);
  k_correct<<<blocks, ORTH_T, 0, st>>>(G3, R1, Tdiag, ldT, Rout, P, n, b, g, counters, Pf);
  return 1;
}

// ------------------------------------------------------------------------------------------------
// The whole orthonormalisation of one block in one cooperative launch.  The launch sequence above
// (gram, update + gram, Cholesky, update + gram, correction: 8 kernels, each a launch and a pass
// of memory latency) becomes phases of one kernel separated by grid barriers: every CTA owns a
// contiguous chunk of rows for all phases; a Gram is formed as per-CTA partials, a barrier, the
// fixed-order sums spread over all CTAs (one warp per entry), and a barrier; every CTA factors
// the b x b block itself (the same warp code on the same data gives the same R1 everywhere), so
// the Cholesky costs no barrier.  Same arithmetic and summation structure as the launch
// sequence, so the coefficients and the orthonormality level are those of the sequence.
// ------------------------------------------------------------------------------------------------
// G[e] = sum over k < nblk of partial[k E + e] for the entries e of this CTA's warps (warp-uniform
// loop); lane l sums k = l, l + 32, ... and the lanes combine by butterfly: a fixed order.  With
// Tcol, the coefficient entries e < ncoef also go to Tcol as Gprev + G.  partial and Gprev may have
// been written by other CTAs of the same kernel: read through L2.
__device__ void reduce_entries(const double* __restrict__ partial, int nblk, int E, double* __restrict__ G,
                               const double* __restrict__ Gprev, double* __restrict__ Tcol, int ldT, int ncoef,
                               int b, unsigned int* err = nullptr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int e = blockIdx.x * nw + warp; e < E; e += gridDim.x * nw) {
    double s = 0.0;
    int k = lane;
    for (; k + 96 < nblk; k += 128) {
      const double v0 = __ldcg(partial + (long long)k * E + e);
      const double v1 = __ldcg(partial + (long long)(k + 32) * E + e);
      const double v2 = __ldcg(partial + (long long)(k + 64) * E + e);
      const double v3 = __ldcg(partial + (long long)(k + 96) * E + e);
      s += (v0 + v1) + (v2 + v3);
    }
    for (; k < nblk; k += 32) s += __ldcg(partial + (long long)k * E + e);
    s = warp_sum(s);
    if (lane == 0) {
      if (err && !isfinite(s)) svt_set_error(err, SVT_DEVERR_NONFINITE);
      G[e] = s;
      if (Tcol && e < ncoef) {
        const int i = e / b, j = e - i * b;
        Tcol[i * ldT + j] = (Gprev ? __ldcg(Gprev + e) : 0.0) + s;
      }
    }
  }
}

// Tdiag = A B for upper triangular b x b A, B in shared memory (the composed diagonal block of a
// repeated pass).  All threads of one CTA.
__device__ void compose_upper(const double* __restrict__ sA, const double* __restrict__ sB, int b,
                              double* __restrict__ Tdiag, int ldT) {
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - i * b;
    double v = 0.0;
    for (int k = i; k <= j; ++k) v += sA[i * b + k] * sB[k * b + j];
    Tdiag[i * ldT + j] = v;
  }
}

// Tcol += (C3 + C4) R1 with C3, C4 the coefficient rows (K x b) of the repeated pass in G1 / G2 and
// R1 (upper triangular, shared memory) the first pass's factor: the first pass wrote Tcol = C1 + C2.
// Entries spread over all threads of the grid; G1, G2 and Tcol were written by other CTAs of the
// same kernel and are read through L2.
__device__ void compose_coefs(const double* __restrict__ G1, const double* __restrict__ G2,
                              const double* __restrict__ sR1, int K, int b, double* __restrict__ Tcol, int ldT) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * b; e += gridDim.x * blockDim.x) {
    const int i = e / b, j = e - i * b;
    double v = 0.0;
    for (int k = 0; k <= j; ++k) v += (__ldcg(G1 + i * b + k) + __ldcg(G2 + i * b + k)) * sR1[k * b + j];
    Tcol[i * ldT + j] = __ldcg(Tcol + i * ldT + j) + v;
  }
}

struct OrthCoopArgs {
  double* P;                  // rows x b, orthonormalised in place
  const double* Q;            // nq blocks of rows x b, q_stride apart
  long long q_stride;
  int nq, n, g, rpc;          // rpc: rows per CTA
  double *partial, *G1, *G2, *G3;
  double *Tcol, *Tdiag;       // coefficient outputs (may be NULL), leading dimension ldT
  int ldT;
  float* Pf;                  // float32 copy of the result (may be NULL)
  unsigned long long* counters;
  unsigned int* err;
  unsigned int* bar;          // grid barrier word
  int twoc;                   // second first-order correction
  double repass;              // defect of the first pass above which the whole pass is repeated
                              // (<= 0: never)
  unsigned int spin_limit;    // polls of a barrier wait before it gives up
  int tc;                     // first-pass Gram C1 = Q^T P on the tensor cores (TF32)
};

static constexpr size_t orth_coop_smem(int B) {
  return (size_t)(OB_MAXK * B + 4 * B * B + B) * sizeof(double);
}

// max |E| over the live columns of U(E) in shared memory (the quantity correct_defect records),
// returned to every lane of the calling warp.  Integer operations on the bit patterns.
__device__ double defect_warp(const double* __restrict__ sU, int b) {
  constexpr long long kAbs = 0x7FFFFFFFFFFFFFFFLL, kInf = 0x7FF0000000000000LL, kQuarter = 0x3FD0000000000000LL;
  const int lane = threadIdx.x & 31;
  long long off = 0, dia = 0;
  for (int e = lane; e < b * b; e += 32) {
    const int i = e / b, j = e - i * b;
    if (j < i) continue;
    const long long xi = __double_as_longlong(sU[i * b + i]), xj = __double_as_longlong(sU[j * b + j]);
    const bool li = (xi >= 0 && xi <= kInf) || (xi & kAbs) < kQuarter;
    const bool lj = (xj >= 0 && xj <= kInf) || (xj & kAbs) < kQuarter;
    const long long x = __double_as_longlong(sU[e]) & kAbs;
    if (li && lj && x <= kInf) {
      if (i == j) dia = max(dia, x);
      else off = max(off, x);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    off = max(off, __shfl_xor_sync(0xffffffffu, off, o));
    dia = max(dia, __shfl_xor_sync(0xffffffffu, dia, o));
  }
  return fmax(__longlong_as_double(off), 2.0 * __longlong_as_double(dia));
}

#define SVT_BARRIER_OR_RETURN()                     \
  do {                                              \
    if (!svt_grid_barrier(a.bar, a.err, a.spin_limit)) return;   \
  } while (0)

template <int B>
__global__ void __launch_bounds__(ORTH_T, 2) k_orth_coop(OrthCoopArgs a) {
  extern __shared__ double sm_orth[];
  double* sC = sm_orth;                 // K x B coefficients (C1, then C2)
  double* sR = sC + OB_MAXK * B;        // R of the current pass
  double* sU = sR + B * B;              // U(E)
  double* sR2 = sU + B * B;             // R diag(1 / diag(R)); then (I + U(E)) R of a first correction
  double* sD = sR2 + B * B;             // 1 / diag(R)
  double* sR1 = sD + B;                 // R of the first pass, kept when the pass is repeated
  __shared__ int s_repass;
  // a barrier of an earlier cooperative kernel gave up: the whole grid returns at once
  if (*(volatile unsigned int*)a.err & SVT_DEVERR_BARRIER) return;
  const int K = a.nq * B;
  const int nb = gridDim.x;
  const int r0 = blockIdx.x * a.rpc;
  const int r1 = min(a.n, r0 + a.rpc);
  const int step = ORTH_T / a.g;
  // Pass 0 is block CGS2 + Cholesky QR.  When its result is far from orthonormal (a block with
  // nearly dependent columns: Cholesky QR loses orthogonality as cond(P)^2 eps, and a column that
  // lost most of its norm to the projections keeps components along Q of eps / (its norm ratio)),
  // pass 1 repeats CGS2 + Cholesky QR on that result (the Cholesky QR2 remedy), and the
  // coefficients compose: P_in = Q (C_a + C_b R_a) + P_out (R_b R_a).
  for (int pass = 0; pass < 2; ++pass) {
    // the first pass may take its C1 from the tensor cores; a repeated pass is float64 throughout
    const bool tcp = a.tc && pass == 0 && a.nq > 0;
    if (a.nq > 0) {
      // C1 = Q^T P (with the diagonal of P^T P): TF32 tensor cores or float64
      if (tcp) gram_chunk_tc<B>(a.Q, a.q_stride, a.nq, a.P, r0, r1, a.partial);
      else gram_chunk(a.Q, a.q_stride, a.nq, a.P, B, r0, r1, a.partial, true);
      SVT_BARRIER_OR_RETURN();
      reduce_entries(a.partial, nb, gram_entries(a.nq, B, true), a.G1, nullptr, nullptr, 0, 0, B, a.err);
      SVT_BARRIER_OR_RETURN();
      // P <- P - Q C1; [C2; A] = [Q, P]^T P; coefficients C1 + C2 -> Tcol (first pass)
      for (int t = threadIdx.x; t < K * B; t += blockDim.x) sC[t] = __ldcg(a.G1 + t);
      __syncthreads();
      update_rows(0, a.Q, a.q_stride, a.nq, sC, nullptr, nullptr, a.P, B, a.g, r0, r1);
      __syncthreads();
      gram_chunk(a.Q, a.q_stride, a.nq, a.P, B, r0, r1, a.partial, false);
      SVT_BARRIER_OR_RETURN();
      reduce_entries(a.partial, nb, gram_entries(a.nq, B, false), a.G2, a.G1, pass == 0 ? a.Tcol : nullptr, a.ldT,
                     K * B, B);
      SVT_BARRIER_OR_RETURN();
    } else {
      gram_chunk(nullptr, 0, 0, a.P, B, r0, r1, a.partial, false);
      SVT_BARRIER_OR_RETURN();
      reduce_entries(a.partial, nb, gram_entries(0, B, false), a.G2, nullptr, nullptr, 0, 0, B, a.err);
      SVT_BARRIER_OR_RETURN();
    }
    if (tcp) {
      // After a tensor-core C1 the second-pass coefficients C2 are of the size of its error (float32
      // accumulation, ~1e-6 of |P|), too large to leave out of the Gram of the twice-projected block:
      // A <- A - C2^T C2 (Pythagoras, Q orthonormal), in float64.  A block that brings little new
      // direction (a thick restart's residual block, |P''| ~ 1e-10 |P|) has pivots far below
      // |C2|^2, so the subtraction must not add more than float64 rounding of |C2|^2; float32
      // products here deflated such columns.  A goes to sU, which is free until the corrections.
      for (int t = threadIdx.x; t < K * B; t += blockDim.x) sC[t] = __ldcg(a.G2 + t);
      __syncthreads();
      for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
        const int i = e / B, j = e - i * B;
        if (i <= j) {
          double acc = 0.0;
          for (int m = 0; m < K; ++m) acc = fma(sC[m * B + i], sC[m * B + j], acc);
          sU[e] = __ldcg(a.G2 + K * B + upper_index(i, j, B)) - acc;
        }
      }
      __syncthreads();
    }
    // R = chol(A) in every CTA, by warp 0, while warps 1.. project P <- P - Q C2; then
    // P <- P R^-1 (forward substitution) by the whole CTA; E = P^T P - I
    if (threadIdx.x < 32) {
      // deflated columns are counted in the first pass (a repeated pass sees them again as zeros)
      chol_warp<B>(a.nq > 0 ? a.G1 : nullptr, a.G2, a.nq, sR, sD,
                   (blockIdx.x == 0 && pass == 0) ? a.counters : nullptr, tcp ? sU : nullptr);
    } else if (a.nq > 0) {
      if (!tcp)
        for (int t = threadIdx.x - 32; t < K * B; t += blockDim.x - 32) sC[t] = __ldcg(a.G2 + t);
      asm volatile("bar.sync 1, %0;" ::"r"(ORTH_T - 32));   // warps 1.. only
      update_rows(0, a.Q, a.q_stride, a.nq, sC, nullptr, nullptr, a.P, B, a.g, r0, r1, 32, ORTH_T - 32);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < B * B; t += blockDim.x) sR2[t] = sR[t] * sD[t % B];
    __syncthreads();
    update_rows(1, nullptr, 0, 0, nullptr, sR2, sD, a.P, B, a.g, r0, r1);
    if (pass == 0 && a.repass > 0.0) {
      // Deflated columns (zero rows of R: numerically dependent on Q and on the block's other
      // columns) are replaced by fresh random directions, and the pass is repeated to make them
      // orthonormal to Q and to the rest of the block: the block keeps its width, so the Krylov
      // space keeps growing (block Lanczos breakdown).  A deflated column has no coefficient in
      // P_in = Q C_a + P R_a, so the relation still holds.  The seed comes from R, identical in
      // every CTA and different from block to block.
      int ndef = 0;
      for (int j = 0; j < B; ++j) ndef += sD[j] == 0.0 ? 1 : 0;
      if (ndef > 0) {
        __syncthreads();   // the substitution above wrote these rows
        const unsigned long long seed =
            (unsigned long long)__double_as_longlong(sR[0]) ^ ((unsigned long long)a.nq << 40) ^ (unsigned long long)a.n;
        for (int e = threadIdx.x; e < (r1 - r0) * B; e += blockDim.x) {
          const int i = r0 + e / B, j = e - (e / B) * B;
          if (sD[j] == 0.0) a.P[(long long)i * B + j] = svt_uniform_pm1(seed, (unsigned long long)i * B + j);
        }
        for (int t = threadIdx.x; t < B * B; t += blockDim.x) sR1[t] = sR[t];
        if (threadIdx.x == 0 && blockIdx.x == 0 && a.counters) atomicAdd(&a.counters[4], 1ull);
        __syncthreads();
        continue;
      }
    }
    __syncthreads();
    gram_chunk(nullptr, 0, 0, a.P, B, r0, r1, a.partial, false);
    SVT_BARRIER_OR_RETURN();
    reduce_entries(a.partial, nb, gram_entries(0, B, false), a.G3, nullptr, nullptr, 0, 0, B);
    SVT_BARRIER_OR_RETURN();
    correct_load_U(a.G3, B, sU);
    __syncthreads();
    if (pass == 0 && a.repass > 0.0) {
      // every CTA takes the same decision from the same G3
      if (threadIdx.x < 32) {
        const double d0 = defect_warp(sU, B);
        if (threadIdx.x == 0) {
          s_repass = d0 > a.repass ? 1 : 0;
          if (s_repass && blockIdx.x == 0 && a.counters) {
            atomicAdd(&a.counters[4], 1ull);
            atomicMax(&a.counters[5], (unsigned long long)__double_as_longlong(d0));
          }
        }
      }
      __syncthreads();
      if (s_repass) {
        for (int t = threadIdx.x; t < B * B; t += blockDim.x) sR1[t] = sR[t];
        __syncthreads();
        continue;
      }
    }
    const bool second = pass == 1;
    if (!a.twoc) {
      // the coefficients by the last CTA, the defect by the last warp of CTA 0: off the rows'
      // critical path where a CTA has fewer rows than warps
      if (blockIdx.x == nb - 1) {
        if (!second) {
          correct_coefs(sU, sR, B, a.Tdiag, a.ldT, nullptr, nullptr);
        } else if (a.Tdiag) {
          correct_coefs(sU, sR, B, nullptr, 0, nullptr, sR2);
          __syncthreads();
          compose_upper(sR2, sR1, B, a.Tdiag, a.ldT);
        }
      }
      if (blockIdx.x == 0 && a.counters && threadIdx.x >= ORTH_T - 32) correct_defect(sU, B, a.counters);
      if (second && a.Tcol && a.nq > 0) compose_coefs(a.G1, a.G2, sR1, K, B, a.Tcol, a.ldT);
      correct_rows(sU, a.P, B, a.g, r0, r1, step, a.Pf);
      return;
    }
    // two first-order corrections: P^T P = I up to O(|E|^4)
    correct_coefs(sU, sR, B, nullptr, 0, nullptr, sR2);
    if (blockIdx.x == 0 && a.counters && threadIdx.x >= ORTH_T - 32) correct_defect(sU, B, a.counters);
    correct_rows(sU, a.P, B, a.g, r0, r1, step, nullptr);
    __syncthreads();
    gram_chunk(nullptr, 0, 0, a.P, B, r0, r1, a.partial, false);
    SVT_BARRIER_OR_RETURN();
    reduce_entries(a.partial, nb, gram_entries(0, B, false), a.G3, nullptr, nullptr, 0, 0, B);
    SVT_BARRIER_OR_RETURN();
    correct_load_U(a.G3, B, sU);
    __syncthreads();
    if (blockIdx.x == nb - 1) {
      if (!second) {
        correct_coefs(sU, sR2, B, a.Tdiag, a.ldT, nullptr, nullptr);
      } else if (a.Tdiag) {
        correct_coefs(sU, sR2, B, nullptr, 0, nullptr, sR);
        __syncthreads();
        compose_upper(sR, sR1, B, a.Tdiag, a.ldT);
      }
    }
    if (second && a.Tcol && a.nq > 0) compose_coefs(a.G1, a.G2, sR1, K, B, a.Tcol, a.ldT);
    correct_rows(sU, a.P, B, a.g, r0, r1, step, a.Pf);
    return;
  }
}

#undef SVT_BARRIER_OR_RETURN

template <int B>
static bool orth_coop_attr() {
  return cudaFuncSetAttribute(k_orth_coop<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)orth_coop_smem(B)) == cudaSuccess;
}

template <int B>
static int orth_coop_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_orth_coop<B>, ORTH_T, orth_coop_smem(B)) != cudaSuccess)
    return 0;
  return nb;
}

// Largest co-resident grid of the cooperative kernel for every block size (the same bound is
// used for all, the smallest of them), capped at two CTAs per SM.  0 if unavailable.
int orth_coop_init() {
  // once per process (contexts may be created from several threads)
  static std::once_flag once;
  static int grid = 0;
  std::call_once(once, [] {
    int dev = 0, sms = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
      (void)cudaGetLastError();
      return;
    }
    if (!orth_coop_attr<8>() || !orth_coop_attr<16>() || !orth_coop_attr<24>() || !orth_coop_attr<32>()) {
      (void)cudaGetLastError();
      return;
    }
    int bps = std::min(std::min(orth_coop_blocks_per_sm<8>(), orth_coop_blocks_per_sm<16>()),
                       std::min(orth_coop_blocks_per_sm<24>(), orth_coop_blocks_per_sm<32>()));
    bps = std::min(bps, 2);
    grid = bps * sms;
  });
  return grid;
}

int launch_orth_coop(double* P, const double* Q, long long q_stride, int nq, int n, int b, double* partial,
                     double* G1, double* G2, double* G3, double* Tcol, double* Tdiag, int ldT, float* Pf,
                     unsigned long long* counters, unsigned int* err, void* bar, int twoc, int max_grid,
                     cudaStream_t st, double repass, unsigned int spin_limit, int tc) {
  const int gmax = std::min(orth_coop_init(), max_grid);
  if (gmax <= 0 || n <= 0) return 0;
  // at least GRAM_SUB rows per CTA, and at most gmax CTAs
  int rpc = std::max(GRAM_SUB, (n + gmax - 1) / gmax);
  const int grid = (n + rpc - 1) / rpc;
  OrthCoopArgs a;
  a.P = P; a.Q = Q; a.q_stride = q_stride; a.nq = nq; a.n = n; a.g = row_group(b); a.rpc = rpc;
  a.partial = partial; a.G1 = G1; a.G2 = G2; a.G3 = G3;
  a.Tcol = Tcol; a.Tdiag = Tdiag; a.ldT = ldT; a.Pf = Pf;
  a.counters = counters; a.err = err; a.bar = static_cast<unsigned int*>(bar); a.twoc = twoc;
  a.repass = repass;
  a.spin_limit = spin_limit;
  a.tc = tc;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(ORTH_T);
  cfg.dynamicSmemBytes = orth_coop_smem(b);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  switch (b) {
    case 8: e = cudaLaunchKernelEx(&cfg, k_orth_coop<8>, a); break;
    case 16: e = cudaLaunchKernelEx(&cfg, k_orth_coop<16>, a); break;
    case 24: e = cudaLaunchKernelEx(&cfg, k_orth_coop<24>, a); break;
    case 32: e = cudaLaunchKernelEx(&cfg, k_orth_coop<32>, a); break;
    default: return 0;
  }
  return e == cudaSuccess ? 1 : 0;
}

}  // namespace svt
