// Block orthonormalisation of the Lanczos partial SVD (Sec. 5.1.1: the Lanczos bidiagonalisation
// needs an orthonormal basis; here every new n x b block is made orthogonal to all previous ones
// by classical Gram-Schmidt applied twice, then orthonormalised).
//
// GB300 executes float64 with a dependent-operation latency of ~64 cycles (divide and square
// root ~650), so the sequence avoids long float64 dependency chains on a single SM:
//   1. C1 = Q^T P                      (Gram, all SMs)
//   2. P <- P - Q C1, [C2; A] = [Q, P]^T P   (one fused kernel: update + Gram of the same rows)
//      R1 = chol(A)                    (one warp; float32 reciprocal square-root seed + one float64
//                                       Newton step per pivot; columns that lost all but 1e-12 of
//                                       their norm to the projections are deflated to zero)
//   3. P <- (P - Q C2) R1^-1, E = P^T P - I  (fused; per-row forward substitution, no inverse)
//      P <- P (I - U(E)),  R2 = I + U(E)   with U(E) the upper triangle of E, halved diagonal: the
//                                       Cholesky factor of I + E to first order, so P^T P = I up to
//                                       O(|E|^2) (|E| is at rounding level after step 2 unless P was
//                                       ill conditioned; the host then adds a second step 3, giving
//                                       O(|E|^4))
// The coefficients satisfy P_in = Q (C1 + C2) + P_out R2 R1 exactly for the factors used; C1 + C2
// and R2 R1 are the entries of the projected block bidiagonal matrix.
#include "common.cuh"
#include "internal.h"

namespace svt {

static constexpr int ORTH_T = 256;
static constexpr int OB_MAXB = 32;
static constexpr int OB_MAXK = 96;
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
static constexpr int GRAM_MAXW = 128;     // (nq + 1) b <= 128
static constexpr int GRAM_MAXE = GRAM_MAXW * 32;
static constexpr int GRAM_EPT = GRAM_MAXE / ORTH_T;  // entries per thread (16)

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

// Partial Gram of rows [r0, r1) into partial[blockIdx.x * E ...).  Called by all threads.
__device__ void gram_chunk(const double* __restrict__ Q, long long q_stride, int nq, const double* __restrict__ P,
                           int b, int r0, int r1, double* __restrict__ partial) {
  __shared__ double tile[GRAM_SUB][GRAM_MAXW];
  const int W = (nq + 1) * b;
  const int E = W * b;
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
        int c = e / b, d = e - c * b;
        double s = acc[k];
        for (int rr = 0; rr < nr; ++rr) s += tile[rr][c] * tile[rr][nq * b + d];
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

__global__ void __launch_bounds__(ORTH_T)
k_gram_partial(const double* __restrict__ Q, long long q_stride, int nq, const double* __restrict__ P, int n, int b,
               int rows_per_cta, double* __restrict__ partial) {
  const int r0 = blockIdx.x * rows_per_cta;
  gram_chunk(Q, q_stride, nq, P, b, r0, min(n, r0 + rows_per_cta), partial);
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
  return 1 + gram_reduce_launch(partial, nblk, (nq + 1) * b * b, G, st, Gprev, Tcol, ldT, nq * b * b, b);
}

// ------------------------------------------------------------------------------------------------
// Fused update + partial Gram: every CTA updates the rows of its chunk, then (after a barrier, so
// its own writes are visible) forms the partial Gram of the same rows.
//   mode 0: P <- P - Q C,             partial of [Q, P]^T P   (second projection pass follows)
//   mode 1: P <- (P - Q C) R^-1,      partial of P^T P        (correction pass follows)
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(ORTH_T)
k_update_gram(int mode, const double* __restrict__ Q, long long q_stride, int nq, const double* __restrict__ C,
              const double* __restrict__ R, const double* __restrict__ dinv, double* __restrict__ P, int n, int b,
              int g, int rows_per_cta, double* __restrict__ partial) {
  __shared__ double sC[OB_MAXK * OB_MAXB];
  __shared__ double sR[OB_MAXB * OB_MAXB];
  __shared__ double sD[OB_MAXB];
  const int K = nq * b;
  for (int t = threadIdx.x; t < K * b; t += blockDim.x) sC[t] = C[t];
  if (mode == 1) {
    for (int t = threadIdx.x; t < b * b; t += blockDim.x) sR[t] = R[t];
    for (int t = threadIdx.x; t < b; t += blockDim.x) sD[t] = dinv[t];
  }
  __syncthreads();
  const int r0 = blockIdx.x * rows_per_cta;
  const int r1 = min(n, r0 + rows_per_cta);
  const int rows_per_iter = ORTH_T / g;
  const int rl = threadIdx.x / g, d = threadIdx.x - rl * g;
  const int gbase = (threadIdx.x & 31) & ~(g - 1);
  for (int ib = r0; ib < r1; ib += rows_per_iter) {   // uniform trip count for the whole CTA
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
          a0 += qrow[c] * ccol[c * b];
          a1 += qrow[c + 1] * ccol[(c + 1) * b];
          a2 += qrow[c + 2] * ccol[(c + 2) * b];
          a3 += qrow[c + 3] * ccol[(c + 3) * b];
        }
        for (; c < b; ++c) a0 += qrow[c] * ccol[c * b];
      }
      v = P[(long long)i * b + d] - ((a0 + a1) + (a2 + a3));
    }
    if (mode == 1) {
      // forward substitution: out_e = (v_e - sum_{k<e} out_k R[k][e]) * dinv[e]
      double out = 0.0;
      for (int e = 0; e < b; ++e) {
        const double oe = v * sD[e];
        const double ob = __shfl_sync(0xffffffffu, oe, gbase + e);
        if (d == e) out = ob;
        if (d > e) v -= ob * sR[e * b + d];
      }
      v = out;
    }
    if (live) P[(long long)i * b + d] = v;
  }
  __syncthreads();
  gram_chunk(Q, q_stride, mode == 0 ? nq : 0, P, b, r0, r1, partial);
}

int launch_update_gram(int mode, const double* Q, long long q_stride, int nq, const double* C, const double* R,
                       const double* dinv, double* P, int n, int b, double* partial, double* G, cudaStream_t st,
                       const double* Gprev, double* Tcol, int ldT) {
  const int g = row_group(b);
  const int rows = gram_rows_per_cta(n);
  const int nblk = (n + rows - 1) / rows;
  k_update_gram<<<nblk, ORTH_T, 0, st>>>(mode, Q, q_stride, nq, C, R, dinv, P, n, b, g, rows, partial);
  const int nqg = mode == 0 ? nq : 0;
  const int E = (nqg + 1) * b * b;
  return 1 + gram_reduce_launch(partial, nblk, E, G, st, Gprev, Tcol, ldT, nqg * b * b, b);
}

// ------------------------------------------------------------------------------------------------
// Cholesky with deflation of the b x b block A of G2 (one warp, lane t owns column t; B = compile-
// time block size so every loop has exact bounds).  Pivots: float32 reciprocal square root refined
// by one float64 Newton step (relative error ~1e-14; the float32 seed alone would leave errors of
// 1e-7 times the condition number of the Gram, which reaches 1e3 - 1e4 in Krylov blocks).
// ------------------------------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(32)
k_chol(const double* __restrict__ G1, const double* __restrict__ G2, int nq, double* __restrict__ R,
       double* __restrict__ dinv, unsigned long long* __restrict__ counters) {
  const int t = threadIdx.x;
  const int K = nq * B;
  double a[B];
#pragma unroll
  for (int i = 0; i < B; ++i) a[i] = (t < B && i <= t) ? G2[(K + i) * B + t] : 0.0;
  const double ref = (t < B) ? ((G1 && nq > 0) ? G1[(K + t) * B + t] : G2[(K + t) * B + t]) : 0.0;
  double rcol[B];
  int deflated = 0;
#pragma unroll
  for (int j = 0; j < B; ++j) {
    const double d = __shfl_sync(0xffffffffu, a[j], j);
    const double refj = __shfl_sync(0xffffffffu, ref, j);
    const bool defl = !(d > DEFLATE_REL2 * refj) || !(d > 0.0);
    double y = 0.0;
    if (!defl) {
      const double y0 = (double)rsqrtf((float)d);
      y = y0 * (1.5 - 0.5 * d * y0 * y0);  // one Newton step: relative error ~1e-14
    }
    deflated += defl ? 1 : 0;
    const double rjt = (t > j) ? a[j] * y : ((t == j) ? d * y : 0.0);
    rcol[j] = rjt;
    if (t == j) dinv[j] = y;
#pragma unroll
    for (int i = j + 1; i < B; ++i) {
      const double rji = __shfl_sync(0xffffffffu, rjt, i);
      if (t >= i) a[i] -= rji * rjt;
    }
  }
#pragma unroll
  for (int j = 0; j < B; ++j)
    if (t < B) R[j * B + t] = (j <= t) ? rcol[j] : 0.0;
  if (t == 0 && deflated && counters) atomicAdd(&counters[2], (unsigned long long)deflated);
}

// ------------------------------------------------------------------------------------------------
// P <- P (I - U(E)) with E = G3 - I; block 0 writes (I + U(E)) R1 (upper triangular) to Tdiag
// and/or Rout, and records max |E| over non-deflated columns in counters[3].
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(ORTH_T)
k_correct(const double* __restrict__ G3, const double* __restrict__ R1, double* __restrict__ Tdiag, int ldT,
          double* __restrict__ Rout, double* __restrict__ P, int n, int b, int g,
          unsigned long long* __restrict__ counters, float* __restrict__ Pf) {
  __shared__ double sU[OB_MAXB * OB_MAXB];   // U(E)
  __shared__ double sR[OB_MAXB * OB_MAXB];
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    int i = e / b, j = e - i * b;
    double x = G3[e] - (i == j ? 1.0 : 0.0);
    sU[e] = (j > i) ? x : ((i == j) ? 0.5 * x : 0.0);
    if (blockIdx.x == 0) sR[e] = R1[e];   // only block 0 forms the product with R1
  }
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
      int i = e / b, j = e - i * b;
      double v = 0.0;
      if (i <= j) {
        v = sR[i * b + j];
        for (int k = i; k <= j; ++k) v += sU[i * b + k] * sR[k * b + j];
      }
      if (Tdiag) Tdiag[i * ldT + j] = v;
      if (Rout) Rout[e] = v;
    }
    if (counters && threadIdx.x < 32) {
      double mx = 0.0;
      for (int e = threadIdx.x; e < b * b; e += 32) {
        int i = e / b, j = e - i * b;
        if (G3[i * b + i] > 0.5 && G3[j * b + j] > 0.5) mx = fmax(mx, fabs(G3[e] - (i == j ? 1.0 : 0.0)));
      }
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (threadIdx.x == 0) atomicMax(&counters[3], (unsigned long long)__double_as_longlong(mx));
    }
  }
  const int rows_per_block = ORTH_T / g;
  const int rl = threadIdx.x / g, d = threadIdx.x - rl * g;
  const int gbase = (threadIdx.x & 31) & ~(g - 1);
  // uniform trip count for every lane of the block; row values are exchanged with shuffles so
  // that no lane reads an element another lane has already overwritten
  for (int ib = blockIdx.x * rows_per_block; ib < n; ib += gridDim.x * rows_per_block) {
    const int i = ib + rl;
    const bool live = i < n && d < b;
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

}  // namespace svt
