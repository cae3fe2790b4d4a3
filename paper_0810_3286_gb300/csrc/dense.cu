// Dense kernels of the block Lanczos partial SVD (Sec. 5.1.1: the dominant singular triplets of
// the sparse iterate, computed from products with Y and Y^T only):
//   * Gram of a tall n x b block against the basis, split over row chunks (deterministic reduce)
//   * block update P <- (P - Q C) Rinv
//   * small b x b step of block CGS2 + Cholesky QR (with deflation of dependent columns)
//   * one-sided Jacobi SVD of the projected K x K matrix, sorted triplets, Ritz residuals
//   * Ritz-vector assembly (basis times small matrix, scaled columns)
// All float64: GB300 executes float64 at ~1/64 of the float32 rate, so these kernels keep the
// float64 work per SM small and spread the tall products over all SMs.
#include "common.cuh"
#include "internal.h"

namespace svt {

// ------------------------------------------------------------------------------------------------
// Gram: G = [Q_0 .. Q_{nq-1}, P]^T P
// ------------------------------------------------------------------------------------------------
static constexpr int GRAM_THREADS = 256;
static constexpr int GRAM_SUB = 8;        // rows staged in shared memory at a time
static constexpr int GRAM_MAXW = 128;     // (nq + 1) b <= 128
static constexpr int GRAM_MAXE = GRAM_MAXW * 32;
static constexpr int GRAM_EPT = GRAM_MAXE / GRAM_THREADS;  // entries per thread (16)

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

__global__ void __launch_bounds__(GRAM_THREADS)
k_gram_partial(const double* __restrict__ Q, long long q_stride, int nq, const double* __restrict__ P, int n, int b,
               int rows_per_cta, double* __restrict__ partial) {
  __shared__ double tile[GRAM_SUB][GRAM_MAXW];
  const int W = (nq + 1) * b;
  const int E = W * b;
  double acc[GRAM_EPT];
#pragma unroll
  for (int k = 0; k < GRAM_EPT; ++k) acc[k] = 0.0;
  const int r0 = blockIdx.x * rows_per_cta;
  const int r1 = min(n, r0 + rows_per_cta);
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
      int e = threadIdx.x + k * GRAM_THREADS;
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
    int e = threadIdx.x + k * GRAM_THREADS;
    if (e < E) partial[(long long)blockIdx.x * E + e] = acc[k];
  }
}

__global__ void k_gram_reduce(const double* __restrict__ partial, int nblk, int E, double* __restrict__ G) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double s = 0.0;
  for (int k = 0; k < nblk; ++k) s += partial[(long long)k * E + e];
  G[e] = s;
}

int launch_gram(const double* Q, long long q_stride, int nq, const double* P, int n, int b, double* partial, double* G,
                cudaStream_t st) {
  const int rows = gram_rows_per_cta(n);
  const int nblk = (n + rows - 1) / rows;
  const int E = (nq + 1) * b * b;
  k_gram_partial<<<nblk, GRAM_THREADS, 0, st>>>(Q, q_stride, nq, P, n, b, rows, partial);
  k_gram_reduce<<<(E + 255) / 256, 256, 0, st>>>(partial, nblk, E, G);
  return 2;
}

// ------------------------------------------------------------------------------------------------
// P <- (P - Q C) Rinv
// ------------------------------------------------------------------------------------------------
static constexpr int UPD_T = 256;
static constexpr int MAXB = 32;
static constexpr int MAXK = 96;

__global__ void __launch_bounds__(UPD_T)
k_block_update(const double* __restrict__ Q, long long q_stride, int nq, const double* __restrict__ C,
               const double* __restrict__ Rinv, double* __restrict__ P, int n, int b) {
  __shared__ double sC[MAXK * MAXB];
  __shared__ double sR[MAXB * MAXB];
  __shared__ double sT[UPD_T];
  const int K = nq * b;
  for (int t = threadIdx.x; t < K * b; t += blockDim.x) sC[t] = C[t];
  if (Rinv)
    for (int t = threadIdx.x; t < b * b; t += blockDim.x) sR[t] = Rinv[t];
  __syncthreads();
  const int rows_per_block = UPD_T / b;
  const int rl = threadIdx.x / b, d = threadIdx.x - rl * b;
  for (int rbase = blockIdx.x * rows_per_block; rbase < n; rbase += gridDim.x * rows_per_block) {
    const int i = rbase + rl;
    const bool live = rl < rows_per_block && i < n;
    double v = 0.0;
    if (live) {
      v = P[(long long)i * b + d];
      for (int blk = 0; blk < nq; ++blk) {
        const double* qrow = Q + blk * q_stride + (long long)i * b;
        const double* ccol = sC + blk * b * b + d;
        for (int c = 0; c < b; ++c) v -= qrow[c] * ccol[c * b];
      }
    }
    if (Rinv) {
      sT[threadIdx.x] = v;
      __syncthreads();
      if (live) {
        double w = 0.0;
        const double* trow = sT + rl * b;
        for (int c = 0; c <= d; ++c) w += trow[c] * sR[c * b + d];
        v = w;
      }
      __syncthreads();
    }
    if (live) P[(long long)i * b + d] = v;
  }
}

int launch_block_update(const double* Q, long long q_stride, int nq, const double* C, const double* Rinv, double* P,
                        int n, int b, cudaStream_t st) {
  const int rows_per_block = UPD_T / b;
  int blocks = (int)svt_min_ll(svt_ceil_div(n, rows_per_block), 152LL * 8);
  k_block_update<<<blocks, UPD_T, 0, st>>>(Q, q_stride, nq, C, Rinv, P, n, b);
  return 1;
}

// ------------------------------------------------------------------------------------------------
// Small step of CGS2 + Cholesky QR (one block of b <= 32 threads per column).
// ------------------------------------------------------------------------------------------------
static constexpr double DEFLATE_REL = 1e-24;   // squared norm ratio below which a column is dependent

// Upper Cholesky of the b x b symmetric matrix A (row-major, in shared memory) into R, with
// deflation: a pivot below DEFLATE_REL * ref[j] (or non-positive) zeroes row j of R.  Then Rinv =
// inverse of R with deflated rows replaced by unit rows, and the deflated columns of Rinv zeroed.
__device__ void chol_deflate(const double* A, const double* ref, double* R, double* Rinv, int b, unsigned int* err) {
  const int t = threadIdx.x;
  for (int j = 0; j < b; ++j) {
    __syncthreads();
    if (t == 0) {
      double d = A[j * b + j];
      for (int k = 0; k < j; ++k) d -= R[k * b + j] * R[k * b + j];
      bool defl = !(d > DEFLATE_REL * ref[j]) || !(d > 0.0);
      R[j * b + j] = defl ? 0.0 : sqrt(d);
    }
    __syncthreads();
    const double rjj = R[j * b + j];
    if (t > j && t < b) {
      double v = 0.0;
      if (rjj > 0.0) {
        v = A[j * b + t];
        for (int k = 0; k < j; ++k) v -= R[k * b + j] * R[k * b + t];
        v /= rjj;
      }
      R[j * b + t] = v;
    }
    if (t < j) R[j * b + t] = 0.0;
  }
  __syncthreads();
  // Inverse of the upper triangular matrix with deflated rows set to unit rows: column c by
  // back substitution (thread c).
  if (t < b) {
    const int c = t;
    for (int i = b - 1; i >= 0; --i) {
      double v = 0.0;
      if (i <= c) {
        double rii = R[i * b + i];
        if (rii > 0.0) {
          v = (i == c) ? 1.0 : 0.0;
          for (int k = i + 1; k <= c; ++k) v -= R[i * b + k] * Rinv[k * b + c];
          v /= rii;
        } else {
          v = (i == c) ? 1.0 : 0.0;  // unit row
        }
      }
      Rinv[i * b + c] = v;
    }
  }
  __syncthreads();
  // zero the deflated columns of Rinv (the corresponding output columns become exactly zero)
  if (t < b && !(R[t * b + t] > 0.0))
    for (int i = 0; i < b; ++i) Rinv[i * b + t] = 0.0;
  __syncthreads();
}

__global__ void k_orth_small(int mode, const double* __restrict__ G, int nq, int b, double* __restrict__ coef,
                             double* __restrict__ coef2, double* __restrict__ colnorm0, double* __restrict__ Rinv,
                             double* __restrict__ Rkeep, double* __restrict__ Tcol, int ldT, double* __restrict__ Tdiag,
                             unsigned int* err) {
  __shared__ double A[MAXB * MAXB];
  __shared__ double R[MAXB * MAXB];
  __shared__ double Ri[MAXB * MAXB];
  __shared__ double ref[MAXB];
  const int t = threadIdx.x;
  const int K = nq * b;
  if (mode == 0) {
    for (int e = t; e < K * b; e += blockDim.x) coef[e] = G[e];
    if (t < b) colnorm0[t] = G[(K + t) * b + t];
    return;
  }
  if (mode == 1) {
    // C2 and P^T P - C2^T C2 (Pythagoras; Q has orthonormal columns)
    for (int e = t; e < K * b; e += blockDim.x) coef2[e] = G[e];
    for (int e = t; e < b * b; e += blockDim.x) {
      int i = e / b, j = e - i * b;
      double v = G[(K + i) * b + j];
      for (int c = 0; c < K; ++c) v -= G[c * b + i] * G[c * b + j];
      A[e] = v;
    }
    if (t < b) ref[t] = nq > 0 ? colnorm0[t] : G[(K + t) * b + t];
    if (nq == 0 && t < b) colnorm0[t] = ref[t];
    __syncthreads();
    chol_deflate(A, ref, R, Ri, b, err);
    for (int e = t; e < b * b; e += blockDim.x) {
      Rinv[e] = Ri[e];
      Rkeep[e] = R[e];
    }
    return;
  }
  // mode 2: G = P^T P after the first Cholesky pass
  for (int e = t; e < b * b; e += blockDim.x) A[e] = G[e];
  if (t < b) ref[t] = colnorm0[t];
  __syncthreads();
  chol_deflate(A, ref, R, Ri, b, err);
  for (int e = t; e < b * b; e += blockDim.x) Rinv[e] = Ri[e];
  // Tdiag = R2 R1 (both upper triangular), Tcol = C1 + C2
  for (int e = t; e < b * b; e += blockDim.x) {
    int i = e / b, j = e - i * b;
    double v = 0.0;
    for (int k = i; k <= j; ++k) v += R[i * b + k] * Rkeep[k * b + j];
    if (Tdiag) Tdiag[i * ldT + j] = (i <= j) ? v : 0.0;
  }
  if (Tcol)
    for (int e = t; e < K * b; e += blockDim.x) {
      int i = e / b, j = e - i * b;
      Tcol[i * ldT + j] = (coef ? coef[e] : 0.0) + (coef2 ? coef2[e] : 0.0);
    }
}

int launch_orth_small(int mode, const double* G, int nq, int b, double* coef, double* coef2, double* colnorm0,
                      double* Rinv, double* Rkeep, double* Tcol, int ldT, double* Tdiag, unsigned int* err,
                      cudaStream_t st) {
  k_orth_small<<<1, 128, 0, st>>>(mode, G, nq, b, coef, coef2, colnorm0, Rinv, Rkeep, Tcol, ldT, Tdiag, err);
  return 1;
}

// ------------------------------------------------------------------------------------------------
// One-sided Jacobi SVD of the projected K x K matrix (K even, K <= 96), one CTA.
// Columns of G = T are rotated pairwise (round-robin tournament: K/2 disjoint pairs per round,
// K - 1 rounds per sweep) until every pair is orthogonal to `tol`; G = Xl diag(theta), T = G Wr^T.
// ------------------------------------------------------------------------------------------------
static constexpr int JAC_THREADS = 256;

__global__ void __launch_bounds__(JAC_THREADS)
k_small_svd(const double* __restrict__ T, int ldT, int K, const double* __restrict__ S, int b,
            double* __restrict__ theta, double* __restrict__ Xl, double* __restrict__ Wr, double* __restrict__ res,
            int nres, double tol, int max_sweeps, unsigned int* err) {
  extern __shared__ double sm[];
  double* G = sm;               // column-major: G[c * K + i]
  double* W = sm + K * K;       // column-major
  double* nrm = W + K * K;      // K
  int* order = (int*)(nrm + K); // K
  __shared__ int rotated;
  const int t = threadIdx.x;
  for (int e = t; e < K * K; e += blockDim.x) {
    int i = e / K, c = e - i * K;
    G[c * K + i] = T[i * ldT + c];
    W[c * K + i] = (i == c) ? 1.0 : 0.0;
  }
  const int npairs = K / 2;
  int tpp = JAC_THREADS / npairs;  // threads per pair, power of two <= 32
  int p2 = 1;
  while (p2 * 2 <= tpp && p2 < 32) p2 *= 2;
  tpp = p2;
  const int pair = t / tpp, gl = t - pair * tpp;
  const bool has_pair = pair < npairs;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (t == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < K - 1; ++round) {
      int p = 0, q = 0;
      if (has_pair) {
        if (pair == 0) {
          p = K - 1; q = round;
        } else {
          p = (round + pair) % (K - 1);
          q = (round - pair + (K - 1)) % (K - 1);
        }
        if (p > q) { int x = p; p = q; q = x; }
      }
      double al = 0.0, be = 0.0, ga = 0.0;
      if (has_pair) {
        const double* gp = G + p * K;
        const double* gq = G + q * K;
        for (int i = gl; i < K; i += tpp) {
          double a = gp[i], bq = gq[i];
          al += a * a; be += bq * bq; ga += a * bq;
        }
      }
      for (int o = 1; o < tpp; o <<= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o);
        be += __shfl_xor_sync(0xffffffffu, be, o);
        ga += __shfl_xor_sync(0xffffffffu, ga, o);
      }
      if (has_pair && ga != 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
        double zeta = (be - al) / (2.0 * ga);
        double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + tt * tt);
        double sn = cs * tt;
        double* gp = G + p * K;
        double* gq = G + q * K;
        double* wp = W + p * K;
        double* wq = W + q * K;
        for (int i = gl; i < K; i += tpp) {
          double a = gp[i], bq = gq[i];
          gp[i] = cs * a - sn * bq;
          gq[i] = sn * a + cs * bq;
          double wa = wp[i], wb = wq[i];
          wp[i] = cs * wa - sn * wb;
          wq[i] = sn * wa + cs * wb;
        }
        if (gl == 0) rotated = 1;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  if (sweep >= max_sweeps && t == 0) svt_set_error(err, SVT_DEVERR_JACOBI);
  // column norms and decreasing order (ties by index)
  for (int c = t; c < K; c += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < K; ++i) s += G[c * K + i] * G[c * K + i];
    nrm[c] = sqrt(s);
  }
  __syncthreads();
  for (int c = t; c < K; c += blockDim.x) {
    int rank = 0;
    for (int c2 = 0; c2 < K; ++c2)
      if (nrm[c2] > nrm[c] || (nrm[c2] == nrm[c] && c2 < c)) ++rank;
    order[rank] = c;
  }
  __syncthreads();
  for (int e = t; e < K * K; e += blockDim.x) {
    int i = e / K, k = e - i * K;  // row i, sorted triplet k
    int c = order[k];
    double th = nrm[c];
    Xl[i * K + k] = th > 0.0 ? G[c * K + i] / th : 0.0;
    Wr[i * K + k] = W[c * K + i];
  }
  for (int k = t; k < K; k += blockDim.x) theta[k] = nrm[order[k]];
  __syncthreads();
  // residual estimates ||S x_k[last b rows]|| for the first nres triplets
  for (int k = t; k < nres; k += blockDim.x) {
    double s2 = 0.0;
    if (S) {
      int c = order[k];
      double th = nrm[c];
      for (int e = 0; e < b; ++e) {
        double v = 0.0;
        for (int d = e; d < b; ++d) {
          double x = th > 0.0 ? G[c * K + (K - b + d)] / th : 0.0;
          v += S[e * b + d] * x;
        }
        s2 += v * v;
      }
    }
    res[k] = sqrt(s2);
  }
}

int launch_small_svd(const double* T, int ldT, int K, const double* S, int b, double* theta, double* Xl, double* Wr,
                     double* res, double tol, int max_sweeps, unsigned int* err, cudaStream_t st) {
  size_t smem = (size_t)(2 * K * K + K) * sizeof(double) + (size_t)K * sizeof(int);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_small_svd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((2 * MAXK * MAXK + MAXK) * sizeof(double) + MAXK * sizeof(int)));
    attr_set = true;
  }
  k_small_svd<<<1, JAC_THREADS, smem, st>>>(T, ldT, K, S, b, theta, Xl, Wr, res, K, tol, max_sweeps, err);
  return 1;
}

// ------------------------------------------------------------------------------------------------
// Out (n x s) = [B_0 .. B_{nb-1}] W[:, 0:s] diag(scale)
// ------------------------------------------------------------------------------------------------
static constexpr int CMB_T = 256;

__global__ void __launch_bounds__(CMB_T)
k_basis_combine(const double* __restrict__ B, long long b_stride, int nb, int b, int n, const double* __restrict__ W,
                int ldW, int s, const double* __restrict__ scale, double* __restrict__ Out) {
  extern __shared__ double sW[];  // K x s
  const int K = nb * b;
  for (int e = threadIdx.x; e < K * s; e += blockDim.x) {
    int k = e / s, c = e - k * s;
    sW[e] = W[k * ldW + c] * (scale ? scale[c] : 1.0);
  }
  __syncthreads();
  const int rows_per_block = CMB_T / s;
  const int rl = threadIdx.x / s, c = threadIdx.x - rl * s;
  if (rl >= rows_per_block) return;
  for (int rbase = blockIdx.x * rows_per_block; rbase < n; rbase += gridDim.x * rows_per_block) {
    const int i = rbase + rl;
    if (i >= n) continue;
    double v = 0.0;
    for (int blk = 0; blk < nb; ++blk) {
      const double* brow = B + blk * b_stride + (long long)i * b;
      const double* wcol = sW + (blk * b) * s + c;
      for (int d = 0; d < b; ++d) v += brow[d] * wcol[d * s];
    }
    Out[(long long)i * s + c] = v;
  }
}

int launch_basis_combine(const double* B, long long b_stride, int nb, int b, int n, const double* W, int ldW, int s,
                         const double* scale, double* Out, cudaStream_t st) {
  if (s <= 0 || n <= 0) return 0;
  const int rows_per_block = CMB_T / s;
  int blocks = (int)svt_min_ll(svt_ceil_div(n, rows_per_block), 152LL * 8);
  size_t smem = (size_t)nb * b * s * sizeof(double);
  k_basis_combine<<<blocks, CMB_T, smem, st>>>(B, b_stride, nb, b, n, W, ldW, s, scale, Out);
  return 1;
}

// ------------------------------------------------------------------------------------------------
// Random start columns: uniform(-1, 1) from SplitMix64 on the element index.
// ------------------------------------------------------------------------------------------------
__global__ void k_random_block(double* __restrict__ P, int n, int b, int c0, unsigned long long seed) {
  long long total = (long long)n * b;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    int c = (int)(e % b);
    if (c < c0) continue;
    unsigned long long z = seed + ((unsigned long long)e + 1ULL) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    P[e] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

int launch_random_block(double* P, int n, int b, int c0, uint64_t seed, cudaStream_t st) {
  long long total = (long long)n * b;
  int blocks = (int)svt_min_ll(svt_ceil_div(total, 256), 152LL * 8);
  if (blocks < 1) return 0;
  k_random_block<<<blocks, 256, 0, st>>>(P, n, b, c0, seed);
  return 1;
}

}  // namespace svt
