// Dense kernels of the block Lanczos partial SVD (Sec. 5.1.1: the dominant singular triplets of
// the sparse iterate, computed from products with Y and Y^T only):
//   * Ritz-vector assembly (basis times small matrix, scaled columns)
// (the block orthonormalisation and its Gram products are in orth.cu, the projected SVD in
// jacobi.cu).  All float64: GB300 executes float64 at ~1/64 of the float32 rate, so these kernels
// spread the tall products over all SMs.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace svt {

// ------------------------------------------------------------------------------------------------
// Out (n x s) = [B_0 .. B_{nb-1}] W[:, 0:s] diag(scale)
// ------------------------------------------------------------------------------------------------
static constexpr int CMB_T = 256;

__global__ void __launch_bounds__(CMB_T)
k_basis_combine(const double* __restrict__ B, long long b_stride, int nb, int b, int n, const double* __restrict__ W,
                int ldW, int s, const double* __restrict__ scale, double* __restrict__ Out, float* __restrict__ OutF,
                int ldF, const int* __restrict__ s_dev, int ldo) {
  extern __shared__ double sW[];  // K x s
  const int K = nb * b;
  const int s_act = s_dev ? min(*s_dev, s) : s;
  for (int e = threadIdx.x; e < K * s; e += blockDim.x) {
    int k = e / s, c = e - k * s;
    sW[e] = c < s_act ? W[k * ldW + c] * (scale ? scale[c] : 1.0) : 0.0;
  }
  __syncthreads();
  const int rows_per_block = CMB_T / s;
  const int rl = threadIdx.x / s, c = threadIdx.x - rl * s;
  if (rl >= rows_per_block || c >= s_act) return;
  for (int rbase = blockIdx.x * rows_per_block; rbase < n; rbase += gridDim.x * rows_per_block) {
    const int i = rbase + rl;
    if (i >= n) continue;
    double v = 0.0;
    for (int blk = 0; blk < nb; ++blk) {
      const double* brow = B + blk * b_stride + (long long)i * b;
      const double* wcol = sW + (blk * b) * s + c;
      for (int d = 0; d < b; ++d) v = fma(brow[d], wcol[d * s], v);
    }
    Out[(long long)i * ldo + c] = v;
    if (OutF) OutF[(long long)i * ldF + c] = (float)v;
  }
}

int launch_basis_combine(const double* B, long long b_stride, int nb, int b, int n, const double* W, int ldW, int s,
                         const double* scale, double* Out, cudaStream_t st, float* OutF, int ldF, const int* s_dev,
                         int ldo) {
  if (s <= 0 || n <= 0) return 0;
  // W tiles up to 128 x 64 (64 KB) above the default 48 KB of dynamic shared memory
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_basis_combine, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 64 * (int)sizeof(double));
  });
  const int rows_per_block = CMB_T / s;
  int blocks = (int)svt_min_ll(svt_ceil_div(n, rows_per_block), 152LL * 8);
  size_t smem = (size_t)nb * b * s * sizeof(double);
  k_basis_combine<<<blocks, CMB_T, smem, st>>>(B, b_stride, nb, b, n, W, ldW, s, scale, Out, OutF, ldF, s_dev,
                                                ldo > 0 ? ldo : s);
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
    P[e] = svt_uniform_pm1(seed, (unsigned long long)e);
  }
}

int launch_random_block(double* P, int n, int b, int c0, uint64_t seed, cudaStream_t st) {
  long long total = (long long)n * b;
  int blocks = (int)svt_min_ll(svt_ceil_div(total, 256), 152LL * 8);
  if (blocks < 1) return 0;
  k_random_block<<<blocks, 256, 0, st>>>(P, n, b, c0, seed);
  return 1;
}

// ------------------------------------------------------------------------------------------------
// T[i, i] = d[i] for i < b (row-major T, leading dimension ldT).
// ------------------------------------------------------------------------------------------------
__global__ void k_set_diagonal(double* __restrict__ T, int ldT, const double* __restrict__ d, int b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < b) T[(long long)i * ldT + i] = d[i];
}

int launch_set_diagonal(double* T, int ldT, const double* d, int b, cudaStream_t st) {
  if (b <= 0) return 0;
  k_set_diagonal<<<1, 32 * ((b + 31) / 32), 0, st>>>(T, ldT, d, b);
  return 1;
}

}  // namespace svt
