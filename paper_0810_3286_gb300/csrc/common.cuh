// Shared device helpers and launch constants of libsvt (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define SVT_NUM_SMS_HINT 152

// Device error word bits (set by kernels, read by the host at synchronisation points).
enum : unsigned int {
  SVT_DEVERR_INDEX_RANGE = 1u << 0,   // an input (row, col) pair lies outside [0,m) x [0,n)
  SVT_DEVERR_DUPLICATE = 1u << 1,     // the same (row, col) pair appears twice
  SVT_DEVERR_NONFINITE = 1u << 2,     // a NaN or Inf reached a reduction
  SVT_DEVERR_CHOL = 1u << 3,          // a Gram matrix was not numerically positive definite
  SVT_DEVERR_CAPACITY = 1u << 4,      // a device buffer would have overflowed (write skipped)
  SVT_DEVERR_JACOBI = 1u << 5,        // the small Jacobi SVD hit its sweep limit
};

__device__ __forceinline__ void svt_set_error(unsigned int* err, unsigned int bit) {
  if (err) atomicOr(err, bit);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

static inline int svt_ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
static inline long long svt_min_ll(long long a, long long b) { return a < b ? a : b; }
