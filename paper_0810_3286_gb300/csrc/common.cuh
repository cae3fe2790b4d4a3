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
  SVT_DEVERR_BARRIER = 1u << 6,       // a grid barrier of a cooperative kernel gave up waiting
};

__device__ __forceinline__ void svt_set_error(unsigned int* err, unsigned int bit) {
  if (err) atomicOr(err, bit);
}

// Fused multiply-add in the argument type (float: fmaf, double: fma), so that templated kernels
// never promote a float32 accumulation to float64.
__device__ __forceinline__ float fmac(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmac(double a, double b, double c) { return fma(a, b, c); }

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

// Grid-wide barrier of a cooperative launch (all CTAs co-resident), on one 32-bit word: CTA 0 adds
// 2^31 - (nb - 1) and every other CTA adds 1, so one complete barrier changes the word by exactly
// 2^31 and flips its top bit once, while no partial sum of the arrivals reaches it; a CTA waits
// until the top bit differs from the one it saw on arrival.  One atomic per CTA, no reset between
// barriers or launches.  The wait is bounded: after kBarrierSpinLimit polls (far beyond any
// legitimate wait; a smaller limit can be passed to exercise the path) the CTA records
// SVT_DEVERR_BARRIER and the call returns false; the caller then returns from the kernel, and the
// host zeroes the word before the next launch.
static constexpr unsigned int kBarrierSpinLimit = 1u << 22;

__device__ __forceinline__ bool svt_grid_barrier(unsigned int* word, unsigned int* err,
                                                 unsigned int spin_limit = kBarrierSpinLimit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int inc = (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) ? 0x80000000u - (nb - 1u) : 1u;
    __threadfence();
    const unsigned int old = atomicAdd(word, inc);
    volatile unsigned int* vw = word;
    unsigned int it = 0;
    while (((*vw ^ old) & 0x80000000u) == 0u) {
      if (++it > spin_limit) {
        ok = 0;
        svt_set_error(err, SVT_DEVERR_BARRIER);
        break;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Uniform(-1, 1) from output number index + 1 of SplitMix64 started at `seed` (Steele, Lea & Flood
// 2014): the random start columns of the Lanczos blocks and fresh directions for deflated ones.
__device__ __forceinline__ double svt_uniform_pm1(unsigned long long seed, unsigned long long index) {
  unsigned long long z = seed + (index + 1ULL) * 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

static inline int svt_ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
static inline long long svt_min_ll(long long a, long long b) { return a < b ? a : b; }
