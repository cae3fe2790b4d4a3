// Per-iteration kernels that stream Omega: the two sparse products of the Lanczos partial SVD
// (Y V and Y^T U, Sec. 2.2 / Sec. 5.1.1) and the fused X-on-Omega + dual step + residual of
// Algorithm 1 (Sec. 5.1.5; residual of eq. (5.5)).
#include "common.cuh"
#include "internal.h"

namespace svt {

// ------------------------------------------------------------------------------------------------
// SpMM over compressed segments: Out[s, :] = sum_{p in segment s} val[p] * X[idx[p], :].
//
// One warp per segment (row of Y for Y V, column of Y for Y^T U using the column-major copy of
// the values).  A group of G lanes covers one sampled entry, each lane two adjacent columns of
// the b-wide dense row (one 16-byte load of X), so 32/G entries are in flight per warp step and
// every gathered row of X is read as whole 16-byte sectors.  Partial sums of the 32/G groups are
// combined with xor shuffles (fixed order: deterministic).
// ------------------------------------------------------------------------------------------------
template <typename VT, typename AT>
__global__ void __launch_bounds__(256) k_spmm(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                              const VT* __restrict__ val, const double* __restrict__ X,
                                              double* __restrict__ Out, int n_out, int b, int G) {
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  const int gl = lane & (G - 1);         // lane inside its group
  const int grp = lane / G;              // group index
  const int ngrp = 32 / G;
  const int c = 2 * gl;                  // first of the two columns of this lane
  const bool active_col = c < b;
  for (int s = blockIdx.x * warps + (threadIdx.x >> 5); s < n_out; s += gridDim.x * warps) {
    const int a = ptr[s], e = ptr[s + 1];
    AT acc0 = 0, acc1 = 0;
    int p = a + grp;
    // two entries per group per iteration for memory-level parallelism
    for (; p + ngrp < e; p += 2 * ngrp) {
      int j0 = __ldg(idx + p), j1 = __ldg(idx + p + ngrp);
      AT v0 = (AT)__ldg(val + p), v1 = (AT)__ldg(val + p + ngrp);
      if (active_col) {
        double2 x0 = __ldg(reinterpret_cast<const double2*>(X + (long long)j0 * b + c));
        double2 x1 = __ldg(reinterpret_cast<const double2*>(X + (long long)j1 * b + c));
        acc0 += v0 * (AT)x0.x; acc1 += v0 * (AT)x0.y;
        acc0 += v1 * (AT)x1.x; acc1 += v1 * (AT)x1.y;
      }
    }
    if (p < e) {
      int j0 = __ldg(idx + p);
      AT v0 = (AT)__ldg(val + p);
      if (active_col) {
        double2 x0 = __ldg(reinterpret_cast<const double2*>(X + (long long)j0 * b + c));
        acc0 += v0 * (AT)x0.x; acc1 += v0 * (AT)x0.y;
      }
    }
    for (int o = G; o < 32; o <<= 1) {
      acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
      acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
    }
    if (grp == 0 && active_col) {
      double2 w;
      w.x = (double)acc0; w.y = (double)acc1;
      *reinterpret_cast<double2*>(Out + (long long)s * b + c) = w;
    }
  }
}

int launch_spmm(int precision, const int32_t* ptr, const int32_t* idx, const void* val, const double* X, double* Out,
                int n_out, int b, cudaStream_t st) {
  if (n_out <= 0) return 0;
  int G = 1;
  while (2 * G < b) G <<= 1;   // G lanes x 2 columns >= b
  if (G > 32) G = 32;
  const int threads = 256, warps = threads / 32;
  int blocks = (int)svt_min_ll(svt_ceil_div(n_out, warps), 152LL * 16);
  if (precision == 0)
    k_spmm<double, double><<<blocks, threads, 0, st>>>(ptr, idx, (const double*)val, X, Out, n_out, b, G);
  else
    k_spmm<float, float><<<blocks, threads, 0, st>>>(ptr, idx, (const float*)val, X, Out, n_out, b, G);
  return 1;
}

// ------------------------------------------------------------------------------------------------
// Fused X-on-Omega + dual step + residual.  One warp per row i of Omega: the row Ut[i, :] (r <= 64
// values) sits in two registers per lane and is broadcast with shuffles; each lane owns one
// sampled entry p = (i, j) per step, gathers V[j, :] (r contiguous doubles), forms
// x = <Ut[i,:], V[j,:]>, e = M_p - x, writes y_out[p] = y_in[p] + delta e (and the column-major
// copy), and accumulates e^2.  Block partial sums are summed in a fixed order afterwards.
// ------------------------------------------------------------------------------------------------
static constexpr int UPD_THREADS = 256;
static constexpr int UPD_BLOCKS = 152 * 8;

template <typename VT, typename AT>
__global__ void __launch_bounds__(UPD_THREADS)
k_sddmm_update(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
               const int32_t* __restrict__ csr_to_csc, const VT* __restrict__ M, const VT* __restrict__ y_in,
               VT* __restrict__ y_out, VT* __restrict__ y_out_csc, const double* __restrict__ Ut,
               const double* __restrict__ V, int r, int n_rows, AT delta, double* __restrict__ partial,
               unsigned int* err) {
  __shared__ double red[UPD_THREADS / 32];
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  double acc = 0.0;
  for (int i = blockIdx.x * warps + (threadIdx.x >> 5); i < n_rows; i += gridDim.x * warps) {
    const int a = row_ptr[i], e = row_ptr[i + 1];
    if (a == e) continue;
    AT u0 = lane < r ? (AT)Ut[(long long)i * r + lane] : (AT)0;
    AT u1 = lane + 32 < r ? (AT)Ut[(long long)i * r + lane + 32] : (AT)0;
    for (int base = a; base < e; base += 32) {
      const int p = base + lane;
      const bool live = p < e;
      const int j = live ? col_idx[p] : 0;
      const double* vj = V + (long long)j * r;
      AT x = 0;
      for (int t = 0; t < r && t < 32; ++t) {
        AT ut = __shfl_sync(0xffffffffu, u0, t);
        if (live) x += ut * (AT)__ldg(vj + t);
      }
      for (int t = 32; t < r; ++t) {
        AT ut = __shfl_sync(0xffffffffu, u1, t - 32);
        if (live) x += ut * (AT)__ldg(vj + t);
      }
      if (live) {
        AT ev = (AT)M[p] - x;
        VT yn = (VT)((AT)y_in[p] + delta * ev);
        y_out[p] = yn;
        if (y_out_csc) y_out_csc[csr_to_csc[p]] = yn;
        acc += (double)ev * (double)ev;
      }
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < warps ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) {
      partial[blockIdx.x] = v;
      if (!isfinite(v)) svt_set_error(err, SVT_DEVERR_NONFINITE);
    }
  }
}

__global__ void k_sum_fixed(const double* __restrict__ partial, int np, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partial[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *out = v;
  }
}

int sddmm_partial_doubles() { return UPD_BLOCKS; }

int launch_sddmm_update(int precision, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* csr_to_csc,
                        const void* M, const void* y_in, void* y_out, void* y_out_csc, const double* Ut,
                        const double* V, int r, int n_rows, double delta, double* partial, double* res2,
                        unsigned int* err, cudaStream_t st) {
  if (precision == 0)
    k_sddmm_update<double, double><<<UPD_BLOCKS, UPD_THREADS, 0, st>>>(
        row_ptr, col_idx, csr_to_csc, (const double*)M, (const double*)y_in, (double*)y_out, (double*)y_out_csc, Ut, V,
        r, n_rows, delta, partial, err);
  else
    k_sddmm_update<float, float><<<UPD_BLOCKS, UPD_THREADS, 0, st>>>(
        row_ptr, col_idx, csr_to_csc, (const float*)M, (const float*)y_in, (float*)y_out, (float*)y_out_csc, Ut, V,
        r, n_rows, (float)delta, partial, err);
  k_sum_fixed<<<1, 1024, 0, st>>>(partial, UPD_BLOCKS, res2);
  return 2;
}

// ------------------------------------------------------------------------------------------------
// Value-array helpers (kick, load/store in the context's value type).
// ------------------------------------------------------------------------------------------------
template <typename VT>
__global__ void k_scale_values(const VT* __restrict__ M, double alpha, VT* __restrict__ y, VT* __restrict__ y_csc,
                               const int32_t* __restrict__ csr_to_csc, long long nnz) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x) {
    VT v = (VT)(alpha * (double)M[p]);
    y[p] = v;
    if (y_csc) y_csc[csr_to_csc[p]] = v;
  }
}

int launch_scale_values(int precision, const void* M, double alpha, void* y, void* y_csc, const int32_t* csr_to_csc,
                        long long nnz, cudaStream_t st) {
  int blocks = (int)svt_min_ll(svt_ceil_div(nnz, 256), 152LL * 16);
  if (blocks < 1) return 0;
  if (precision == 0)
    k_scale_values<double><<<blocks, 256, 0, st>>>((const double*)M, alpha, (double*)y, (double*)y_csc, csr_to_csc, nnz);
  else
    k_scale_values<float><<<blocks, 256, 0, st>>>((const float*)M, alpha, (float*)y, (float*)y_csc, csr_to_csc, nnz);
  return 1;
}

template <typename VT>
__global__ void k_load_values(const double* __restrict__ src, VT* __restrict__ y, VT* __restrict__ y_csc,
                              const int32_t* __restrict__ csr_to_csc, long long nnz) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x) {
    VT v = (VT)src[p];
    y[p] = v;
    if (y_csc) y_csc[csr_to_csc[p]] = v;
  }
}

int launch_load_values(int precision, const double* src, void* y, void* y_csc, const int32_t* csr_to_csc,
                       long long nnz, cudaStream_t st) {
  int blocks = (int)svt_min_ll(svt_ceil_div(nnz, 256), 152LL * 16);
  if (blocks < 1) return 0;
  if (precision == 0)
    k_load_values<double><<<blocks, 256, 0, st>>>(src, (double*)y, (double*)y_csc, csr_to_csc, nnz);
  else
    k_load_values<float><<<blocks, 256, 0, st>>>(src, (float*)y, (float*)y_csc, csr_to_csc, nnz);
  return 1;
}

template <typename VT>
__global__ void k_store_values(const VT* __restrict__ y, double* __restrict__ dst, long long nnz) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x)
    dst[p] = (double)y[p];
}

int launch_store_values(int precision, const void* y, double* dst, long long nnz, cudaStream_t st) {
  int blocks = (int)svt_min_ll(svt_ceil_div(nnz, 256), 152LL * 16);
  if (blocks < 1) return 0;
  if (precision == 0)
    k_store_values<double><<<blocks, 256, 0, st>>>((const double*)y, dst, nnz);
  else
    k_store_values<float><<<blocks, 256, 0, st>>>((const float*)y, dst, nnz);
  return 1;
}

}  // namespace svt
