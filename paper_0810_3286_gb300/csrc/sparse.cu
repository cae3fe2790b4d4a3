// Per-iteration kernels that stream Omega: the two sparse products of the Lanczos partial SVD
// (Y V and Y^T U, Sec. 2.2 / Sec. 5.1.1) and the fused X-on-Omega + dual step + residual of
// Algorithm 1 (Sec. 5.1.5; residual of eq. (5.5)).
#include "common.cuh"
#include "internal.h"

namespace svt {

// ------------------------------------------------------------------------------------------------
// SpMM over compressed segments: Out[s, :] = sum_{p in segment s} val[p] * X[idx[p], :].
//
// WPR warps share one segment (row of Y for Y V, column of Y for Y^T U using the column-major copy
// of the values), each taking a contiguous slice of its entries, so that short products still
// put enough warps on every SM to hide the gather latency.  Inside a warp a group of G lanes
// covers one sampled entry, each lane two adjacent columns of the b-wide dense row (one 16-byte
// load of X); 32/G entries are in flight per step, four steps are unrolled.  Lane partials are
// combined with xor shuffles and the WPR warp partials in shared memory, always in the same order
// (deterministic, no atomics).
// ------------------------------------------------------------------------------------------------
static constexpr int SPMM_T = 256;

template <typename VT, typename AT>
__global__ void __launch_bounds__(SPMM_T)
k_spmm(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx, const VT* __restrict__ val,
       const double* __restrict__ X, double* __restrict__ Out, int n_out, int b, int G, int WPR) {
  __shared__ double part[SPMM_T / 32][64];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int segs_per_block = (SPMM_T / 32) / WPR;
  const int slot = warp / WPR, wp = warp - slot * WPR;
  const int gl = lane & (G - 1);
  const int grp = lane / G;
  const int ngrp = 32 / G;
  const int c = 2 * gl;
  const bool active_col = c < b;
  for (int s0 = blockIdx.x * segs_per_block; s0 < n_out; s0 += gridDim.x * segs_per_block) {
    const int s = s0 + slot;
    AT acc0 = 0, acc1 = 0;
    if (s < n_out) {
      const int a = ptr[s], e = ptr[s + 1];
      const int len = e - a;
      const int chunk = (len + WPR - 1) / WPR;
      const int lo = a + wp * chunk;
      const int hi = min(e, lo + chunk);
      int p = lo + grp;
      for (; p + 3 * ngrp < hi; p += 4 * ngrp) {
        int j0 = __ldg(idx + p), j1 = __ldg(idx + p + ngrp), j2 = __ldg(idx + p + 2 * ngrp),
            j3 = __ldg(idx + p + 3 * ngrp);
        AT v0 = (AT)__ldg(val + p), v1 = (AT)__ldg(val + p + ngrp), v2 = (AT)__ldg(val + p + 2 * ngrp),
           v3 = (AT)__ldg(val + p + 3 * ngrp);
        if (active_col) {
          double2 x0 = __ldg(reinterpret_cast<const double2*>(X + (long long)j0 * b + c));
          double2 x1 = __ldg(reinterpret_cast<const double2*>(X + (long long)j1 * b + c));
          double2 x2 = __ldg(reinterpret_cast<const double2*>(X + (long long)j2 * b + c));
          double2 x3 = __ldg(reinterpret_cast<const double2*>(X + (long long)j3 * b + c));
          acc0 += v0 * (AT)x0.x; acc1 += v0 * (AT)x0.y;
          acc0 += v1 * (AT)x1.x; acc1 += v1 * (AT)x1.y;
          acc0 += v2 * (AT)x2.x; acc1 += v2 * (AT)x2.y;
          acc0 += v3 * (AT)x3.x; acc1 += v3 * (AT)x3.y;
        }
      }
      for (; p < hi; p += ngrp) {
        int j0 = __ldg(idx + p);
        AT v0 = (AT)__ldg(val + p);
        if (active_col) {
          double2 x0 = __ldg(reinterpret_cast<const double2*>(X + (long long)j0 * b + c));
          acc0 += v0 * (AT)x0.x; acc1 += v0 * (AT)x0.y;
        }
      }
    }
    for (int o = G; o < 32; o <<= 1) {
      acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
      acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
    }
    if (WPR == 1) {
      if (s < n_out && grp == 0 && active_col) {
        double2 w;
        w.x = (double)acc0; w.y = (double)acc1;
        *reinterpret_cast<double2*>(Out + (long long)s * b + c) = w;
      }
    } else {
      if (grp == 0 && active_col) {
        part[warp][c] = (double)acc0;
        part[warp][c + 1] = (double)acc1;
      }
      __syncthreads();
      if (wp == 0 && s < n_out && grp == 0 && active_col) {
        double w0 = 0.0, w1 = 0.0;
        for (int k = 0; k < WPR; ++k) {
          w0 += part[warp + k][c];
          w1 += part[warp + k][c + 1];
        }
        double2 w;
        w.x = w0; w.y = w1;
        *reinterpret_cast<double2*>(Out + (long long)s * b + c) = w;
      }
      __syncthreads();
    }
  }
}

int launch_spmm(int precision, const int32_t* ptr, const int32_t* idx, const void* val, const double* X, double* Out,
                int n_out, int b, cudaStream_t st, long long nnz) {
  if (n_out <= 0) return 0;
  int G = 1;
  while (2 * G < b) G <<= 1;   // G lanes x 2 columns >= b
  if (G > 32) G = 32;
  // warps per segment from the mean segment length (entries per warp step = 32 / G)
  const double mean_len = nnz > 0 ? (double)nnz / n_out : 0.0;
  int WPR = 1;
  while (WPR < 8 && mean_len / WPR > 8.0 * (32 / G)) WPR <<= 1;
  const int segs_per_block = (SPMM_T / 32) / WPR;
  int blocks = (int)svt_min_ll(svt_ceil_div(n_out, segs_per_block), 152LL * 16);
  if (precision == 0)
    k_spmm<double, double><<<blocks, SPMM_T, 0, st>>>(ptr, idx, (const double*)val, X, Out, n_out, b, G, WPR);
  else
    k_spmm<float, float><<<blocks, SPMM_T, 0, st>>>(ptr, idx, (const float*)val, X, Out, n_out, b, G, WPR);
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

// RMAX: compile-time bound on r (16, 32 or 64) so that the gathered row V[j, :] lives in registers:
// all r loads of a lane are issued before the dot product, one gather round trip per entry.
template <typename VT, typename AT, int RMAX>
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
      double vr[RMAX];
#pragma unroll
      for (int t = 0; t < RMAX; ++t) vr[t] = (live && t < r) ? __ldg(vj + t) : 0.0;
      const AT mp = live ? (AT)M[p] : (AT)0;
      const AT yp = live ? (AT)y_in[p] : (AT)0;
      const int q = (live && y_out_csc) ? csr_to_csc[p] : 0;
      AT x0 = 0, x1 = 0;
#pragma unroll
      for (int t = 0; t < RMAX; ++t) {
        if (t >= r) break;
        AT ut = t < 32 ? __shfl_sync(0xffffffffu, u0, t) : __shfl_sync(0xffffffffu, u1, t - 32);
        if (t & 1) x1 += ut * (AT)vr[t];
        else x0 += ut * (AT)vr[t];
      }
      if (live) {
        AT ev = mp - (x0 + x1);
        VT yn = (VT)(yp + delta * ev);
        y_out[p] = yn;
        if (y_out_csc) y_out_csc[q] = yn;
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

template <typename VT, typename AT>
static void sddmm_dispatch(int rmax, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* csr_to_csc,
                           const VT* M, const VT* y_in, VT* y_out, VT* y_out_csc, const double* Ut, const double* V,
                           int r, int n_rows, AT delta, double* partial, unsigned int* err, cudaStream_t st) {
  if (rmax <= 16)
    k_sddmm_update<VT, AT, 16><<<UPD_BLOCKS, UPD_THREADS, 0, st>>>(row_ptr, col_idx, csr_to_csc, M, y_in, y_out,
                                                                    y_out_csc, Ut, V, r, n_rows, delta, partial, err);
  else if (rmax <= 32)
    k_sddmm_update<VT, AT, 32><<<UPD_BLOCKS, UPD_THREADS, 0, st>>>(row_ptr, col_idx, csr_to_csc, M, y_in, y_out,
                                                                    y_out_csc, Ut, V, r, n_rows, delta, partial, err);
  else
    k_sddmm_update<VT, AT, 64><<<UPD_BLOCKS, UPD_THREADS, 0, st>>>(row_ptr, col_idx, csr_to_csc, M, y_in, y_out,
                                                                    y_out_csc, Ut, V, r, n_rows, delta, partial, err);
}

int launch_sddmm_update(int precision, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* csr_to_csc,
                        const void* M, const void* y_in, void* y_out, void* y_out_csc, const double* Ut,
                        const double* V, int r, int n_rows, double delta, double* partial, double* res2,
                        unsigned int* err, cudaStream_t st) {
  if (precision == 0)
    sddmm_dispatch<double, double>(r, row_ptr, col_idx, csr_to_csc, (const double*)M, (const double*)y_in,
                                   (double*)y_out, (double*)y_out_csc, Ut, V, r, n_rows, delta, partial, err, st);
  else
    sddmm_dispatch<float, float>(r, row_ptr, col_idx, csr_to_csc, (const float*)M, (const float*)y_in, (float*)y_out,
                                 (float*)y_out_csc, Ut, V, r, n_rows, (float)delta, partial, err, st);
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

namespace svt {

// Same fused kernel with a caller-chosen grid and partial-sum buffer (one partial per CTA), for the
// entry point that works without device allocations.
int launch_sddmm_update_grid(const int32_t* row_ptr, const int32_t* col_idx, const double* M, const double* y_in,
                             double* y_out, const double* Ut, const double* V, int r, int n_rows, double delta,
                             int blocks, double* partial, double* res2, cudaStream_t st) {
  if (r <= 16)
    k_sddmm_update<double, double, 16><<<blocks, UPD_THREADS, 0, st>>>(row_ptr, col_idx, nullptr, M, y_in, y_out,
                                                                        nullptr, Ut, V, r, n_rows, delta, partial,
                                                                        nullptr);
  else if (r <= 32)
    k_sddmm_update<double, double, 32><<<blocks, UPD_THREADS, 0, st>>>(row_ptr, col_idx, nullptr, M, y_in, y_out,
                                                                        nullptr, Ut, V, r, n_rows, delta, partial,
                                                                        nullptr);
  else
    k_sddmm_update<double, double, 64><<<blocks, UPD_THREADS, 0, st>>>(row_ptr, col_idx, nullptr, M, y_in, y_out,
                                                                        nullptr, Ut, V, r, n_rows, delta, partial,
                                                                        nullptr);
  k_sum_fixed<<<1, 1024, 0, st>>>(partial, blocks, res2);
  return 2;
}

}  // namespace svt
