// Per-iteration kernels that stream Omega: the two sparse products of the Lanczos partial SVD
// (Y V and Y^T U, Sec. 2.2 / Sec. 5.1.1) and the fused X-on-Omega + dual step + residual of
// Algorithm 1 (Sec. 5.1.5; residual of eq. (5.5)).
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace svt {

// ------------------------------------------------------------------------------------------------
// SpMM over compressed segments: Out[s, :] = sum_{p in segment s} val[p] * X[idx[p], :].
//
// WPR warps share one segment (row of Y for Y V, column of Y for Y^T U using the column-major copy
// of the values), each taking a contiguous slice of its entries, so that short products still
// put enough warps on every SM to hide the gather latency.  Inside a warp a group of G lanes
// covers one sampled entry, each lane CPL adjacent columns of the b-wide dense row (one 16-byte
// load of X: two float64 or four float32 columns); 32/G entries are in flight per step, four
// steps are unrolled.  Lane partials are combined with xor shuffles and the WPR warp partials in
// shared memory, always in the same order (deterministic, no atomics).  Out is float64.
//
// The float32 path reads a float32 copy of the dense block and accumulates in float32: no
// float64 instruction per sampled entry (GB300 issues float64 at 1/64 of the float32 rate, and
// a float64 -> float32 conversion per gathered element made this kernel float64-pipe bound).
// ------------------------------------------------------------------------------------------------
static constexpr int SPMM_T = 256;

template <typename XT> struct XRow;
template <> struct XRow<double> { static constexpr int CPL = 2; using V = double2; };
template <> struct XRow<float> { static constexpr int CPL = 4; using V = float4; };

__device__ __forceinline__ double xcomp(const double2& v, int q) { return q == 0 ? v.x : v.y; }
__device__ __forceinline__ float xcomp(const float4& v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}

template <typename XT, typename AT, int CPL>
__device__ __forceinline__ void spmm_fma(AT (&acc)[CPL], AT v, const XT* __restrict__ src) {
  const typename XRow<XT>::V x = __ldg(reinterpret_cast<const typename XRow<XT>::V*>(src));
#pragma unroll
  for (int q = 0; q < CPL; ++q) acc[q] = fmac(v, (AT)xcomp(x, q), acc[q]);
}

// The segments s0 .. s0 + (SPMM_T / 32) / WPR - 1 of one product, by the whole CTA.
template <typename VT, typename XT, typename AT>
__device__ __forceinline__ void spmm_tile(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                          const VT* __restrict__ val, const XT* __restrict__ X,
                                          double* __restrict__ Out, int n_out, int b, int G, int WPR, int s0) {
  constexpr int CPL = XRow<XT>::CPL;
  __shared__ double part[SPMM_T / 32][64];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int slot = warp / WPR, wp = warp - slot * WPR;
  const int gl = lane & (G - 1);
  const int grp = lane / G;
  const int ngrp = 32 / G;
  const int c = CPL * gl;
  const bool active_col = c < b;
  {
    const int s = s0 + slot;
    AT acc[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) acc[q] = (AT)0;
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
          spmm_fma<XT, AT, CPL>(acc, v0, X + (long long)j0 * b + c);
          spmm_fma<XT, AT, CPL>(acc, v1, X + (long long)j1 * b + c);
          spmm_fma<XT, AT, CPL>(acc, v2, X + (long long)j2 * b + c);
          spmm_fma<XT, AT, CPL>(acc, v3, X + (long long)j3 * b + c);
        }
      }
      for (; p < hi; p += ngrp) {
        int j0 = __ldg(idx + p);
        AT v0 = (AT)__ldg(val + p);
        if (active_col) spmm_fma<XT, AT, CPL>(acc, v0, X + (long long)j0 * b + c);
      }
    }
    for (int o = G; o < 32; o <<= 1) {
#pragma unroll
      for (int q = 0; q < CPL; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    }
    if (WPR == 1) {
      if (s < n_out && grp == 0 && active_col) {
        double* dst = Out + (long long)s * b + c;
#pragma unroll
        for (int q = 0; q < CPL; q += 2) {
          double2 w;
          w.x = (double)acc[q]; w.y = (double)acc[q + 1];
          *reinterpret_cast<double2*>(dst + q) = w;
        }
      }
    } else {
      if (grp == 0 && active_col) {
#pragma unroll
        for (int q = 0; q < CPL; ++q) part[warp][c + q] = (double)acc[q];
      }
      __syncthreads();
      if (wp == 0 && s < n_out && grp == 0 && active_col) {
        double w[CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) w[q] = 0.0;
        for (int k = 0; k < WPR; ++k) {
#pragma unroll
          for (int q = 0; q < CPL; ++q) w[q] += part[warp + k][c + q];
        }
        double* dst = Out + (long long)s * b + c;
#pragma unroll
        for (int q = 0; q < CPL; q += 2) {
          double2 v2;
          v2.x = w[q]; v2.y = w[q + 1];
          *reinterpret_cast<double2*>(dst + q) = v2;
        }
      }
      __syncthreads();
    }
  }
}

template <typename VT, typename XT, typename AT>
__global__ void __launch_bounds__(SPMM_T)
k_spmm(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx, const VT* __restrict__ val,
       const XT* __restrict__ X, double* __restrict__ Out, int n_out, int b, int G, int WPR) {
  const int segs_per_block = (SPMM_T / 32) / WPR;
  for (int s0 = blockIdx.x * segs_per_block; s0 < n_out; s0 += gridDim.x * segs_per_block)
    spmm_tile<VT, XT, AT>(ptr, idx, val, X, Out, n_out, b, G, WPR, s0);
}

// Ragged persistent form over a job list (batched engine): the tiles of all listed products form
// one index space (job k owns tiles tile0 .. tile0 + ceil(n_out / segments per tile) - 1); each CTA
// takes tiles grid-stride and finds the job of a tile by a scan of the (at most kBatchMaxJobs)
// offsets.  Every segment is computed exactly as k_spmm computes it with the same G and WPR.
template <typename VT, typename XT, typename AT>
__global__ void __launch_bounds__(SPMM_T) k_spmm_jobs(const __grid_constant__ SpmmJobTable tab) {
  for (int t = blockIdx.x; t < tab.tiles; t += gridDim.x) {
    int k = 0;
    while (k + 1 < tab.n && tab.job[k + 1].tile0 <= t) ++k;
    const SpmmJobDev& J = tab.job[k];
    const int segs_per_block = (SPMM_T / 32) / J.WPR;
    spmm_tile<VT, XT, AT>(J.ptr, J.idx, static_cast<const VT*>(J.val), static_cast<const XT*>(J.X), J.Out, J.n_out,
                          J.b, J.G, J.WPR, (t - J.tile0) * segs_per_block);
  }
}

// Lanes per sampled entry (G) and warps per segment (WPR) of a product with b columns and mean
// segment length nnz / n_out.  wpr_override > 0 replaces the rule (the batched engine's tuner).
static void spmm_shape(int CPL, int b, long long nnz, int n_out, int wpr_override, int* G_out, int* WPR_out) {
  int G = 1;
  while (CPL * G < b) G <<= 1;   // G lanes x CPL columns >= b
  if (G > 32) G = 32;
  // warps per segment from the mean segment length (entries per warp step = 32 / G)
  const double mean_len = nnz > 0 ? (double)nnz / n_out : 0.0;
  int WPR = 1;
  while (WPR < 8 && mean_len / WPR > 8.0 * (32 / G)) WPR <<= 1;
  if (wpr_override == 1 || wpr_override == 2 || wpr_override == 4 || wpr_override == 8) WPR = wpr_override;
  *G_out = G;
  *WPR_out = WPR;
}

template <typename VT, typename XT, typename AT>
static void spmm_launch(const int32_t* ptr, const int32_t* idx, const VT* val, const XT* X, double* Out, int n_out,
                        int b, cudaStream_t st, long long nnz) {
  constexpr int CPL = XRow<XT>::CPL;
  int G = 1, WPR = 1;
  spmm_shape(CPL, b, nnz, n_out, 0, &G, &WPR);
  const int segs_per_block = (SPMM_T / 32) / WPR;
  int blocks = (int)svt_min_ll(svt_ceil_div(n_out, segs_per_block), 152LL * 16);
  k_spmm<VT, XT, AT><<<blocks, SPMM_T, 0, st>>>(ptr, idx, val, X, Out, n_out, b, G, WPR);
}

// One launch for the products of a job list: precision as launch_spmm (0 float64, 1 float32 values
// with the float32 block copies, 2 bfloat16 values with them); the jobs' tile offsets are set here.
int launch_spmm_jobs(int precision, const SpmmJob* jobs, int n, int grid, cudaStream_t st) {
  if (n <= 0 || n > kBatchMaxJobs) return 0;
  SpmmJobTable tab{};
  tab.n = 0;
  int tiles = 0;
  const int CPL = precision == 0 ? XRow<double>::CPL : XRow<float>::CPL;
  for (int k = 0; k < n; ++k) {
    const SpmmJob& J = jobs[k];
    if (J.n_out <= 0) continue;
    SpmmJobDev& d = tab.job[tab.n++];
    d.ptr = J.ptr; d.idx = J.idx; d.val = J.val; d.Out = J.Out; d.n_out = J.n_out; d.b = J.b;
    d.X = precision == 0 ? static_cast<const void*>(J.X) : static_cast<const void*>(J.Xf);
    if (!d.X) return 0;
    spmm_shape(CPL, J.b, J.nnz, J.n_out, J.wpr, &d.G, &d.WPR);
    d.tile0 = tiles;
    tiles += (J.n_out + (SPMM_T / 32) / d.WPR - 1) / ((SPMM_T / 32) / d.WPR);
  }
  if (tab.n == 0) return 0;
  tab.tiles = tiles;
  const int blocks = std::max(1, std::min(tiles, grid > 0 ? grid : 152 * 16));
  if (precision == 2) k_spmm_jobs<__nv_bfloat16, float, float><<<blocks, SPMM_T, 0, st>>>(tab);
  else if (precision == 0) k_spmm_jobs<double, double, double><<<blocks, SPMM_T, 0, st>>>(tab);
  else k_spmm_jobs<float, float, float><<<blocks, SPMM_T, 0, st>>>(tab);
  return 1;
}

int launch_spmm(int precision, const int32_t* ptr, const int32_t* idx, const void* val, const double* X,
                const float* Xf, double* Out, int n_out, int b, cudaStream_t st, long long nnz) {
  if (n_out <= 0) return 0;
  if (precision == 2) {
    if (!Xf) return 0;   // bfloat16 values are read only with the float32 copy of the dense block
    spmm_launch<__nv_bfloat16, float, float>(ptr, idx, (const __nv_bfloat16*)val, Xf, Out, n_out, b, st, nnz);
    return 1;
  }
  if (precision == 0)
    spmm_launch<double, double, double>(ptr, idx, (const double*)val, X, Out, n_out, b, st, nnz);
  else if (Xf)
    spmm_launch<float, float, float>(ptr, idx, (const float*)val, Xf, Out, n_out, b, st, nnz);
  else
    spmm_launch<float, double, float>(ptr, idx, (const float*)val, X, Out, n_out, b, st, nnz);
  return 1;
}

// ------------------------------------------------------------------------------------------------
// Fused X-on-Omega + dual step + residual.  One warp per row i of Omega: the row Ut[i, :] (r <= 64
// values) sits in two registers per lane and is broadcast with shuffles; each lane owns one
// sampled entry p = (i, j) per step, gathers V[j, :] (r contiguous values), forms
// x = <Ut[i,:], V[j,:]>, e = M_p - x, writes y_out[p] = y_in[p] + delta e (and the column-major
// copy), and accumulates e^2 (per lane in the accumulation type, then float64 across lanes and
// CTAs).  Block partial sums are summed in a fixed order afterwards.
//
// FT is the factor type.  The float32 path passes float32 factors whose rows are padded to a
// multiple of four (ldf), so a gathered row is ceil(r / 4) 16-byte loads and no float64
// instruction runs per sampled entry; the float64 path and the float64 entry points pass float64
// factors with ldf = r.
// ------------------------------------------------------------------------------------------------
static constexpr int UPD_THREADS = 256;
static constexpr int UPD_BLOCKS = 152 * 8;

// DS (the matrix Dantzig selector, iteration (iterDS2) of Sec. 3.3): the two multipliers Y_+, Y_- of
// the constraints B - X <= E and X - B <= E are updated as Y_+' = [Y_+ + delta (e - E)]_+ and
// Y_-' = [Y_- + delta (-e - E)]_+ (e = B - X), the operand of the next shrink is Y_+' - Y_-', and the
// reduction sums the constraint violation [|e| - E]_+^2 instead of e^2.
template <typename VT>
struct DualArgs {
  const VT* yp_in;
  const VT* ym_in;
  VT* yp_out;
  VT* ym_out;
  double E;
};

// RMAX: compile-time bound on r (16, 32 or 64) so that the gathered row V[j, :] lives in registers:
// all loads of a lane are issued before the dot product, one gather round trip per entry.
// Row i of the fused update, by one warp: e^2 (or the Dantzig violation) of its entries is added to
// this lane's acc.
template <typename VT, typename AT, typename FT, int RMAX, bool DS>
__device__ __forceinline__ void upd_row(int i, int lane, const int32_t* __restrict__ row_ptr,
                                        const int32_t* __restrict__ col_idx, const int32_t* __restrict__ csr_to_csc,
                                        const VT* __restrict__ M, const VT* __restrict__ y_in, VT* __restrict__ y_out,
                                        VT* __restrict__ y_out_csc, const FT* __restrict__ Ut,
                                        const FT* __restrict__ V, int r, int ldf, AT delta, const DualArgs<VT>& ds,
                                        __nv_bfloat16* __restrict__ ys_out, __nv_bfloat16* __restrict__ ys_out_csc,
                                        AT& acc) {
  const int a = row_ptr[i], e = row_ptr[i + 1];
  if (a == e) return;
  AT u0 = lane < r ? (AT)Ut[(long long)i * ldf + lane] : (AT)0;
  AT u1 = lane + 32 < r ? (AT)Ut[(long long)i * ldf + lane + 32] : (AT)0;
  for (int base = a; base < e; base += 32) {
    const int p = base + lane;
    const bool live = p < e;
    const int j = live ? col_idx[p] : 0;
    const FT* vj = V + (long long)j * ldf;
    FT vr[RMAX];
    if constexpr (sizeof(FT) == 4) {
#pragma unroll
      for (int t4 = 0; t4 < RMAX / 4; ++t4) {
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
        if (live && 4 * t4 < r) w = __ldg(reinterpret_cast<const float4*>(vj) + t4);
        vr[4 * t4] = w.x; vr[4 * t4 + 1] = w.y; vr[4 * t4 + 2] = w.z; vr[4 * t4 + 3] = w.w;
      }
    } else {
#pragma unroll
      for (int t = 0; t < RMAX; ++t) vr[t] = (live && t < r) ? __ldg(vj + t) : (FT)0;
    }
    const AT mp = live ? (AT)M[p] : (AT)0;
    AT yp = (AT)0, ypl = (AT)0, ymi = (AT)0;
    if constexpr (DS) {
      ypl = live ? (AT)ds.yp_in[p] : (AT)0;
      ymi = live ? (AT)ds.ym_in[p] : (AT)0;
    } else {
      yp = live ? (AT)y_in[p] : (AT)0;
    }
    const int q = (live && (y_out_csc || ys_out)) ? csr_to_csc[p] : 0;
    AT x0 = 0, x1 = 0;
#pragma unroll
    for (int t = 0; t < RMAX; ++t) {
      if (t >= r) break;
      AT ut = t < 32 ? __shfl_sync(0xffffffffu, u0, t) : __shfl_sync(0xffffffffu, u1, t - 32);
      if (t & 1) x1 = fmac(ut, (AT)vr[t], x1);
      else x0 = fmac(ut, (AT)vr[t], x0);
    }
    if (live) {
      AT ev = mp - (x0 + x1);
      if constexpr (DS) {
        const AT E = (AT)ds.E;
        const AT ypn = fmax(ypl + delta * (ev - E), (AT)0);
        const AT ymn = fmax(ymi + delta * (-ev - E), (AT)0);
        ds.yp_out[p] = (VT)ypn;
        ds.ym_out[p] = (VT)ymn;
        const VT yn = (VT)(ypn - ymn);
        y_out[p] = yn;
        if (y_out_csc) y_out_csc[q] = yn;
        if (ys_out) {
          const __nv_bfloat16 yb = __float2bfloat16_rn((float)yn);
          ys_out[p] = yb;
          ys_out_csc[q] = yb;
        }
        const AT v = fmax(fabs(ev) - E, (AT)0);
        acc += v * v;
      } else {
        VT yn = (VT)(yp + delta * ev);
        y_out[p] = yn;
        if (y_out_csc) y_out_csc[q] = yn;
        if (ys_out) {
          const __nv_bfloat16 yb = __float2bfloat16_rn((float)yn);
          ys_out[p] = yb;
          ys_out_csc[q] = yb;
        }
        acc += ev * ev;
      }
    }
  }
}

template <typename VT, typename AT, typename FT, int RMAX, bool DS>
__global__ void __launch_bounds__(UPD_THREADS)
k_sddmm_update(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
               const int32_t* __restrict__ csr_to_csc, const VT* __restrict__ M, const VT* __restrict__ y_in,
               VT* __restrict__ y_out, VT* __restrict__ y_out_csc, const FT* __restrict__ Ut,
               const FT* __restrict__ V, int r, int ldf, int n_rows, AT delta, double* __restrict__ partial,
               unsigned int* err, DualArgs<VT> ds, __nv_bfloat16* __restrict__ ys_out,
               __nv_bfloat16* __restrict__ ys_out_csc, const int* __restrict__ r_dev) {
  __shared__ double red[UPD_THREADS / 32];
  if (r_dev) r = min(*r_dev, r);
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  AT acc = (AT)0;
  for (int i = blockIdx.x * warps + (threadIdx.x >> 5); i < n_rows; i += gridDim.x * warps) {
    upd_row<VT, AT, FT, RMAX, DS>(i, lane, row_ptr, col_idx, csr_to_csc, M, y_in, y_out, y_out_csc, Ut, V, r, ldf,
                                  delta, ds, ys_out, ys_out_csc, acc);
  }
  double accd = warp_sum((double)acc);
  if (lane == 0) red[threadIdx.x >> 5] = accd;
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

template <typename VT, typename AT, typename FT, bool DS>
static void sddmm_dispatch(const int32_t* row_ptr, const int32_t* col_idx, const int32_t* csr_to_csc, const VT* M,
                           const VT* y_in, VT* y_out, VT* y_out_csc, const FT* Ut, const FT* V, int r, int ldf,
                           int n_rows, AT delta, int blocks, double* partial, unsigned int* err, cudaStream_t st,
                           DualArgs<VT> ds, __nv_bfloat16* ys = nullptr, __nv_bfloat16* ys_csc = nullptr,
                           const int* r_dev = nullptr) {
  if (r <= 16)
    k_sddmm_update<VT, AT, FT, 16, DS><<<blocks, UPD_THREADS, 0, st>>>(row_ptr, col_idx, csr_to_csc, M,
        y_in, y_out, y_out_csc, Ut, V, r, ldf, n_rows, delta, partial, err, ds, ys, ys_csc, r_dev);
  else if (r <= 32)
    k_sddmm_update<VT, AT, FT, 32, DS><<<blocks, UPD_THREADS, 0, st>>>(row_ptr, col_idx, csr_to_csc, M,
        y_in, y_out, y_out_csc, Ut, V, r, ldf, n_rows, delta, partial, err, ds, ys, ys_csc, r_dev);
  else
    k_sddmm_update<VT, AT, FT, 64, DS><<<blocks, UPD_THREADS, 0, st>>>(row_ptr, col_idx, csr_to_csc, M,
        y_in, y_out, y_out_csc, Ut, V, r, ldf, n_rows, delta, partial, err, ds, ys, ys_csc, r_dev);
}

int launch_sddmm_update(int precision, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* csr_to_csc,
                        const void* M, const void* y_in, void* y_out, void* y_out_csc, const double* Ut,
                        const double* V, const float* Utf, const float* Vf32, int ldf, int r, int n_rows,
                        double delta, double* partial, double* res2, unsigned int* err, cudaStream_t st,
                        const SddmmDual* dual, void* ys_out, void* ys_out_csc, const int* r_dev, int ld64) {
  if (ld64 <= 0) ld64 = r;
  __nv_bfloat16* ys = static_cast<__nv_bfloat16*>(ys_out);
  __nv_bfloat16* ysc = static_cast<__nv_bfloat16*>(ys_out_csc);
  if ((ys != nullptr) != (ysc != nullptr) || (ys && !y_out_csc)) return 0;
  if (precision == 0) {
    DualArgs<double> ds{};
    if (dual) {
      ds = {(const double*)dual->yp_in, (const double*)dual->ym_in, (double*)dual->yp_out, (double*)dual->ym_out, dual->E};
      sddmm_dispatch<double, double, double, true>(row_ptr, col_idx, csr_to_csc, (const double*)M, nullptr,
                                                   (double*)y_out, (double*)y_out_csc, Ut, V, r, ld64, n_rows, delta,
                                                   UPD_BLOCKS, partial, err, st, ds, nullptr, nullptr, r_dev);
    } else {
      sddmm_dispatch<double, double, double, false>(row_ptr, col_idx, csr_to_csc, (const double*)M,
                                                    (const double*)y_in, (double*)y_out, (double*)y_out_csc, Ut, V,
                                                    r, ld64, n_rows, delta, UPD_BLOCKS, partial, err, st, ds, nullptr,
                                                    nullptr, r_dev);
    }
  } else if (Utf && Vf32) {
    DualArgs<float> ds{};
    if (dual) {
      ds = {(const float*)dual->yp_in, (const float*)dual->ym_in, (float*)dual->yp_out, (float*)dual->ym_out, dual->E};
      sddmm_dispatch<float, float, float, true>(row_ptr, col_idx, csr_to_csc, (const float*)M, nullptr,
                                                (float*)y_out, (float*)y_out_csc, Utf, Vf32, r, ldf, n_rows,
                                                (float)delta, UPD_BLOCKS, partial, err, st, ds, ys, ysc, r_dev);
    } else {
      sddmm_dispatch<float, float, float, false>(row_ptr, col_idx, csr_to_csc, (const float*)M, (const float*)y_in,
                                                 (float*)y_out, (float*)y_out_csc, Utf, Vf32, r, ldf, n_rows,
                                                 (float)delta, UPD_BLOCKS, partial, err, st, ds, ys, ysc, r_dev);
    }
  } else {
    if (dual) return 0;   // the two-multiplier form runs only with the float32 copies of the factors
    DualArgs<float> ds{};
    sddmm_dispatch<float, float, double, false>(row_ptr, col_idx, csr_to_csc, (const float*)M, (const float*)y_in,
                                                (float*)y_out, (float*)y_out_csc, Ut, V, r, ld64, n_rows, (float)delta,
                                                UPD_BLOCKS, partial, err, st, ds, nullptr, nullptr, r_dev);
  }
  k_sum_fixed<<<1, 1024, 0, st>>>(partial, UPD_BLOCKS, res2);
  return 2;
}

// ------------------------------------------------------------------------------------------------
// Fused update over a job list (batched engine): tiles of 64 rows; the tiles of all jobs form one
// index space, taken grid-stride by a persistent grid.  Each tile's e^2 sum goes to partial[tile];
// k_sum_jobs then adds the partials of each job in tile order (one CTA per job).  Entry values are
// computed exactly as k_sddmm_update computes them; only the grouping of the residual sum differs.
// ------------------------------------------------------------------------------------------------
static constexpr int UPD_TILE_ROWS = 64;

long long upd_jobs_tiles(const int* m, int n) {
  long long t = 0;
  for (int k = 0; k < n; ++k) t += (m[k] + UPD_TILE_ROWS - 1) / UPD_TILE_ROWS;
  return t;
}

template <typename VT, typename AT, typename FT, int RMAX>
__global__ void __launch_bounds__(UPD_THREADS)
k_sddmm_update_jobs(const __grid_constant__ UpdJobTable tab, double* __restrict__ partial, unsigned int* err) {
  __shared__ double red[UPD_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  const DualArgs<VT> ds{};
  for (int t = blockIdx.x; t < tab.tiles; t += gridDim.x) {
    int k = 0;
    while (k + 1 < tab.n && tab.job[k + 1].tile0 <= t) ++k;
    const UpdJobDev& J = tab.job[k];
    const int i0 = (t - J.tile0) * UPD_TILE_ROWS;
    const int i1 = min(J.m, i0 + UPD_TILE_ROWS);
    AT acc = (AT)0;
    for (int i = i0 + warp; i < i1; i += warps)
      upd_row<VT, AT, FT, RMAX, false>(i, lane, J.row_ptr, J.col_idx, J.csr_to_csc, static_cast<const VT*>(J.M),
                                       static_cast<const VT*>(J.y_in), static_cast<VT*>(J.y_out),
                                       static_cast<VT*>(J.y_out_csc), static_cast<const FT*>(J.Ut),
                                       static_cast<const FT*>(J.V), J.r, J.ldf, (AT)J.delta, ds, nullptr, nullptr, acc);
    const double accd = warp_sum((double)acc);
    if (lane == 0) red[warp] = accd;
    __syncthreads();
    if (threadIdx.x < 32) {
      double v = threadIdx.x < warps ? red[threadIdx.x] : 0.0;
      v = warp_sum(v);
      if (threadIdx.x == 0) {
        partial[t] = v;
        if (!isfinite(v)) svt_set_error(err, SVT_DEVERR_NONFINITE);
      }
    }
    __syncthreads();
  }
}

__global__ void k_sum_jobs(const __grid_constant__ UpdJobTable tab, const double* __restrict__ partial) {
  __shared__ double red[32];
  const int k = blockIdx.x;
  const int t0 = tab.job[k].tile0, t1 = k + 1 < tab.n ? tab.job[k + 1].tile0 : tab.tiles;
  double acc = 0.0;
  for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) acc += partial[t];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *tab.job[k].res2 = v;
  }
}

template <typename VT, typename AT, typename FT>
static void upd_jobs_dispatch(const UpdJobTable& tab, int rmax, int blocks, double* partial, unsigned int* err,
                              cudaStream_t st) {
  if (rmax <= 16) k_sddmm_update_jobs<VT, AT, FT, 16><<<blocks, UPD_THREADS, 0, st>>>(tab, partial, err);
  else if (rmax <= 32) k_sddmm_update_jobs<VT, AT, FT, 32><<<blocks, UPD_THREADS, 0, st>>>(tab, partial, err);
  else k_sddmm_update_jobs<VT, AT, FT, 64><<<blocks, UPD_THREADS, 0, st>>>(tab, partial, err);
}

int launch_sddmm_update_jobs(int precision, const UpdJob* jobs, int n, double* partial, long long partial_cap,
                             unsigned int* err, int grid, cudaStream_t st) {
  if (n <= 0 || n > kBatchMaxJobs || precision == 2) return 0;
  UpdJobTable tab{};
  int tiles = 0, rmax = 0;
  for (int k = 0; k < n; ++k) {
    const UpdJob& J = jobs[k];
    if (J.m <= 0 || J.r < 0 || J.r > 64 || !J.res2) return 0;
    UpdJobDev& d = tab.job[tab.n++];
    d.row_ptr = J.row_ptr; d.col_idx = J.col_idx; d.csr_to_csc = J.csr_to_csc; d.M = J.M; d.y_in = J.y_in;
    d.y_out = J.y_out; d.y_out_csc = J.y_out_csc; d.Ut = J.Ut; d.V = J.V; d.res2 = J.res2; d.delta = J.delta;
    d.r = J.r; d.ldf = J.ldf > 0 ? J.ldf : J.r; d.m = J.m; d.tile0 = tiles;
    tiles += (J.m + UPD_TILE_ROWS - 1) / UPD_TILE_ROWS;
    rmax = std::max(rmax, J.r);
  }
  if (tiles > partial_cap) return 0;
  tab.tiles = tiles;
  const int blocks = std::max(1, std::min(tiles, grid > 0 ? grid : UPD_BLOCKS));
  if (precision == 0) upd_jobs_dispatch<double, double, double>(tab, rmax, blocks, partial, err, st);
  else upd_jobs_dispatch<float, float, float>(tab, rmax, blocks, partial, err, st);
  k_sum_jobs<<<tab.n, 256, 0, st>>>(tab, partial);
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

// bfloat16 copies (round to nearest) of float32 values, row-major and column-major order.
__global__ void k_to_bf16(const float* __restrict__ y, const float* __restrict__ y_csc, __nv_bfloat16* __restrict__ yb,
                          __nv_bfloat16* __restrict__ yb_csc, long long nnz) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x) {
    yb[p] = __float2bfloat16_rn(y[p]);
    yb_csc[p] = __float2bfloat16_rn(y_csc[p]);
  }
}

int launch_to_bf16(const float* y, const float* y_csc, void* yb, void* yb_csc, long long nnz, cudaStream_t st) {
  int blocks = (int)svt_min_ll(svt_ceil_div(nnz, 256), 152LL * 16);
  if (blocks < 1) return 0;
  k_to_bf16<<<blocks, 256, 0, st>>>(y, y_csc, (__nv_bfloat16*)yb, (__nv_bfloat16*)yb_csc, nnz);
  return 1;
}

// Dantzig-selector kick (Sec. 3.3 with the device of Sec. 5.1.3): y = alpha soft_E(B) (row-major and
// column-major), and, when yp / ym are given, yp = alpha [B - E]_+ and ym = alpha [-B - E]_+.
template <typename VT>
__global__ void k_dual_kick(const VT* __restrict__ B, double alpha, double E, VT* __restrict__ y,
                            VT* __restrict__ y_csc, VT* __restrict__ yp, VT* __restrict__ ym,
                            const int32_t* __restrict__ csr_to_csc, long long nnz) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x) {
    const double b = (double)B[p];
    const double up = fmax(b - E, 0.0), dn = fmax(-b - E, 0.0);
    const VT v = (VT)(alpha * up - alpha * dn);
    y[p] = v;
    if (y_csc) y_csc[csr_to_csc[p]] = v;
    if (yp) yp[p] = (VT)(alpha * up);
    if (ym) ym[p] = (VT)(alpha * dn);
  }
}

int launch_dual_kick(int precision, const void* B, double alpha, double E, void* y, void* y_csc, void* yp, void* ym,
                     const int32_t* csr_to_csc, long long nnz, cudaStream_t st) {
  int blocks = (int)svt_min_ll(svt_ceil_div(nnz, 256), 152LL * 16);
  if (blocks < 1) return 0;
  if (precision == 0)
    k_dual_kick<double><<<blocks, 256, 0, st>>>((const double*)B, alpha, E, (double*)y, (double*)y_csc, (double*)yp,
                                                (double*)ym, csr_to_csc, nnz);
  else
    k_dual_kick<float><<<blocks, 256, 0, st>>>((const float*)B, alpha, E, (float*)y, (float*)y_csc, (float*)yp,
                                               (float*)ym, csr_to_csc, nnz);
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
  sddmm_dispatch<double, double, double, false>(row_ptr, col_idx, nullptr, M, y_in, y_out, nullptr, Ut, V, r, r,
                                                n_rows, delta, blocks, partial, nullptr, st, DualArgs<double>{}, nullptr,
                                                nullptr);
  k_sum_fixed<<<1, 1024, 0, st>>>(partial, blocks, res2);
  return 2;
}

}  // namespace svt
