// Projected SVD of the Lanczos partial SVD: T (K x K, K = J b <= 96) = Xl diag(theta) Wr^T by the
// one-sided (Hestenes) Jacobi method, in one CTA.  Sec. 5.1.1: the singular values of the small
// projected matrix are the Ritz values of Y, compared against tau by the rank policy.
//
// Layout: columns of G (= T, rotated in place) and of W (the accumulated rotations) live in shared
// memory, column-major.  One warp per column pair: in each of the K-1 rounds of a sweep the K/2
// disjoint pairs of a round-robin tournament are rotated in parallel; a warp holds its two columns
// of G and W in registers (rows lane, lane+32, lane+64), reduces the three inner products with
// butterfly shuffles, rotates and writes back; one barrier per round.
//
// Two arithmetic variants:
//   * float64 path: rotations in float64.  GB300's float64 divide and square root take ~650
//     cycles each, so the rotation parameters use float32 reciprocal / reciprocal-square-root
//     seeds refined by Newton steps in float64 (two steps for the cosine, which keeps every
//     rotation orthogonal to float64 rounding).
//   * float32 path: rotations in float32 (the float64 rate is 1/64 of float32 on GB300); then, for
//     the leading nvec right vectors w (renormalised in float64), theta = ||T w|| and
//     x = T w / theta are formed in float64, so the values compared against tau are float64
//     Rayleigh quotients, exact to second order in the float32 angle error of w.  The rotations act
//     on the rows of T (the columns of T^T), so the rotated columns are the right vectors; the
//     rotations themselves (the left vectors) are not accumulated.
// Residual estimates of the Lanczos relation: res_k = || S x_k[last b rows] || with S the b x b
// upper triangular factor of the last block (Y^T U_J = V T^T + V_{J+1} S E_J^T).
#include <cooperative_groups.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace svt {

static constexpr int JMAXK = 128;
// 1: the float32-rotation variant rotates the rows of T (one-sided Jacobi on T^T).  T is upper
// triangular (block bidiagonal with triangular diagonal blocks, leading diagonal graded by the
// warm start), and on its rows the sweeps converge in ~10% fewer sweeps than on its columns.
static constexpr int kJacobiOnRows = 1;

// Reciprocal and reciprocal square root in float64 by Newton's iteration from the float32 hardware
// approximations (GB300's float64 divide and square root take ~650 cycles): each step squares the
// relative error, 2^-23 -> ~1e-14 -> rounding.
__device__ __forceinline__ double rcp_nr(double x) {
  double y = (double)__frcp_rn((float)x);
  y = y * (2.0 - x * y);
  y = y * (2.0 - x * y);
  return y;
}
__device__ __forceinline__ double rcp_nr1(double x) {
  const double y = (double)__frcp_rn((float)x);
  return y * (2.0 - x * y);
}
__device__ __forceinline__ double rsqrt_nr(double x, int steps) {
  double y = (double)rsqrtf((float)x);
  for (int i = 0; i < steps; ++i) y = y * (1.5 - 0.5 * x * y * y);
  return y;
}

template <typename R>
struct Rot;

template <>
struct Rot<float> {
  // zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2),
  // from the hardware reciprocal / reciprocal-square-root approximations (a few ulp): c^2 + s^2 = 1
  // to ~1e-7, the level of the float32 rotations themselves.  For |zeta| >= 2^40, sqrt(1 + zeta^2)
  // is taken as |zeta| (t ~ 1 / (2 zeta)), which also keeps zeta^2 clear of overflow.
  static __device__ __forceinline__ void params(float al, float be, float ga, float& c, float& s, float& t) {
    const float zeta = __fdividef(be - al, 2.f * ga);
    const float az = fabsf(zeta);
    const float z2 = fmaf(zeta, zeta, 1.f);
    const float h = az < 1.0995116e12f ? z2 * rsqrtf(z2) : az;
    t = copysignf(__fdividef(1.f, az + h), zeta);
    c = rsqrtf(fmaf(t, t, 1.f));
    s = c * t;
  }
  // |cos| of the angle between the two columns (a few ulp; only compared with the tolerance)
  static __device__ __forceinline__ float cosang(float al, float be, float ga) {
    return fabsf(ga) * (rsqrtf(al) * rsqrtf(be));
  }
};

template <>
struct Rot<double> {
  // One Newton step on each float32 seed (reciprocal y <- y (2 - x y), reciprocal square root
  // y <- y (3/2 - x y^2 / 2)): relative errors ~1e-14, so c^2 + s^2 = 1 to ~1e-14 -- ample for the
  // finishing sweep, whose rotations are within 1e-5 of the identity -- with half the dependent
  // float64 operations of two steps.
  static __device__ __forceinline__ void params(double al, double be, double ga, double& c, double& s, double& t) {
    const double zeta = (be - al) * rcp_nr1(2.0 * ga);
    const double z2 = fma(zeta, zeta, 1.0);
    const double h = z2 * rsqrt_nr(z2, 1);                 // sqrt(1 + zeta^2)
    t = copysign(1.0, zeta) * rcp_nr1(fabs(zeta) + h);
    c = rsqrt_nr(fma(t, t, 1.0), 1);
    s = c * t;
  }
  static __device__ __forceinline__ double cosang(double al, double be, double ga) {
    return fabs(ga) / (sqrt(al) * sqrt(be));
  }
};

__device__ __forceinline__ float shfl_xor_r(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor_r(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }

// Sweeps of the one-sided Jacobi method on G (K x K, column-major in shared memory), accumulating
// the rotations in W when ACC (otherwise W is not touched).  JL lanes per column pair (JR = ceil(96 / JL) rows each), 32 / JL pairs per
// warp: the rotation parameters of four pairs come out of one warp instruction, and the inner
// products need only log2(JL) butterfly steps.  Returns the number of sweeps taken.
static constexpr int JL = 8;

template <typename R>
__device__ __forceinline__ R shfl_grp(R v, int o) { return shfl_xor_r(v, o); }

// TRACK: the squared column norms are kept in nrm2 (shared memory, filled by the caller) and
// updated by every rotation (al' = al - t ga, be' = be + t ga with t = s / c), so a pair needs one
// inner product instead of three.
// JLv: lanes per pair (JL by default; fewer lanes put more pairs in one warp instruction, which
// pays where the instruction count is the bound: the float64 pipe).
template <typename R, int JR, bool ACC, bool TRACK = false, int JLv = JL>   // JR = rows per lane = ceil(K / JLv)
__device__ int jacobi_sweeps(R* G, R* W, const unsigned char* sched, int K, R tol, int max_sweeps, int* flag,
                             bool quad_stop = false, R* nrm2 = nullptr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gl = lane & (JLv - 1);                // lane inside the pair group
  const int gsub = lane / JLv;                    // pair slot inside the warp
  const int npairs = K / 2;
  __shared__ float warp_max[32];   // per-warp largest |cos| between a rotated pair in this sweep
  int sweep = 0;
  bool final_sweep = false;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    float my_max = 0.f;   // this lane's largest |cos| over the pairs it rotated in this sweep
    __syncthreads();
    for (int round = 0; round < K - 1; ++round) {
      const unsigned char* rs = sched + 2 * round * npairs;
      for (int base = warp * (32 / JLv); base < npairs; base += nw * (32 / JLv)) {   // warp-uniform
        const int pr = base + gsub;
        const bool has = pr < npairs;
        const int p = has ? rs[2 * pr] : 0, q = has ? rs[2 * pr + 1] : 0;
        R* gp = G + p * K;
        R* gq = G + q * K;
        R* wp = W + p * K;
        R* wq = W + q * K;
        // the rows of both columns of G and of W are loaded together, before the inner products,
        // so the W loads are not on the critical path when the pair is rotated
        R a[JR], bq[JR], wa[JR], wb[JR];
        R al = 0, be = 0, ga = 0;
#pragma unroll
        for (int k = 0; k < JR; ++k) {
          const int r = gl + JLv * k;
          const bool in = has && r < K;
          a[k] = in ? gp[r] : R(0);
          bq[k] = in ? gq[r] : R(0);
          wa[k] = (ACC && in) ? wp[r] : R(0);
          wb[k] = (ACC && in) ? wq[r] : R(0);
        }
#pragma unroll
        for (int k = 0; k < JR; ++k) {
          if (!TRACK) {
            al += a[k] * a[k];
            be += bq[k] * bq[k];
          }
          ga += a[k] * bq[k];
        }
#pragma unroll
        for (int o = 1; o < JLv; o <<= 1) {
          if (!TRACK) {
            al += shfl_grp(al, o);
            be += shfl_grp(be, o);
          }
          ga += shfl_grp(ga, o);
        }
        if (TRACK && has) {
          al = nrm2[p];
          be = nrm2[q];
        }
        if (has && ga != R(0)) {
          const R cs = Rot<R>::cosang(al, be, ga);
          if (cs > tol) {
            my_max = fmaxf(my_max, (float)cs);
            R c, s, t;
            Rot<R>::params(al, be, ga, c, s, t);
            if (TRACK && gl == 0) {
              nrm2[p] = al - t * ga;
              nrm2[q] = be + t * ga;
            }
#pragma unroll
            for (int k = 0; k < JR; ++k) {
              const int r = gl + JLv * k;
              if (r < K) {
                gp[r] = c * a[k] - s * bq[k];
                gq[r] = s * a[k] + c * bq[k];
                if (ACC) {
                  wp[r] = c * wa[k] - s * wb[k];
                  wq[r] = s * wa[k] + c * wb[k];
                }
              }
            }
            if (gl == 0) *flag = 1;
          }
        }
      }
      __syncthreads();
    }
    // largest |cos| of the sweep over all lanes
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_max = fmaxf(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
    if (lane == 0) warp_max[warp] = my_max;
    __syncthreads();
    float sweep_max = 0.f;
    for (int w = 0; w < nw; ++w) sweep_max = fmaxf(sweep_max, warp_max[w]);
    if (!*flag || final_sweep) break;
    // quadratic convergence: once every rotated pair had |cos| <= sqrt(tol), the next sweep leaves
    // them at the tol level, so it is the last one (no further verification sweep); with quad_stop
    // the sweep that rotated them is already the last
    final_sweep = sweep_max <= (float)sqrt(tol);
    if (quad_stop && final_sweep) break;
    __syncthreads();
  }
  return sweep + 1;
}

// Round-robin tournament: in round r, pair 0 is (K-1, r) and pair i >= 1 is
// ((r + i) mod (K-1), (r - i) mod (K-1)); every pair of columns meets once per sweep.
__device__ void build_schedule(unsigned char* sched, int K) {
  const int npairs = K / 2;
  for (int e = threadIdx.x; e < (K - 1) * npairs; e += blockDim.x) {
    const int round = e / npairs, i = e - round * npairs;
    int p, q;
    if (i == 0) { p = K - 1; q = round; }
    else { p = (round + i) % (K - 1); q = (round - i + (K - 1)) % (K - 1); }
    if (p > q) { int x = p; p = q; q = x; }
    sched[2 * e] = (unsigned char)p;
    sched[2 * e + 1] = (unsigned char)q;
  }
}

// Rank of every column norm (decreasing, ties by index) -> order[rank] = column.
template <typename R>
__device__ void sort_columns(const R* nrm, int* order, int K) {
  for (int c = threadIdx.x; c < K; c += blockDim.x) {
    int rank = 0;
    for (int c2 = 0; c2 < K; ++c2)
      if (nrm[c2] > nrm[c] || (nrm[c2] == nrm[c] && c2 < c)) ++rank;
    order[rank] = c;
  }
}

// ------------------------------------------------------------------------------------------------
// float64 path
// ------------------------------------------------------------------------------------------------
// float64 path in two phases.  One float64 rotation costs ~20 dependent float64 operations and its
// column updates run on the float64 pipe (2 FMA per clock per SM on GB300), so full float64 sweeps
// from T take milliseconds.  Instead:
//   A. float32 sweeps on the columns of T with the rotations accumulated in W (float32), until
//      every pair has |cos| <= 2e-6;
//   B. in float64: W <- W (I - (W^T W - I) / 2) (one first-order step back to orthonormality,
//      ~1e-12), G = T W, and float64 sweeps on G from there (column norms tracked through the
//      rotations, W not rotated, four lanes per pair): quadratic convergence takes |cos| from
//      2e-6 to ~1e-11 in one sweep, and a sweep whose pairs all had |cos| <= sqrt(tol) is the
//      last (the caller's tol is 1e-11: Ritz vectors far more accurate than the Lanczos
//      tolerance of 1e-6 sigma_1 they are tested against).  The right vectors of the leading
//      b triplets are then w = T^T g / ||g||^2 for the final columns g = theta x of G.
// The result is a float64 one-sided Jacobi SVD of T; phase A only supplies its starting rotation.
//
// Launched as a thread-block cluster (launch_small_svd: 8 CTAs where the device allows it), the
// dense float64 products are spread over the cluster: CTA 0 holds G / W, the column norms and the
// order in its shared memory and runs phase A and the sweeps alone; E = W^T W - I (entries), W's
// correction (rows), G = T W (columns), the norms of G, the right vectors (entries) and the
// residual estimates (triplets) are shared by all CTAs through distributed shared memory, with a
// cluster barrier between phases.  (Sweeps spread over the cluster, one warp per pair and a cluster
// barrier per round, measured slower: ~12k cycles a round against ~10k in one CTA.)  With one CTA
// the kernel is the single-CTA form.
template <int JR>
__global__ void __launch_bounds__(512)
k_jacobi_f64(const double* __restrict__ T, int ldT, int K, const double* __restrict__ S, int b, int nv,
             double* __restrict__ theta, double* __restrict__ Xl, double* __restrict__ Wr, double* __restrict__ res,
             double tol, int max_sweeps, unsigned int* err, unsigned long long* counters) {
  extern __shared__ double sm64[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), nct = (int)cl.num_blocks();
  auto csync = [&]() {
    if (nct > 1) cl.sync();
    else __syncthreads();
  };
  // One K x K region: phase A keeps its float32 G32 and W32 there, phase B the float64 W, then
  // G = T W in its place (column by column); E = W^T W - I is kept in Xl (global) until Xl is
  // written at the end.
  double* G = sm64;                   // K x K column-major
  double* nrm = G + K * K;            // K
  double* rnrm = nrm + K;             // K: 1 / nrm (0 for a zero column)
  int* order = (int*)(rnrm + K);      // K
  unsigned char* sched = (unsigned char*)(order + K);
  __shared__ int flag;
  // CTA 0's arrays as every CTA of the cluster addresses them
  double* G0 = nct > 1 ? cl.map_shared_rank(G, 0) : G;
  double* nrm0 = nct > 1 ? cl.map_shared_rank(nrm, 0) : nrm;
  build_schedule(sched, K);
  int sweeps_a = 0;
  if (rank == 0) {
    float* G32 = (float*)G;
    float* W32 = G32 + K * K;
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
      const int i = e / K, c = e - i * K;
      G32[c * K + i] = (float)T[i * ldT + c];
      W32[c * K + i] = (i == c) ? 1.f : 0.f;
    }
    __syncthreads();
    // A. float32 sweeps (the float32 rounding level of the angles)
    sweeps_a = jacobi_sweeps<float, JR, true>(G32, W32, sched, K, 2e-6f, max_sweeps, &flag);
    // W (float64) <- W32, in place: W[e] overwrites W32 entries of smaller index only, so chunks of
    // one entry per thread are read, then written
    for (int e0 = 0; e0 < K * K; e0 += blockDim.x) {
      const int e = e0 + threadIdx.x;
      const float v = e < K * K ? W32[e] : 0.f;
      __syncthreads();
      if (e < K * K) G[e] = (double)v;
      __syncthreads();
    }
  }
  csync();
  double* W = G0;
  // work of the float64 phases spread over the cluster's threads / warps
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gtid = rank * blockDim.x + threadIdx.x, gthreads = nct * blockDim.x;
  const int gwarp = rank * nw + warp, gwarps = nct * nw;
  // B1. E = W^T W - I (into Xl, global, symmetric), then W <- W (I - E / 2) row by row (a row of the
  // new W needs only the same row of the old one)
  double* E = Xl;
  for (int e = gtid; e < K * K; e += gthreads) {
    const int p = e / K, q = e - p * K;
    if (q < p) continue;
    const double* wp = W + p * K;
    const double* wq = W + q * K;
    double s0 = 0.0, s1 = 0.0;
    int i = 0;
    for (; i + 1 < K; i += 2) {
      s0 = fma(wp[i], wq[i], s0);
      s1 = fma(wp[i + 1], wq[i + 1], s1);
    }
    if (i < K) s0 = fma(wp[i], wq[i], s0);
    const double v = (s0 + s1) - (p == q ? 1.0 : 0.0);
    E[q * K + p] = v;
    E[p * K + q] = v;
  }
  csync();
  constexpr int NT = (JMAXK + 31) / 32;
  for (int i = gwarp; i < K; i += gwarps) {
    double wi[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int c = lane + 32 * t;
      wi[t] = c < K ? W[c * K + i] : 0.0;
    }
    double out[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) out[t] = wi[t];
#pragma unroll
    for (int tk = 0; tk < NT; ++tk) {
      for (int kk = 0; kk < 32; ++kk) {
        const int k = 32 * tk + kk;
        const double wk = __shfl_sync(0xffffffffu, wi[tk], kk);   // W[i, k], held by lane kk
        if (k >= K) break;                                         // warp-uniform
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const int c = lane + 32 * t;
          if (c < K) out[t] = fma(-0.5 * wk, __ldcg(E + k * K + c), out[t]);
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int c = lane + 32 * t;
      if (c < K) W[c * K + i] = out[t];
    }
  }
  csync();
  // B2. G = T W, one column per warp in place (T block upper triangular: row i has no entries left
  // of its diagonal block)
  for (int c = gwarp; c < K; c += gwarps) {
    const double* wc = W + c * K;
    double g[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int i = lane + 32 * t;
      double s0 = 0.0, s1 = 0.0;
      if (i < K) {
        const double* trow = T + (long long)i * ldT;
        int k = (i / b) * b;
        for (; k + 1 < K; k += 2) {
          s0 = fma(trow[k], wc[k], s0);
          s1 = fma(trow[k + 1], wc[k + 1], s1);
        }
        if (k < K) s0 = fma(trow[k], wc[k], s0);
      }
      g[t] = s0 + s1;
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int i = lane + 32 * t;
      if (i < K) G0[c * K + i] = g[t];
    }
  }
  csync();
  // B3. float64 sweeps from the float32-level angles on G alone (tracked column norms); the right
  // vectors are formed afterwards from T^T
  for (int c = gwarp; c < K; c += gwarps) {
    double s2 = 0.0;
    for (int i = lane; i < K; i += 32) s2 = fma(G0[c * K + i], G0[c * K + i], s2);
    s2 = warp_sum(s2);
    if (lane == 0) nrm0[c] = s2;
  }
  csync();
  int sweeps_b = 0;
  if (rank == 0) {
    if constexpr (JR <= 6)
      sweeps_b = jacobi_sweeps<double, 2 * JR, false, true, JL / 2>(G, G, sched, K, tol, max_sweeps, &flag, true, nrm);
    else
      sweeps_b = jacobi_sweeps<double, JR, false, true, JL>(G, G, sched, K, tol, max_sweeps, &flag, true, nrm);
    const int sweeps = sweeps_a + sweeps_b;
    if (threadIdx.x == 0) {
      if (sweeps_a > max_sweeps || sweeps_b > max_sweeps) svt_set_error(err, SVT_DEVERR_JACOBI);
      if (counters) {
        atomicAdd(&counters[0], 1ULL);
        atomicAdd(&counters[1], (unsigned long long)sweeps);
      }
    }
    // column norms (one warp per column)
    for (int c = warp; c < K; c += nw) {
      double s2 = 0.0;
      for (int i = lane; i < K; i += 32) s2 = fma(G[c * K + i], G[c * K + i], s2);
      s2 = warp_sum(s2);
      if (lane == 0) {
        const double th = s2 > 0.0 ? s2 * rsqrt_nr(s2, 2) : 0.0;
        nrm[c] = th;
        rnrm[c] = th > 0.0 ? rcp_nr(th) : 0.0;
      }
    }
    __syncthreads();
    sort_columns<double>(nrm, order, K);
    __syncthreads();
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
      const int i = e / K, k = e - i * K;
      const int c = order[k];
      Xl[i * K + k] = G[c * K + i] * rnrm[c];
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) theta[k] = nrm[order[k]];
  }
  csync();
  const double* rn0 = nct > 1 ? cl.map_shared_rank(rnrm, 0) : rnrm;
  const int* ord0 = nct > 1 ? cl.map_shared_rank(order, 0) : order;
  // right vectors of the leading nv triplets: w_k = T^T x_k / theta_k = T^T g_k / theta_k^2 (column
  // i of T has no entries below its diagonal block); the others are not used by the solver and are
  // left zero
  if (nv > K) nv = K;
  for (int e = gtid; e < K * K; e += gthreads) {
    const int i = e / K, k = e - i * K;
    double v = 0.0;
    if (k < nv) {
      const int c = ord0[k];
      const double* gc = G0 + c * K;
      const int rend = min(K, (i / b + 1) * b);
      double s0 = 0.0, s1 = 0.0;
      int r = 0;
      for (; r + 1 < rend; r += 2) {
        s0 = fma(T[(long long)r * ldT + i], gc[r], s0);
        s1 = fma(T[(long long)(r + 1) * ldT + i], gc[r + 1], s1);
      }
      if (r < rend) s0 = fma(T[(long long)r * ldT + i], gc[r], s0);
      const double rc = rn0[c];
      v = (s0 + s1) * (rc * rc);
    }
    Wr[i * K + k] = v;
  }
  // residual estimates, one warp per triplet
  for (int k = gwarp; k < K; k += gwarps) {
    double r2 = 0.0;
    if (S) {
      const int c = ord0[k];
      const double inv = rn0[c];
      for (int e = lane; e < b; e += 32) {
        double v = 0.0;
        for (int d = e; d < b; ++d) v = fma(S[e * b + d], G0[c * K + (K - b + d)], v);
        v *= inv;
        r2 = fma(v, v, r2);
      }
      r2 = warp_sum(r2);
    }
    if (lane == 0) res[k] = sqrt(r2);
  }
  // CTA 0's shared memory is read until here
  csync();
}

// ------------------------------------------------------------------------------------------------
// float32 rotations + float64 Ritz values
// ------------------------------------------------------------------------------------------------
template <int JR>
__global__ void __launch_bounds__(512)
k_jacobi_mixed(const double* __restrict__ T, int ldT, int K, double* __restrict__ theta, double* __restrict__ Xl,
               double* __restrict__ Wr, double* __restrict__ res, int nvec, float* __restrict__ wsrc, float tol,
               int max_sweeps, unsigned int* err, unsigned long long* counters, int trans) {
  extern __shared__ double smm[];
  float* G = (float*)smm;                   // K x K column-major
  float* W = G + K * K;                     // K x K column-major
  float* nrm = W + K * K;                   // K
  int* order = (int*)(nrm + K);             // K
  unsigned char* sched = (unsigned char*)(order + K);
  __shared__ int flag;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int i = e / K, c = e - i * K;
    const double v = T[i * ldT + c];
    // trans: the rotations act on the rows of T (the columns of T^T)
    if (trans) G[i * K + c] = (float)v;
    else G[c * K + i] = (float)v;
    if (!trans) W[c * K + i] = (i == c) ? 1.f : 0.f;
  }
  build_schedule(sched, K);
  __syncthreads();
  // with trans the accumulated rotations would be the left vectors, which are formed in float64
  // from T w for the leading nvec triplets instead: W is not accumulated
  const int sweeps = trans ? jacobi_sweeps<float, JR, false>(G, W, sched, K, tol, max_sweeps, &flag)
                           : jacobi_sweeps<float, JR, true>(G, W, sched, K, tol, max_sweeps, &flag);
  if (threadIdx.x == 0) {
    if (sweeps > max_sweeps) svt_set_error(err, SVT_DEVERR_JACOBI);
    if (counters) {
      atomicAdd(&counters[0], 1ULL);
      atomicAdd(&counters[1], (unsigned long long)sweeps);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < K; c += nw) {
    float s2 = 0.f;
    for (int i = lane; i < K; i += 32) s2 = fmaf(G[c * K + i], G[c * K + i], s2);
    s2 = warp_sum(s2);
    if (lane == 0) nrm[c] = sqrtf(s2);
  }
  __syncthreads();
  sort_columns<float>(nrm, order, K);
  __syncthreads();
  // right singular vectors of T: the accumulated rotations W, or with trans the rotated columns
  // of T^T; the leading nvec go to wsrc (float32, in decreasing order) for the float64 refinement
  const float* Rv = trans ? G : W;
  const float* Lv = trans ? W : G;
  for (int e = threadIdx.x; e < nvec * K; e += blockDim.x) {
    const int k = e / K, i = e - k * K;
    wsrc[e] = Rv[order[k] * K + i];
  }
  // remaining triplets (not used by the rank policy, the restart or the shrink): float32 values
  // and right vectors; with trans no left vectors (zero columns of Xl)
  for (int e = threadIdx.x; e < (K - nvec) * K; e += blockDim.x) {
    const int kk = nvec + e / K, i = e % K;
    const int c = order[kk];
    const float th = nrm[c];
    Xl[i * K + kk] = trans ? 0.0 : (th > 0.f ? (double)(Lv[c * K + i] / th) : 0.0);
    Wr[i * K + kk] = trans ? (th > 0.f ? (double)(Rv[c * K + i] / th) : 0.0) : (double)Rv[c * K + i];
  }
  for (int kk = nvec + threadIdx.x; kk < K; kk += blockDim.x) {
    theta[kk] = (double)nrm[order[kk]];
    res[kk] = INFINITY;
  }
}

// Float64 Ritz triplets of the leading nvec right vectors of the float32 Jacobi: one CTA per
// triplet k (spread over SMs: GB300 runs float64 at 2 FMA per clock per SM).  w = wsrc_k
// normalised, x = T w / theta with theta = ||T w|| (a Rayleigh value, exact to second order in the
// float32 angle error of w), and the Lanczos residual estimate res_k = || S x[last b rows] ||.
__global__ void __launch_bounds__(128)
k_ritz_refine(const double* __restrict__ T, int ldT, int K, const double* __restrict__ S, int b,
              const float* __restrict__ wsrc, double* __restrict__ theta, double* __restrict__ Xl,
              double* __restrict__ Wr, double* __restrict__ res) {
  __shared__ double wv[JMAXK];
  __shared__ double gx[JMAXK];
  const int k = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* w = wsrc + (long long)k * K;
  if (warp == 0) {
    double s2 = 0.0;
    for (int i = lane; i < K; i += 32) {
      const double v = (double)w[i];
      s2 += v * v;
    }
    s2 = warp_sum(s2);
    const double inv = rsqrt_nr(s2, 2);
    for (int i = lane; i < K; i += 32) wv[i] = (double)w[i] * inv;
  }
  __syncthreads();
  // T w: one thread per row, four independent accumulation chains
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    const double* trow = T + (long long)i * ldT;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    int cc = 0;
    for (; cc + 3 < K; cc += 4) {
      v0 += trow[cc] * wv[cc];
      v1 += trow[cc + 1] * wv[cc + 1];
      v2 += trow[cc + 2] * wv[cc + 2];
      v3 += trow[cc + 3] * wv[cc + 3];
    }
    for (; cc < K; ++cc) v0 += trow[cc] * wv[cc];
    gx[i] = (v0 + v1) + (v2 + v3);
  }
  __syncthreads();
  if (warp != 0) return;
  double s2 = 0.0;
  for (int i = lane; i < K; i += 32) s2 += gx[i] * gx[i];
  s2 = warp_sum(s2);
  const double th = s2 > 0.0 ? s2 * rsqrt_nr(s2, 2) : 0.0;
  const double inv = th > 0.0 ? rcp_nr(th) : 0.0;
  for (int i = lane; i < K; i += 32) {
    Xl[i * K + k] = gx[i] * inv;
    Wr[i * K + k] = wv[i];
  }
  if (lane == 0) theta[k] = th;
  double r2 = 0.0;
  if (S) {
    for (int e2 = lane; e2 < b; e2 += 32) {
      double v = 0.0;
      for (int d = e2; d < b; ++d) v += S[e2 * b + d] * gx[K - b + d];
      v *= inv;
      r2 += v * v;
    }
    r2 = warp_sum(r2);
  }
  if (lane == 0) res[k] = sqrt(r2);
}

// Self-test of the Newton reciprocal / reciprocal-square-root helpers: out[5 i + 0..3] =
// rcp_nr(x_i), rcp_nr1(x_i), rsqrt_nr(x_i, 2), rsqrt_nr(x_i, 1) (slot 4 is the orthonormalisation's
// pivot helper, filled by launch_pivot_selftest).
__global__ void k_newton_selftest(const double* __restrict__ x, long long n, double* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    out[5 * i + 0] = rcp_nr(v);
    out[5 * i + 1] = rcp_nr1(v);
    out[5 * i + 2] = rsqrt_nr(v, 2);
    out[5 * i + 3] = rsqrt_nr(v, 1);
  }
}

int launch_newton_selftest(const double* x, long long n, double* out, cudaStream_t st) {
  if (n <= 0) return 0;
  const int blocks = (int)svt_min_ll(svt_ceil_div(n, 256), 152LL * 4);
  k_newton_selftest<<<blocks, 256, 0, st>>>(x, n, out);
  return 1;
}

static int jacobi_threads(int K) {
  // one pair per JL lanes, at least 8 warps for the epilogue loops
  int warps = (K / 2 + (32 / JL) - 1) / (32 / JL);
  if (warps < 8) warps = 8;
  if (warps > 16) warps = 16;   // launch bound 512 threads (K <= 128 needs at most 16 warps)
  return 32 * warps;
}

static size_t sched_bytes(int K) { return (size_t)(K - 1) * (K / 2) * 2; }

template <int JR>
static void set_smem_attrs(size_t mx64, size_t mxmixed) {
  cudaFuncSetAttribute(k_jacobi_f64<JR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx64);
  cudaFuncSetAttribute(k_jacobi_mixed<JR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mxmixed);
}

bool jacobi_attrs();
int init_jacobi_attributes() { return jacobi_attrs() ? 0 : 1; }

bool jacobi_attrs() {
  // once per process (contexts may be created from several threads)
  static std::once_flag once;
  static int state = 0;  // 1 ok, 2 failed
  std::call_once(once, [] {
    const size_t mx64 =
        (size_t)(JMAXK * JMAXK + 2 * JMAXK) * sizeof(double) + JMAXK * sizeof(int) + sched_bytes(JMAXK);
    const size_t mxm = (size_t)(2 * JMAXK * JMAXK + JMAXK) * sizeof(float) + (size_t)JMAXK * sizeof(int) +
                       sched_bytes(JMAXK);
    set_smem_attrs<3>(mx64, mxm);
    set_smem_attrs<6>(mx64, mxm);
    set_smem_attrs<9>(mx64, mxm);
    set_smem_attrs<12>(mx64, mxm);
    set_smem_attrs<16>(mx64, mxm);
    state = cudaGetLastError() == cudaSuccess ? 1 : 2;
  });
  return state == 1;
}

// CTAs of the cluster that runs the float64 projected SVD (1 where a cluster launch is not possible).
static constexpr int kJacobiCluster = 8;

template <int JR>
static int jacobi_f64_cluster_size(size_t smem_max) {
  static std::once_flag once;
  static int size = 1;
  std::call_once(once, [smem_max] {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kJacobiCluster);
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = smem_max;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kJacobiCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_jacobi_f64<JR>, &cfg) == cudaSuccess && nclusters > 0)
      size = kJacobiCluster;
    (void)cudaGetLastError();
  });
  return size;
}

template <int JR>
static int jacobi_f64_launch(const double* T, int ldT, int K, const double* S, int b, int nv, double* theta,
                             double* Xl, double* Wr, double* res, double tol, int max_sweeps, unsigned int* err,
                             unsigned long long* counters, size_t smem, int thr, cudaStream_t st, int cluster) {
  const size_t mx64 = (size_t)(JMAXK * JMAXK + 2 * JMAXK) * sizeof(double) + JMAXK * sizeof(int) + sched_bytes(JMAXK);
  const int nct = cluster == 1 ? 1 : jacobi_f64_cluster_size<JR>(mx64);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nct);
  cfg.blockDim = dim3(thr);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nct;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = nct > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_jacobi_f64<JR>, T, ldT, K, S, b, nv, theta, Xl, Wr, res, tol, max_sweeps, err,
                            counters) == cudaSuccess
             ? 1
             : 0;
}

int launch_small_svd(const double* T, int ldT, int K, const double* S, int b, int nv, double* theta, double* Xl,
                     double* Wr, double* res, double tol, int max_sweeps, unsigned int* err,
                     unsigned long long* counters, cudaStream_t st, int cluster) {
  if (!jacobi_attrs() || K > JMAXK) return 0;  // no launch; the caller's checks report the failure
  const size_t smem = (size_t)(K * K + 2 * K) * sizeof(double) + (size_t)K * sizeof(int) + sched_bytes(K);
  const int thr = jacobi_threads(K);
  const int rpl = (K + JL - 1) / JL;
#define SVT_JF64(JRV) \
  jacobi_f64_launch<JRV>(T, ldT, K, S, b, nv, theta, Xl, Wr, res, tol, max_sweeps, err, counters, smem, thr, st, \
                         cluster)
  if (rpl <= 3) return SVT_JF64(3);
  if (rpl <= 6) return SVT_JF64(6);
  if (rpl <= 9) return SVT_JF64(9);
  if (rpl <= 12) return SVT_JF64(12);
  return SVT_JF64(16);
#undef SVT_JF64
}

int launch_small_svd_mixed(const double* T, int ldT, int K, const double* S, int b, double* theta, double* Xl,
                           double* Wr, double* res, int nvec, float* wsrc, double tol, int max_sweeps,
                           unsigned int* err, unsigned long long* counters, cudaStream_t st) {
  if (nvec > K) nvec = K;
  if (!jacobi_attrs() || K > JMAXK) return 0;  // no launch; the caller's checks report the failure
  const size_t smem = (size_t)(2 * K * K + K) * sizeof(float) + (size_t)K * sizeof(int) + sched_bytes(K);
  const int thr = jacobi_threads(K);
  const int rpl = (K + JL - 1) / JL;
  const float ft = (float)tol;
  const int tr = kJacobiOnRows;
  if (rpl <= 3)
    k_jacobi_mixed<3><<<1, thr, smem, st>>>(T, ldT, K, theta, Xl, Wr, res, nvec, wsrc, ft, max_sweeps, err, counters,
                                            tr);
  else if (rpl <= 6)
    k_jacobi_mixed<6><<<1, thr, smem, st>>>(T, ldT, K, theta, Xl, Wr, res, nvec, wsrc, ft, max_sweeps, err, counters,
                                            tr);
  else if (rpl <= 9)
    k_jacobi_mixed<9><<<1, thr, smem, st>>>(T, ldT, K, theta, Xl, Wr, res, nvec, wsrc, ft, max_sweeps, err, counters,
                                            tr);
  else if (rpl <= 12)
    k_jacobi_mixed<12><<<1, thr, smem, st>>>(T, ldT, K, theta, Xl, Wr, res, nvec, wsrc, ft, max_sweeps, err,
                                             counters, tr);
  else
    k_jacobi_mixed<16><<<1, thr, smem, st>>>(T, ldT, K, theta, Xl, Wr, res, nvec, wsrc, ft, max_sweeps, err,
                                             counters, tr);
  k_ritz_refine<<<nvec, 128, 0, st>>>(T, ldT, K, S, b, wsrc, theta, Xl, Wr, res);
  return 2;
}

}  // namespace svt
