// Storage and sampling of the fixed sampled set Omega (Sec. 2.2: Y^k vanishes off Omega for all
// k, so the iterate is stored only on Omega; Sec. 5.2.1: Omega uniform among subsets of size m).
//
// Storage build: counting sort by the major index (atomic histogram, exclusive scan, atomic
// scatter), then every segment is sorted by the minor index with a bitonic network in shared
// memory.  Because a valid Omega has no repeated pair, the sorted result is unique, so the
// order of the atomic scatter does not show in the output: the build is deterministic.
//
// Sampler: random keys.  key(id) = output number id + 1 of SplitMix64 started at `seed`; Omega is
// the m ids with the smallest (key, id).  A threshold filter keeps ~m(1+O(1/sqrt m)) candidates,
// an MSB-first radix select over the 128-bit (key, id) finds the m-th smallest pair, and an
// ordered compaction over all ids writes the selected ids in increasing order.
#include "common.cuh"
#include "internal.h"

namespace svt {

// ------------------------------------------------------------------------------------------------
// Exclusive scan (int32), three phases: block sums, scan of block sums, block scan + offset.
// ------------------------------------------------------------------------------------------------
static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_ITEMS = 8;
static constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int block_exclusive_scan_int(int v, int* total) {
  __shared__ int warp_tot[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  int nw = blockDim.x >> 5;
  if (wid == 0) {
    int t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_tot[lane] = t;  // inclusive
  }
  __syncthreads();
  int before = (wid > 0 ? warp_tot[wid - 1] : 0) + x - v;
  if (total) *total = warp_tot[nw - 1];
  __syncthreads();
  return before;
}

__global__ void k_scan_block_sums(const int32_t* __restrict__ in, long long n, int32_t* __restrict__ sums) {
  long long base = (long long)blockIdx.x * SCAN_TILE;
  int acc = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    long long i = base + (long long)k * SCAN_THREADS + threadIdx.x;
    if (i < n) acc += in[i];
  }
  int tot;
  block_exclusive_scan_int(acc, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of `sums` (n entries) in place, grand total to sums[n].
__global__ void k_scan_sums(int32_t* sums, long long n) {
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long long base = 0; base < n; base += blockDim.x) {
    long long i = base + threadIdx.x;
    int v = i < n ? sums[i] : 0;
    int tot;
    int ex = block_exclusive_scan_int(v, &tot);
    if (i < n) sums[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[n] = carry;
}

__global__ void k_scan_apply(const int32_t* __restrict__ in, long long n, const int32_t* __restrict__ sums,
                             int32_t* __restrict__ out) {
  long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS];
  int acc = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    long long i = base + k;
    v[k] = i < n ? in[i] : 0;
    acc += v[k];
  }
  int ex = block_exclusive_scan_int(acc, nullptr) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    long long i = base + k;
    if (i < n) out[i] = ex;
    ex += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

long long scan_scratch_ints(long long n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

int launch_exclusive_scan(const int32_t* in, int32_t* out, long long n, int32_t* scratch, cudaStream_t st) {
  if (n <= 0) {
    cudaMemsetAsync(out, 0, sizeof(int32_t), st);
    return 0;
  }
  int nb = svt_ceil_div(n, SCAN_TILE);
  k_scan_block_sums<<<nb, SCAN_THREADS, 0, st>>>(in, n, scratch);
  k_scan_sums<<<1, 1024, 0, st>>>(scratch, nb);
  k_scan_apply<<<nb, SCAN_THREADS, 0, st>>>(in, n, scratch, out);
  return 3;
}

// ------------------------------------------------------------------------------------------------
// Segment build
// ------------------------------------------------------------------------------------------------
__global__ void k_count_major(const int32_t* __restrict__ major, const int32_t* __restrict__ minor, long long nnz,
                              int n_major, int n_minor, int32_t* __restrict__ counts, unsigned int* err) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x) {
    int a = major[p], b = minor[p];
    if (a < 0 || a >= n_major || b < 0 || b >= n_minor) {
      svt_set_error(err, SVT_DEVERR_INDEX_RANGE);
      continue;
    }
    atomicAdd(&counts[a], 1);
  }
}

int launch_count_major(const int32_t* major, const int32_t* minor, long long nnz, int n_major, int n_minor,
                       int32_t* counts, unsigned int* err, cudaStream_t st) {
  int blocks = (int)svt_min_ll(svt_ceil_div(nnz, 256), 152LL * 16);
  if (blocks < 1) blocks = 1;
  k_count_major<<<blocks, 256, 0, st>>>(major, minor, nnz, n_major, n_minor, counts, err);
  return 1;
}

__global__ void k_scatter_segments(const int32_t* __restrict__ major, const int32_t* __restrict__ minor,
                                   const int32_t* __restrict__ payload, long long nnz, int n_major, int n_minor,
                                   const int32_t* __restrict__ ptr, int32_t* __restrict__ cursor,
                                   int32_t* __restrict__ out_minor, int32_t* __restrict__ out_payload) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x) {
    int a = major[p], b = minor[p];
    if (a < 0 || a >= n_major || b < 0 || b >= n_minor) continue;
    int pos = ptr[a] + atomicAdd(&cursor[a], 1);
    if (pos < ptr[a + 1]) {
      out_minor[pos] = b;
      out_payload[pos] = payload ? payload[p] : (int32_t)p;
    }
  }
}

int launch_scatter_segments(const int32_t* major, const int32_t* minor, const int32_t* payload, long long nnz,
                            int n_major, int n_minor, const int32_t* ptr, int32_t* cursor, int32_t* out_minor,
                            int32_t* out_payload, cudaStream_t st) {
  int blocks = (int)svt_min_ll(svt_ceil_div(nnz, 256), 152LL * 16);
  if (blocks < 1) blocks = 1;
  k_scatter_segments<<<blocks, 256, 0, st>>>(major, minor, payload, nnz, n_major, n_minor, ptr, cursor, out_minor,
                                             out_payload);
  return 1;
}

static constexpr int SEG_CAP = 4096;  // segment length sorted in shared memory (2 x 16 KB)
static constexpr int SEG_THREADS = 256;

int segment_smem_capacity() { return SEG_CAP; }

// Bitonic sort of (key, val) pairs, length L = power of two, ascending by key.  `key`/`val` may be
// shared or global memory of this block; the caller synchronises before and after.
__device__ void bitonic_sort_pairs(int32_t* key, int32_t* val, int L) {
  for (int size = 2; size <= L; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < (L >> 1); t += blockDim.x) {
        int lo = 2 * t - (t & (stride - 1));
        int hi = lo + stride;
        bool up = (lo & size) == 0;
        int ka = key[lo], kb = key[hi];
        if ((ka > kb) == up) {
          key[lo] = kb; key[hi] = ka;
          int va = val[lo]; val[lo] = val[hi]; val[hi] = va;
        }
      }
      __syncthreads();
    }
  }
}

__global__ void k_sort_segments(const int32_t* __restrict__ ptr, int n_seg, int32_t* __restrict__ minor,
                                int32_t* __restrict__ payload) {
  __shared__ int32_t skey[SEG_CAP];
  __shared__ int32_t sval[SEG_CAP];
  for (int s = blockIdx.x; s < n_seg; s += gridDim.x) {
    int a = ptr[s], len = ptr[s + 1] - a;
    if (len <= 1 || len > SEG_CAP) continue;
    int L = 1;
    while (L < len) L <<= 1;
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
      skey[t] = t < len ? minor[a + t] : 0x7fffffff;
      sval[t] = t < len ? payload[a + t] : 0;
    }
    __syncthreads();
    bitonic_sort_pairs(skey, sval, L);
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
      minor[a + t] = skey[t];
      payload[a + t] = sval[t];
    }
    __syncthreads();
  }
}

int launch_sort_segments(const int32_t* ptr, int n_seg, int32_t* minor, int32_t* payload, cudaStream_t st) {
  if (n_seg <= 0) return 0;
  int blocks = min(n_seg, 152 * 8);
  k_sort_segments<<<blocks, SEG_THREADS, 0, st>>>(ptr, n_seg, minor, payload);
  return 1;
}

__global__ void k_sort_long_segment(int32_t* minor, int32_t* payload, int len, int L, int32_t* skey, int32_t* sval) {
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    skey[t] = t < len ? minor[t] : 0x7fffffff;
    sval[t] = t < len ? payload[t] : 0;
  }
  __syncthreads();
  bitonic_sort_pairs(skey, sval, L);
  for (int t = threadIdx.x; t < len; t += blockDim.x) {
    minor[t] = skey[t];
    payload[t] = sval[t];
  }
}

int launch_sort_long_segment(int32_t* minor, int32_t* payload, int len, int32_t* scratch, cudaStream_t st) {
  int L = 1;
  while (L < len) L <<= 1;
  k_sort_long_segment<<<1, 1024, 0, st>>>(minor, payload, len, L, scratch, scratch + L);
  return 1;
}

__global__ void k_max_segment(const int32_t* __restrict__ ptr, int n_seg, int32_t* out) {
  int best = 0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_seg; s += gridDim.x * blockDim.x)
    best = max(best, ptr[s + 1] - ptr[s]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

int launch_max_segment(const int32_t* ptr, int n_seg, int32_t* out, cudaStream_t st) {
  cudaMemsetAsync(out, 0, sizeof(int32_t), st);
  if (n_seg <= 0) return 0;
  int blocks = min(svt_ceil_div(n_seg, 256), 152 * 4);
  k_max_segment<<<blocks, 256, 0, st>>>(ptr, n_seg, out);
  return 1;
}

__global__ void k_check_duplicates(const int32_t* __restrict__ ptr, int n_seg, const int32_t* __restrict__ minor,
                                   unsigned int* err) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_seg; s += gridDim.x * blockDim.x) {
    int a = ptr[s], b = ptr[s + 1];
    for (int p = a + 1; p < b; ++p)
      if (minor[p] == minor[p - 1]) {
        svt_set_error(err, SVT_DEVERR_DUPLICATE);
        break;
      }
  }
}

int launch_check_duplicates(const int32_t* ptr, int n_seg, const int32_t* minor, unsigned int* err, cudaStream_t st) {
  if (n_seg <= 0) return 0;
  int blocks = min(svt_ceil_div(n_seg, 256), 152 * 4);
  k_check_duplicates<<<blocks, 256, 0, st>>>(ptr, n_seg, minor, err);
  return 1;
}

__global__ void k_expand_ptr(const int32_t* __restrict__ ptr, int n_seg, int32_t* __restrict__ out) {
  for (int s = blockIdx.x; s < n_seg; s += gridDim.x) {
    int a = ptr[s], b = ptr[s + 1];
    for (int p = a + threadIdx.x; p < b; p += blockDim.x) out[p] = s;
  }
}

int launch_expand_ptr(const int32_t* ptr, int n_seg, int32_t* out, cudaStream_t st) {
  if (n_seg <= 0) return 0;
  k_expand_ptr<<<min(n_seg, 152 * 16), 128, 0, st>>>(ptr, n_seg, out);
  return 1;
}

__global__ void k_gather_f64(const double* __restrict__ in, const int32_t* __restrict__ perm, long long n,
                             double* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = in[perm[i]];
}
__global__ void k_gather_f64_to_f32(const double* __restrict__ in, const int32_t* __restrict__ perm, long long n,
                                    float* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[perm[i]];
}
int launch_gather_f64(const double* in, const int32_t* perm, long long n, double* out, cudaStream_t st) {
  if (n <= 0) return 0;
  k_gather_f64<<<(int)svt_min_ll(svt_ceil_div(n, 256), 152LL * 16), 256, 0, st>>>(in, perm, n, out);
  return 1;
}
int launch_gather_f64_to_f32(const double* in, const int32_t* perm, long long n, float* out, cudaStream_t st) {
  if (n <= 0) return 0;
  k_gather_f64_to_f32<<<(int)svt_min_ll(svt_ceil_div(n, 256), 152LL * 16), 256, 0, st>>>(in, perm, n, out);
  return 1;
}

__global__ void k_invert_perm(const int32_t* __restrict__ perm, long long n, int32_t* __restrict__ inv) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    inv[perm[i]] = (int32_t)i;
}
int launch_invert_perm(const int32_t* perm, long long n, int32_t* inv, cudaStream_t st) {
  if (n <= 0) return 0;
  k_invert_perm<<<(int)svt_min_ll(svt_ceil_div(n, 256), 152LL * 16), 256, 0, st>>>(perm, n, inv);
  return 1;
}

// Deterministic sum of squares: fixed grid of 1024 partials, then one block sums them in order.
__global__ void k_sumsq_partial(const double* __restrict__ x, long long n, double* __restrict__ partial) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc += x[i] * x[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
}
__global__ void k_sum_partials(const double* __restrict__ partial, int np, double* out) {
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
int launch_sumsq_f64(const double* x, long long n, double* partial, double* out, cudaStream_t st) {
  k_sumsq_partial<<<1024, 256, 0, st>>>(x, n, partial);
  k_sum_partials<<<1, 1024, 0, st>>>(partial, 1024, out);
  return 2;
}

// ------------------------------------------------------------------------------------------------
// Omega sampler
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long index) {
  unsigned long long z = seed + index * 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

__global__ void k_omega_filter(unsigned long long seed, long long N, unsigned long long thresh,
                               unsigned long long* __restrict__ cand_key, unsigned long long* __restrict__ cand_id,
                               long long cap, unsigned long long* count) {
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < N; id += (long long)gridDim.x * blockDim.x) {
    unsigned long long key = splitmix64_at(seed, (unsigned long long)id + 1ULL);
    if (key <= thresh) {
      unsigned long long slot = atomicAdd(count, 1ULL);
      if ((long long)slot < cap) {
        cand_key[slot] = key;
        cand_id[slot] = (unsigned long long)id;
      }
    }
  }
}

int launch_omega_filter(uint64_t seed, long long N, uint64_t thresh, unsigned long long* cand_key,
                        unsigned long long* cand_id, long long cap, unsigned long long* count, cudaStream_t st) {
  cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  int blocks = (int)svt_min_ll(svt_ceil_div(N, 256), 152LL * 32);
  k_omega_filter<<<blocks, 256, 0, st>>>(seed, N, thresh, cand_key, cand_id, cap, count);
  return 1;
}

struct SelectState {
  unsigned long long key_prefix;  // selected high digits of the key
  unsigned long long id_prefix;   // selected high digits of the id
  long long rank;                 // remaining 1-based rank inside the matching set
  unsigned int hist[256];
};

long long omega_select_state_bytes() { return (long long)sizeof(SelectState); }

// Digit d (0..15) of the 128-bit value (key, id), most significant first.
__device__ __forceinline__ unsigned int digit_of(unsigned long long key, unsigned long long id, int d) {
  return d < 8 ? (unsigned int)((key >> (56 - 8 * d)) & 0xff) : (unsigned int)((id >> (56 - 8 * (d - 8))) & 0xff);
}
__device__ __forceinline__ bool prefix_match(unsigned long long key, unsigned long long id, const SelectState* s, int d) {
  // digits 0..d-1 must match
  if (d <= 8) {
    if (d == 0) return true;
    unsigned long long mask = ~0ULL << (64 - 8 * d);
    return (key & mask) == (s->key_prefix & mask);
  }
  if (key != s->key_prefix) return false;
  int di = d - 8;
  if (di == 0) return true;
  unsigned long long mask = ~0ULL << (64 - 8 * di);
  return (id & mask) == (s->id_prefix & mask);
}

__global__ void k_select_hist(const unsigned long long* __restrict__ cand_key, const unsigned long long* __restrict__ cand_id,
                              const unsigned long long* count, long long cap, SelectState* s, int d) {
  __shared__ unsigned int h[256];
  for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
  __syncthreads();
  long long c = (long long)(*count < (unsigned long long)cap ? *count : (unsigned long long)cap);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < c; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long k = cand_key[i], id = cand_id[i];
    if (prefix_match(k, id, s, d)) atomicAdd(&h[digit_of(k, id, d)], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 256; t += blockDim.x)
    if (h[t]) atomicAdd(&s->hist[t], h[t]);
}

__global__ void k_select_pick(SelectState* s, int d) {
  // one warp: find the bin where the running count reaches s->rank
  if (threadIdx.x != 0) return;
  long long acc = 0;
  int bin = 255;
  for (int b = 0; b < 256; ++b) {
    long long c = s->hist[b];
    if (acc + c >= s->rank) { bin = b; break; }
    acc += c;
  }
  s->rank -= acc;
  if (d < 8) s->key_prefix |= (unsigned long long)bin << (56 - 8 * d);
  else s->id_prefix |= (unsigned long long)bin << (56 - 8 * (d - 8));
  for (int b = 0; b < 256; ++b) s->hist[b] = 0;
}

__global__ void k_select_init(SelectState* s, long long rank) {
  if (threadIdx.x == 0) {
    s->key_prefix = 0; s->id_prefix = 0; s->rank = rank;
  }
  for (int b = threadIdx.x; b < 256; b += blockDim.x) s->hist[b] = 0;
}

int launch_omega_select(const unsigned long long* cand_key, const unsigned long long* cand_id,
                        const unsigned long long* count, long long rank, void* state, cudaStream_t st) {
  SelectState* s = (SelectState*)state;
  k_select_init<<<1, 256, 0, st>>>(s, rank);
  int launches = 1;
  const long long cap = 1LL << 40;  // count is already clamped by the filter's capacity check on host
  for (int d = 0; d < 16; ++d) {
    k_select_hist<<<152 * 4, 256, 0, st>>>(cand_key, cand_id, count, cap, s, d);
    k_select_pick<<<1, 32, 0, st>>>(s, d);
    launches += 2;
  }
  return launches;
}

static constexpr int COMPACT_THREADS = 256;
static constexpr int COMPACT_ITEMS = 16;
static constexpr long long COMPACT_TILE = (long long)COMPACT_THREADS * COMPACT_ITEMS;

long long omega_compact_blocks(long long N) { return (N + COMPACT_TILE - 1) / COMPACT_TILE; }

__device__ __forceinline__ bool omega_selected(unsigned long long seed, unsigned long long id, const SelectState* s) {
  unsigned long long key = splitmix64_at(seed, id + 1ULL);
  return key < s->key_prefix || (key == s->key_prefix && id <= s->id_prefix);
}

__global__ void k_omega_count(unsigned long long seed, long long N, const SelectState* __restrict__ s,
                              int32_t* __restrict__ block_counts) {
  long long base = (long long)blockIdx.x * COMPACT_TILE + (long long)threadIdx.x * COMPACT_ITEMS;
  int c = 0;
  for (int k = 0; k < COMPACT_ITEMS; ++k) {
    long long id = base + k;
    if (id < N && omega_selected(seed, (unsigned long long)id, s)) ++c;
  }
  int tot;
  block_exclusive_scan_int(c, &tot);
  if (threadIdx.x == 0) block_counts[blockIdx.x] = tot;
}

__global__ void k_omega_write(unsigned long long seed, long long N, long long n_cols, const SelectState* __restrict__ s,
                              const int32_t* __restrict__ block_offsets, int32_t* __restrict__ rows,
                              int32_t* __restrict__ cols, long long m, unsigned int* err) {
  long long base = (long long)blockIdx.x * COMPACT_TILE + (long long)threadIdx.x * COMPACT_ITEMS;
  unsigned int flags = 0;
  int c = 0;
  for (int k = 0; k < COMPACT_ITEMS; ++k) {
    long long id = base + k;
    if (id < N && omega_selected(seed, (unsigned long long)id, s)) {
      flags |= 1u << k;
      ++c;
    }
  }
  long long pos = (long long)block_offsets[blockIdx.x] + block_exclusive_scan_int(c, nullptr);
  for (int k = 0; k < COMPACT_ITEMS; ++k) {
    if (flags & (1u << k)) {
      long long id = base + k;
      if (pos < m) {
        rows[pos] = (int32_t)(id / n_cols);
        cols[pos] = (int32_t)(id % n_cols);
      } else {
        svt_set_error(err, SVT_DEVERR_CAPACITY);
      }
      ++pos;
    }
  }
}

int launch_omega_compact(uint64_t seed, long long N, long long n_cols, const void* state, int32_t* block_counts,
                         int32_t* block_offsets, int32_t* scan_scratch, int32_t* rows, int32_t* cols, long long m,
                         unsigned int* err, cudaStream_t st) {
  const SelectState* s = (const SelectState*)state;
  long long nb = omega_compact_blocks(N);
  k_omega_count<<<(unsigned)nb, COMPACT_THREADS, 0, st>>>(seed, N, s, block_counts);
  int l = 1 + launch_exclusive_scan(block_counts, block_offsets, nb, scan_scratch, st);
  k_omega_write<<<(unsigned)nb, COMPACT_THREADS, 0, st>>>(seed, N, n_cols, s, block_offsets, rows, cols, m, err);
  return l + 1;
}

}  // namespace svt
