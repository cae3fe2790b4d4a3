// svt_sddmm_update_noalloc: the fused X-on-Omega + dual step + residual kernel for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is already handed out to its
// own pool (a deep-learning framework's caching allocator, an inference server with a fixed
// memory budget), or a real-time loop in which the implicit device synchronisation of cudaMalloc
// and cudaFree would stall other work.  This entry point needs no allocation: the caller passes
// every input and output, and the only scratch (one partial sum per CTA and the final sum) lives
// in a file-scope __device__ array that every GPU loading this library holds until process exit.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/svt.h"
#include "common.cuh"
#include "internal.h"

static constexpr int kScratchDoubles = 4096;   // 32 KB per device
static constexpr int kRowsPerBlock = 64;       // rows reduced by one CTA (8 warps x 8 rows)
static constexpr int64_t kMaxRows = (int64_t)(kScratchDoubles - 1) * kRowsPerBlock;  // 262080
static constexpr int kMaxDevices = 64;

// Partial sums (entries 0 .. blocks-1) and the total (last entry).  Shared by every call on a
// device: calls whose work overlaps on the GPU race on it.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

namespace {

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};   // id of the context the address belongs to
thread_local std::string g_noalloc_error;

// Driver entry points reached through the runtime (the library does not link libcuda): the id of
// the current context tells a cached address from one that died with its context (cudaDeviceReset
// destroys the primary context and the module with it; the next context loads it anew).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    (void)cudaGetLastError();
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

svt_status noalloc_fail(svt_status s, const char* msg, cudaError_t e = cudaSuccess) {
  char buf[384];
  if (e != cudaSuccess) snprintf(buf, sizeof buf, "svt_sddmm_update_noalloc: %s (%s)", msg, cudaGetErrorString(e));
  else snprintf(buf, sizeof buf, "svt_sddmm_update_noalloc: %s", msg);
  g_noalloc_error = buf;
  return s;
}

// Device address of the scratch array on the current device.  In host code the array's name is a
// host-side stand-in, not a device address, so it is looked up once per device with that device
// current, and again when the device's current context is no longer the one the address was
// taken in (after cudaDeviceReset).
svt_status scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(SVT_ERR_CUDA, "cudaGetDevice failed", e);
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(SVT_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return noalloc_fail(SVT_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed", e);
    g_scratch_addr[dev] = static_cast<double*>(p);
    // the lookup made the device's primary context current if no context was
    g_scratch_ctx[dev] = current_context_id();
  }
  *out = g_scratch_addr[dev];
  return SVT_OK;
}

}  // namespace

extern "C" const char* svt_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

extern "C" svt_status svt_sddmm_update_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr,
                                               const int32_t* col_idx, const double* M, const double* Ut,
                                               const double* V, int r, double delta, const double* y_in,
                                               double* y_out, double* res2, void* stream) {
  if (m < 1 || n < 1 || nnz < 0 || n >= (1LL << 31) || nnz >= (1LL << 31))
    return noalloc_fail(SVT_ERR_ARG, "need m, n >= 1, 0 <= nnz < 2^31");
  if (m > kMaxRows) {
    char msg[160];
    snprintf(msg, sizeof msg, "m = %lld rows exceeds the %lld rows its static scratch can reduce", (long long)m,
             (long long)kMaxRows);
    return noalloc_fail(SVT_ERR_ARG, msg);
  }
  if (r < 0 || r > 64) return noalloc_fail(SVT_ERR_ARG, "need 0 <= r <= 64");
  if (!row_ptr || !res2 || (nnz > 0 && (!col_idx || !M || !y_in || !y_out)) || (r > 0 && (!Ut || !V)))
    return noalloc_fail(SVT_ERR_ARG, "NULL pointer argument");
  if (nnz > 0 && (const void*)y_in == (const void*)y_out)
    return noalloc_fail(SVT_ERR_ARG, "y_in and y_out must be different buffers");
  double* scratch = nullptr;
  svt_status s = scratch_address(&scratch);
  if (s != SVT_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = (int)((m + kRowsPerBlock - 1) / kRowsPerBlock);
  // every partial slot 0 .. blocks-1 and the total are written by this call before they are read,
  // so the contents left by an earlier call need no clearing
  svt::launch_sddmm_update_grid(row_ptr, col_idx, M, y_in, y_out, Ut, V, r, (int)m, delta, blocks, scratch,
                                scratch + (kScratchDoubles - 1), st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(SVT_ERR_CUDA, "kernel launch failed", e);
  e = cudaMemcpyAsync(res2, scratch + (kScratchDoubles - 1), sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return noalloc_fail(SVT_ERR_CUDA, "device work failed", e);
  if (!std::isfinite(*res2)) return noalloc_fail(SVT_ERR_NUMERIC, "NaN or Inf in the residual");
  return SVT_OK;
}
