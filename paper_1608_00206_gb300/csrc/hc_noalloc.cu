// hc_convolve_noalloc: the plain forward convolution for callers that must
// not allocate device memory at the call site -- code running while another
// framework owns the device's memory pool, latency-critical loops that cannot
// afford the device-wide synchronisation cudaMalloc and cudaFree imply, or
// plugin hosts that forbid allocation once set up.  Instead of a caller-sized
// workspace, it uses one fixed array in the library's own device memory.
#include <cuda.h>

#include <mutex>

#include "hc_common.cuh"
#include "hc_forward.cuh"

namespace {

// The scratch: a file-scope device array.  This translation unit is its own
// device-code module, which CUDA loads onto a GPU lazily, the first time a
// context on that GPU needs it -- here, at the first hc_convolve_noalloc on
// that device, whose cudaGetSymbolAddress loads the module and with it
// allocates the array.  The GPU then holds the array until the process exits
// (or the context is destroyed).
constexpr size_t kScratchBytes = HC_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device addresses of the array, one per CUDA context that has used it.  A
// context is keyed by its driver-assigned id, which is never reused within a
// process: after a device reset the new primary context gets a new id and a
// fresh look-up, so a stale address from the destroyed context is never
// handed to a kernel.
struct Entry {
  unsigned long long ctx_id;
  void* ptr;
};
constexpr int kEntries = 64;
std::mutex g_mu;
Entry g_cache[kEntries];
int g_n = 0;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_resolved = false;

// The two driver entry points, found through the runtime (the library does
// not link the driver library itself).  Called with g_mu held.
void resolve_driver_entry_points() {
  if (g_resolved) return;
  g_resolved = true;
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
          cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_current = (CtxGetCurrentFn)f;
  f = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
          cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_id = (CtxGetIdFn)f;
  cudaGetLastError();
}

// Id of the calling thread's current context; false when there is none yet
// (no runtime call has made one current on this thread) or the driver does
// not offer the query.
bool current_ctx_id(unsigned long long* id) {
  if (!g_ctx_current || !g_ctx_id) return false;
  CUcontext c = nullptr;
  if (g_ctx_current(&c) != CUDA_SUCCESS || c == nullptr) return false;
  return g_ctx_id(c, id) == CUDA_SUCCESS;
}

// Device address of the array in the current context.  In host code the
// array's name is only a host-side stand-in, so its address is looked up
// with cudaGetSymbolAddress -- once per context, with that context's device
// current -- and remembered.
hc_status scratch_for_current_context(void** out) {
  std::lock_guard<std::mutex> g(g_mu);
  resolve_driver_entry_points();
  unsigned long long id = 0;
  bool have_id = current_ctx_id(&id);
  if (have_id) {
    for (int i = 0; i < g_n; ++i)
      if (g_cache[i].ctx_id == id) {
        *out = g_cache[i].ptr;
        return HC_OK;
      }
  }
  // Set-up: loads this module onto the device (allocating the array) the
  // first time the context needs it, and makes the primary context current.
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return hc::record_cuda_error(e);
  if (!p) return HC_ERR_CUDA;
  if (!have_id) have_id = current_ctx_id(&id);
  if (have_id) {
    if (g_n < kEntries) {
      g_cache[g_n++] = Entry{id, p};
    } else {  // many contexts over the process's life: forget the oldest
      for (int i = 1; i < kEntries; ++i) g_cache[i - 1] = g_cache[i];
      g_cache[kEntries - 1] = Entry{id, p};
    }
  }
  *out = p;
  return HC_OK;
}

}  // namespace

extern "C" hc_status hc_convolve_noalloc(const void* x, const void* y, void* z, int D,
                                         hc_dtype dtype, hc_stream_t stream) {
  if (D < 0 || D > HC_MAX_D) return HC_ERR_ARG;
  if (hc::elem_size(dtype) == 0) return HC_ERR_DTYPE;
  // The built-in chunked schedule, whatever default is installed, so that the
  // size limit stays the documented one.  Problems whose workspace does not
  // fit the fixed array are refused before any CUDA call.
  const hc_schedule builtin = {HC_SCHED_CHUNKED, 0, 0, 0, 0};
  if (hc_workspace_size_schedule(D, dtype, &builtin) > kScratchBytes) return HC_ERR_WORKSPACE;
  void* scratch = nullptr;
  const hc_status s = scratch_for_current_context(&scratch);
  if (s != HC_OK) return s;
  // Same validation and kernels as hc_convolve, with the array as workspace.
  // The schedule clears the counters it needs at zero itself (a memset on the
  // stream); everything else left by the previous call is overwritten.
  return hc::convolve_checked(x, y, z, D, dtype, scratch, kScratchBytes, (cudaStream_t)stream,
                              &builtin);
}
