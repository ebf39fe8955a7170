// hc_convolve_noalloc: the plain forward convolution for callers that must
// not allocate device memory at the call site -- code running while another
// framework owns the device's memory pool, latency-critical loops that cannot
// afford the device-wide synchronisation cudaMalloc and cudaFree imply, or
// plugin hosts that forbid allocation once set up.  Instead of a caller-sized
// workspace, it uses one fixed array in the library's own device memory.
#include <mutex>

#include "hc_common.cuh"
#include "hc_forward.cuh"

namespace {

// The scratch: allocated when the library's device code is loaded onto a GPU
// and held by that GPU until the process exits.
constexpr size_t kScratchBytes = HC_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[64] = {nullptr};

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and remembered.
hc_status scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hc::record_cuda_error(e);
  if (dev < 0 || dev >= 64) return HC_ERR_ARG;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return hc::record_cuda_error(e);
    if (!p) return HC_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return HC_OK;
}

}  // namespace

extern "C" hc_status hc_convolve_noalloc(const void* x, const void* y, void* z, int D,
                                         hc_dtype dtype, hc_stream_t stream) {
  if (D < 0 || D > HC_MAX_D) return HC_ERR_ARG;
  if (hc::elem_size(dtype) == 0) return HC_ERR_DTYPE;
  // The built-in chunked schedule, whatever default is installed, so that the
  // size limit stays the documented one.  Problems whose workspace does not
  // fit the fixed array are refused.
  const hc_schedule builtin = {HC_SCHED_CHUNKED, 0, 0, 0};
  if (hc_workspace_size_schedule(D, dtype, &builtin) > kScratchBytes) return HC_ERR_WORKSPACE;
  void* scratch = nullptr;
  const hc_status s = scratch_for_current_device(&scratch);
  if (s != HC_OK) return s;
  // Same validation and kernels as hc_convolve, with the array as workspace.
  // The schedule clears the counters it needs at zero itself (a memset on the
  // stream); everything else left by the previous call is overwritten.
  return hc::convolve_checked(x, y, z, D, dtype, scratch, kScratchBytes, (cudaStream_t)stream,
                              &builtin);
}
