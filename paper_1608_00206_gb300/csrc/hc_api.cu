// libhc: status codes, argument helpers and the workspace status word.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "hc_common.cuh"

namespace hc {

static thread_local char g_cuda_msg[256] = "no CUDA error";

hc_status record_cuda_error(cudaError_t e) {
  if (e == cudaSuccess) return HC_OK;
  snprintf(g_cuda_msg, sizeof(g_cuda_msg), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return HC_ERR_CUDA;
}

LaunchCaps device_caps() {
  static std::mutex mu;
  static LaunchCaps caps[64];
  static bool have[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  std::lock_guard<std::mutex> g(mu);
  if (!have[dev]) {
    int sms = 0, smem = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    caps[dev].sms = sms > 0 ? sms : 1;
    caps[dev].smem_optin = (size_t)(smem > 0 ? smem : 48 * 1024);
    have[dev] = true;
  }
  return caps[dev];
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  if (!a || !b || na == 0 || nb == 0) return false;
  const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
  return a0 < b0 + nb && b0 < a0 + na;
}

size_t elem_size(hc_dtype dt) {
  switch (dt) {
    case HC_INT64:
    case HC_FP64: return 8;
    case HC_FP32:
    case HC_FP32_MIXED:
    case HC_FP32_FF: return 4;
  }
  return 0;
}

size_t in_size(hc_dtype dt) {
  switch (dt) {
    case HC_INT64:
    case HC_FP64:
    case HC_FP32_FF: return 8;
    case HC_FP32:
    case HC_FP32_MIXED: return 4;
  }
  return 0;
}

size_t w_size(hc_dtype dt) {
  switch (dt) {
    case HC_FP32: return 4;
    case HC_INT64:
    case HC_FP64:
    case HC_FP32_MIXED:
    case HC_FP32_FF: return 8;
  }
  return 0;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace hc

extern "C" int hc_version(void) { return (0 << 16) | (1 << 8) | 0; }

extern "C" const char* hc_status_string(hc_status s) {
  switch (s) {
    case HC_OK: return "HC_OK";
    case HC_ERR_ARG: return "HC_ERR_ARG: invalid argument (D, pointer or count)";
    case HC_ERR_DTYPE: return "HC_ERR_DTYPE: unsupported dtype";
    case HC_ERR_ALIGN: return "HC_ERR_ALIGN: pointer not 16-byte (workspace 256-byte) aligned";
    case HC_ERR_ALIAS: return "HC_ERR_ALIAS: output overlaps an input or the workspace";
    case HC_ERR_WORKSPACE: return "HC_ERR_WORKSPACE: workspace too small";
    case HC_ERR_CUDA: return "HC_ERR_CUDA: CUDA call failed";
    case HC_ERR_TIMEOUT: return "HC_ERR_TIMEOUT: a bounded device-side wait gave up";
  }
  return "unknown hc_status";
}

extern "C" const char* hc_last_cuda_error(void) { return hc::g_cuda_msg; }

extern "C" hc_status hc_device_status(const void* workspace, hc_stream_t stream) {
  if (!workspace) return HC_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return hc::record_cuda_error(e);
  unsigned int st = 0;
  e = cudaMemcpy(&st, workspace, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return hc::record_cuda_error(e);
  return (hc_status)st;
}
