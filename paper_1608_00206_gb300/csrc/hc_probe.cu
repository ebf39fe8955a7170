// hc_probe_alu_rate: a measurement aid for the roofline of the ALU-bound
// float64 path (GB300's FP64 rate is a small fraction of its float32 rate,
// so the float64 kernels are bound by arithmetic, not by HBM).  It times a
// kernel of independent dependency chains of the dtype's round-to-nearest
// add and multiply, the operations the recurrence uses, and reports their
// rate.  The paper has no counterpart.
#include "hc_common.cuh"

namespace hc {

constexpr int kProbeChains = 8;     // independent chains per thread
constexpr int kProbeIters = 4096;   // loop trips; each does 2 operations per chain
constexpr int kProbeThreads = 256;

template <class T>
__device__ __forceinline__ T probe_add(T a, T b);
template <>
__device__ __forceinline__ double probe_add(double a, double b) { return __dadd_rn(a, b); }
template <>
__device__ __forceinline__ float probe_add(float a, float b) { return __fadd_rn(a, b); }
template <class T>
__device__ __forceinline__ T probe_mul(T a, T b);
template <>
__device__ __forceinline__ double probe_mul(double a, double b) { return __dmul_rn(a, b); }
template <>
__device__ __forceinline__ float probe_mul(float a, float b) { return __fmul_rn(a, b); }

// Each chain alternates an addition and a multiplication by values close to
// 0 and 1 (the chains stay finite); the sum of the chains is written so that
// nothing is optimised away.
template <class T>
__global__ void __launch_bounds__(kProbeThreads) alu_probe_kernel(T* out, T inc, T scale) {
  T v[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) v[c] = (T)(threadIdx.x + c);
#pragma unroll 1
  for (int i = 0; i < kProbeIters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) v[c] = probe_mul(probe_add(v[c], inc), scale);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s = probe_add(s, v[c]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
static hc_status probe(double* ops_per_s, cudaStream_t st) {
  const int blocks = device_caps().sms * 8;
  T* out = nullptr;
  // The probe's own scratch: one value per thread, allocated and freed here
  // (a measurement call, not part of any convolution).
  cudaError_t e = cudaMalloc(&out, sizeof(T) * (size_t)blocks * kProbeThreads);
  if (e != cudaSuccess) return record_cuda_error(e);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = -1.0f;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {  // the first run is a warm-up
    cudaEventRecord(e0, st);
    alu_probe_kernel<T><<<blocks, kProbeThreads, 0, st>>>(out, (T)1e-7, (T)0.9999999);
    e = cudaGetLastError();
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && (best < 0.0f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return record_cuda_error(e);
  const double ops = 2.0 * kProbeChains * kProbeIters * (double)blocks * kProbeThreads;
  *ops_per_s = best > 0.0f ? ops / (best * 1e-3) : 0.0;
  return HC_OK;
}

}  // namespace hc

extern "C" hc_status hc_probe_alu_rate(hc_dtype dtype, double* ops_per_s, hc_stream_t stream) {
  if (!ops_per_s) return HC_ERR_ARG;
  if (dtype == HC_FP64) return hc::probe<double>(ops_per_s, (cudaStream_t)stream);
  if (dtype == HC_FP32) return hc::probe<float>(ops_per_s, (cudaStream_t)stream);
  return HC_ERR_DTYPE;
}
