// Kernels and launch helpers shared by the forward, backward and batched
// translation units.
#pragma once

#include "hc_common.cuh"
#include "hc_profile.cuh"

namespace hc {

// ---------------------------------------------------------------------------
// K1: evaluate K axes of a [hi][2^K][lo] array into [hi][3^K][lo], for x and
// y at once (blockIdx.y selects the operand).  One thread per (h, l) column;
// consecutive threads take consecutive l, so every load and store of a warp
// is one contiguous segment.
template <class M, int K>
__global__ void __launch_bounds__(256) eval_pass_kernel(const typename M::In* __restrict__ sx,
                                                        const typename M::In* __restrict__ sy,
                                                        typename M::In* __restrict__ dx,
                                                        typename M::In* __restrict__ dy,
                                                        long long hi, long long lo) {
  typedef typename M::In T;
  const T* src = blockIdx.y ? sy : sx;
  T* dst = blockIdx.y ? dy : dx;
  const long long cols = hi * lo;
#pragma unroll 1
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < cols;
       c += (long long)gridDim.x * blockDim.x) {
    const long long h = c / lo, l = c - h * lo;
    T v[p3(K)];
    const T* s = src + (h * p2(K)) * lo + l;
#pragma unroll
    for (int b = 0; b < p2(K); ++b) v[b] = s[b * lo];
    eval_pencil<M, K>(v);
    T* d = dst + (h * p3(K)) * lo + l;
#pragma unroll
    for (int j = 0; j < p3(K); ++j) d[j * lo] = v[j];
  }
}

template <class K>
inline cudaError_t prep_kernel(K kernel, size_t smem) {
  // Raise the dynamic shared-memory limit once per kernel instantiation.
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

template <class K>
inline int grid_for(K kernel, int threads, size_t smem, long long work_items) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  long long g = (long long)device_caps().sms * per_sm;
  if (work_items < g) g = work_items;
  return (int)(g < 1 ? 1 : g);
}

template <class M, int K>
inline cudaError_t launch_eval_k(const typename M::In* sx, const typename M::In* sy,
                                 typename M::In* dx, typename M::In* dy, long long hi, long long lo,
                                 cudaStream_t st) {
  ProfileScope prof(st, "eval_pass");
  auto k = eval_pass_kernel<M, K>;
  const long long cols = hi * lo;
  long long blocks = (cols + 255) / 256;
  const long long cap = (long long)device_caps().sms * 8;
  if (blocks > cap) blocks = cap;
  k<<<dim3((unsigned)blocks, 2), 256, 0, st>>>(sx, sy, dx, dy, hi, lo);
  return cudaGetLastError();
}

template <class M>
inline cudaError_t launch_eval(int K, const typename M::In* sx, const typename M::In* sy,
                               typename M::In* dx, typename M::In* dy, long long hi, long long lo,
                               cudaStream_t st) {
  switch (K) {
    case 1: return launch_eval_k<M, 1>(sx, sy, dx, dy, hi, lo, st);
    case 2: return launch_eval_k<M, 2>(sx, sy, dx, dy, hi, lo, st);
    case 3: return launch_eval_k<M, 3>(sx, sy, dx, dy, hi, lo, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hc
