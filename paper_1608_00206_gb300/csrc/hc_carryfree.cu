// Carry-free 1D convolution (Discussion of arXiv 1608.00206): for vectors x,
// y of length N, z[k] = sum of x[i] * y[j] over the pairs whose digit-wise
// sum of bits, with no carries, spells k in base 3.  With bit d of a 1D index
// read as axis d (most significant bit first) this is the hypercube
// convolution of the two vectors zero-padded to 2^D, D = ceil(log2 N): the
// padding adds only zero products.
#include "hc_common.cuh"
#include "hc_forward.cuh"
#include "hc_profile.cuh"

namespace hc {

// Copies x[0, n) and y[0, n) into the first n elements of px, py and zeroes
// [n, n2); blockIdx.y selects the operand.  Consecutive threads take
// consecutive elements (coalesced); a grid-stride loop covers any length.
template <class T>
__global__ void __launch_bounds__(256) pad_pair_kernel(const T* __restrict__ x,
                                                       const T* __restrict__ y,
                                                       T* __restrict__ px, T* __restrict__ py,
                                                       long long n, long long n2) {
  const T* s = blockIdx.y ? y : x;
  T* d = blockIdx.y ? py : px;
#pragma unroll 1
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = i < n ? s[i] : T(0);
}

static int ceil_log2(size_t n) {
  int D = 0;
  while (((size_t)1 << D) < n) ++D;
  return D;
}

// Bytes of one zero-padded operand, rounded so the next region stays
// 256-byte aligned; 0 when N is a power of two (no padding needed).
static size_t pad_bytes(size_t N, hc_dtype dt) {
  const int D = ceil_log2(N);
  if (((size_t)1 << D) == N) return 0;
  return align_up(elem_size(dt) << D, 256);
}

}  // namespace hc

extern "C" size_t hc_carryfree_workspace_size(size_t N, hc_dtype dtype) {
  using namespace hc;
  if (N == 0 || elem_size(dtype) == 0) return 0;
  const int D = ceil_log2(N);
  if (D > HC_MAX_D) return 0;
  return 2 * pad_bytes(N, dtype) + hc_workspace_size(D, dtype);
}

extern "C" hc_status hc_carryfree(const void* x, const void* y, void* z, size_t N, hc_dtype dtype,
                                  void* workspace, size_t ws_bytes, hc_stream_t stream) {
  using namespace hc;
  const size_t es = elem_size(dtype);
  if (es == 0) return HC_ERR_DTYPE;
  if (N == 0) return HC_ERR_ARG;
  const int D = ceil_log2(N);
  if (D > HC_MAX_D) return HC_ERR_ARG;
  if (!x || !y || !z) return HC_ERR_ARG;
  if (!aligned(x, 16) || !aligned(y, 16) || !aligned(z, 16)) return HC_ERR_ALIGN;
  const size_t pad = pad_bytes(N, dtype);
  if (pad == 0)  // N = 2^D: the hypercube convolution of the vectors as they are
    return convolve_checked(x, y, z, D, dtype, workspace, ws_bytes, (cudaStream_t)stream,
                            nullptr);
  const size_t need = hc_carryfree_workspace_size(N, dtype);
  if (ws_bytes < need) return HC_ERR_WORKSPACE;
  if (!workspace) return HC_ERR_ARG;
  if (!aligned(workspace, 256)) return HC_ERR_ALIGN;
  const size_t nx = es * N, nz = es * pow3z(D);
  if (overlaps(z, nz, x, nx) || overlaps(z, nz, y, nx)) return HC_ERR_ALIAS;
  if (overlaps(workspace, need, z, nz) || overlaps(workspace, need, x, nx) ||
      overlaps(workspace, need, y, nx))
    return HC_ERR_ALIAS;
  unsigned char* ws = (unsigned char*)workspace;
  void* px = ws;
  void* py = ws + pad;
  unsigned char* conv_ws = ws + 2 * pad;
  const size_t conv_bytes = ws_bytes - 2 * pad;
  cudaStream_t st = (cudaStream_t)stream;
  const long long n2 = (long long)1 << D;
  long long blocks = (n2 + 255) / 256;
  const long long cap = (long long)device_caps().sms * 8;
  if (blocks > cap) blocks = cap;
  {
    ProfileScope prof(st, "pad");
    if (es == 8)
      pad_pair_kernel<unsigned long long><<<dim3((unsigned)blocks, 2), 256, 0, st>>>(
          (const unsigned long long*)x, (const unsigned long long*)y, (unsigned long long*)px,
          (unsigned long long*)py, (long long)N, n2);
    else
      pad_pair_kernel<unsigned int><<<dim3((unsigned)blocks, 2), 256, 0, st>>>(
          (const unsigned int*)x, (const unsigned int*)y, (unsigned int*)px, (unsigned int*)py,
          (long long)N, n2);
    const hc_status s = record_cuda_error(cudaGetLastError());
    if (s != HC_OK) return s;
  }
  return convolve_checked(px, py, z, D, dtype, conv_bytes ? conv_ws : nullptr, conv_bytes, st,
                          nullptr);
}
