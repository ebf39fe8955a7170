// The low-workspace schedule (the paper's memory-saving recursion, Algorithm
// 2's pairing of sub-problems, done correctly): the top r axes are split on
// the host the way the Methods recurrence splits them, one leaf at a time.
// For every digit string a of the top r axes, the leaf inputs are x and y
// evaluated on those axes at a -- per element the sum, as a pairwise tree
// whose first level pairs the outermost digit-1 axis, of the 2^(#1 in a)
// sub-cubes that digit 0 / 1 / 2 select -- and the leaf, a convolution of
// D - r axes, runs the whole-array-pass schedule straight into z's slice a
// (3^(D-r) contiguous outputs).  Whole-array passes then interpolate the top
// r axes in place.  Per element these are the recurrence's operations in its
// order (evaluation axis 1 first, interpolation axis D first), so results
// are bitwise those of every other schedule.  Workspace: the two leaf inputs
// (2^(D-r) elements each) plus one leaf's own workspace (its operands on its
// D - r - c outer axes: 3 MB for a 14-axis int64 leaf) instead of the
// 3^(D-c) * 2^c operand arrays of the other schedules (2.2 GB at D = 20), at
// the same number of sweeps over z when D - r is the tile axes plus whole
// passes (r = 6 at D = 20: leaves of 14 axes).  Exact and plain dtypes only (the float-float
// forms keep a 3^D intermediate).
#include <cstring>

#include "hc_common.cuh"
#include "hc_forward.cuh"
#include "hc_kernels.cuh"
#include "hc_profile.cuh"

namespace hc {

constexpr int kLowMemMaxTop = 6;
constexpr int kLeafMaxOnes = 6;  // sub-cubes summed per leaf element: at most 2^6

// Offsets (elements) of the 2^n sub-cubes summed into a leaf element: entry j
// has, for t = 0..n-1, bit (n - 1 - t) of j as its bit on the t-th digit-1
// axis (outermost first).
struct LeafSlices {
  long long off[1 << kLeafMaxOnes];
};

// The pairwise tree of 2^N values, first level pairing j with j + 2^(N-1)
// (the outermost digit-1 axis), as the recurrence nests its sums.
template <class M, int N>
__device__ __forceinline__ typename M::In leaf_sum(const typename M::In* s, const LeafSlices& o,
                                                  long long i) {
  typedef typename M::In In;
  In v[1 << N];
#pragma unroll
  for (int j = 0; j < (1 << N); ++j) v[j] = s[o.off[j] + i];
#pragma unroll
  for (int L = 0; L < N; ++L) {
    const int stride = 1 << (N - 1 - L);
#pragma unroll
    for (int j = 0; j < stride; ++j) v[j] = M::add(v[j], v[j + stride]);
  }
  return v[0];
}

template <class M, int N>
__global__ void __launch_bounds__(256) leaf_eval_kernel(const typename M::In* __restrict__ x,
                                                        const typename M::In* __restrict__ y,
                                                        typename M::In* __restrict__ xl,
                                                        typename M::In* __restrict__ yl,
                                                        LeafSlices o, long long n) {
  const typename M::In* s = blockIdx.y ? y : x;
  typename M::In* d = blockIdx.y ? yl : xl;
#pragma unroll 1
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = leaf_sum<M, N>(s, o, i);
}

template <class M>
static cudaError_t launch_leaf_eval(int nones, const typename M::In* x, const typename M::In* y,
                                    typename M::In* xl, typename M::In* yl, const LeafSlices& o,
                                    long long n, cudaStream_t st) {
  ProfileScope prof(st, "leaf_eval");
  long long blocks = (n + 255) / 256;
  const long long cap = (long long)device_caps().sms * 8;
  if (blocks > cap) blocks = cap;
  const dim3 g((unsigned)blocks, 2);
  switch (nones) {
    case 0: leaf_eval_kernel<M, 0><<<g, 256, 0, st>>>(x, y, xl, yl, o, n); break;
    case 1: leaf_eval_kernel<M, 1><<<g, 256, 0, st>>>(x, y, xl, yl, o, n); break;
    case 2: leaf_eval_kernel<M, 2><<<g, 256, 0, st>>>(x, y, xl, yl, o, n); break;
    case 3: leaf_eval_kernel<M, 3><<<g, 256, 0, st>>>(x, y, xl, yl, o, n); break;
    case 4: leaf_eval_kernel<M, 4><<<g, 256, 0, st>>>(x, y, xl, yl, o, n); break;
    case 5: leaf_eval_kernel<M, 5><<<g, 256, 0, st>>>(x, y, xl, yl, o, n); break;
    case 6: leaf_eval_kernel<M, 6><<<g, 256, 0, st>>>(x, y, xl, yl, o, n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// r top axes (1..6) handled leaf by leaf; the leaves run the whole-array-pass
// plan of D - r axes (c tile axes, k axes per pass, per-element row copies:
// a leaf's slice of z starts at any element, so no 16-byte row copies); the
// top axes are interpolated by passes of at most k axes of width cols_outer.
LowPlan make_lowmem_plan(int D, hc_dtype dt, int r, int c_req, int kmax_req, int cols,
                         int cols_outer) {
  LowPlan p;
  memset(&p, 0, sizeof(p));
  p.D = D;
  p.dtype = dt;
  p.r = r;
  p.ok = r >= 1 && r <= kLowMemMaxTop && D - r >= 1 &&
         (dt == HC_INT64 || dt == HC_FP64 || dt == HC_FP32);
  if (!p.ok) return p;
  p.leaf = make_fwd_plan(D - r, dt, c_req, kmax_req);
  p.leaf.cols = cols < 0 ? -cols : cols;
  p.leaf.cols_outer = p.leaf.cols;
  const int kmax = kmax_req > 0 ? (kmax_req < 6 ? kmax_req : 6) : 6;
  const int np = (r + kmax - 1) / kmax;
  int end = r;
  for (int i = 0; i < np; ++i) {
    const int rem = np - i;
    const int k = (end + rem - 1) / rem;
    p.top_d0[i] = end - k;
    p.top_k[i] = k;
    end -= k;
  }
  p.n_top = np;
  p.cols_top = cols_outer ? cols_outer : cols;
  const size_t in_sz = in_size(dt);
  size_t off = kWsHeader;
  p.off_xl = off;
  off = align_up(off + (in_sz << (D - r)), 256);
  p.off_yl = off;
  off = align_up(off + (in_sz << (D - r)), 256);
  p.off_leaf = off;
  off = align_up(off + p.leaf.ws_bytes, 256);
  p.ws_bytes = off;
  return p;
}

// w: the caller's array for the intermediate (hc_convolve_out; z then gets
// only the last pass's stores); nullptr: the intermediate is z itself.
template <class M>
static cudaError_t run_lowmem(const LowPlan& p, const void* x, const void* y, void* z,
                              unsigned char* ws, cudaStream_t st, void* w) {
  typedef typename M::In In;
  typedef typename M::Out Out;
  Out* Wz = (Out*)(w ? w : z);
  const int D = p.D, r = p.r, n = D - r;
  In* xl = (In*)(ws + p.off_xl);
  In* yl = (In*)(ws + p.off_yl);
  const long long leaf_in = 1ll << n;
  const size_t leaf_out = pow3z(n);
  cudaError_t e;
  for (long long a = 0; a < (long long)pow3z(r); ++a) {
    int dig[kLowMemMaxTop];
    long long aa = a;
    for (int d = r - 1; d >= 0; --d) {
      dig[d] = (int)(aa % 3);
      aa /= 3;
    }
    long long base = 0;
    long long one_bits[kLowMemMaxTop];
    int nones = 0;
    for (int d = 0; d < r; ++d) {
      const long long bit = 1ll << (D - 1 - d);  // axis d + 1's weight in x's flat index
      if (dig[d] == 2) base += bit;
      if (dig[d] == 1) one_bits[nones++] = bit;
    }
    LeafSlices o;
    for (int j = 0; j < (1 << nones); ++j) {
      long long off = base;
      for (int t = 0; t < nones; ++t)
        if ((j >> (nones - 1 - t)) & 1) off += one_bits[t];
      o.off[j] = off;
    }
    e = launch_leaf_eval<M>(nones, (const In*)x, (const In*)y, xl, yl, o, leaf_in, st);
    if (e != cudaSuccess) return e;
    e = forward_dispatch(p.leaf, xl, yl, Wz + (size_t)a * leaf_out, ws + p.off_leaf, st);
    if (e != cudaSuccess) return e;
  }
  for (int i = 0; i < p.n_top; ++i) {
    const int d0 = p.top_d0[i], k = p.top_k[i];
    const long long hi = (long long)pow3z(d0);
    const long long lo = (long long)pow3z(r - d0 - k) * (long long)leaf_out;
    if (w && i == p.n_top - 1)
      e = launch_interp<M, true>(k, p.cols_top, (const typename M::W*)Wz, z, hi, lo, st);
    else
      e = launch_interp<M, false>(k, p.cols_top, (const typename M::W*)Wz, Wz, hi, lo, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t lowmem_dispatch(const LowPlan& p, const void* x, const void* y, void* z,
                            unsigned char* ws, cudaStream_t st, void* w) {
  switch (p.dtype) {
    case HC_INT64: return run_lowmem<ModeI64>(p, x, y, z, ws, st, w);
    case HC_FP64: return run_lowmem<ModeF64>(p, x, y, z, ws, st, w);
    case HC_FP32: return run_lowmem<ModeF32>(p, x, y, z, ws, st, w);
    default: break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace hc
