// Forward hypercube convolution on sm_103a: z = x * y (arXiv 1608.00206,
// Methods section).
//
// Schedule for D axes, with the C innermost axes handled inside one CTA tile
// and the a = D - C outer axes handled by whole-array passes:
//   K1 eval_pass   : evaluate the outer axes, <= 3 per pass, outer first:
//                    x [2^a][2^C] -> Xo [3^a][2^C]   (same for y)
//   K2 tile_conv   : per outer index alpha, evaluate the C inner axes, take
//                    the 3^C products, interpolate the C inner axes (innermost
//                    first) in shared memory and registers, write W[alpha][:]
//   K3 interp_pass : interpolate the outer axes in place on the 3^D array,
//                    <= 6 axes per pass, innermost pass first
// This is the recurrence's own per-element operation order (evaluation axis
// 1 first, interpolation axis D first), so results are bitwise those of the
// sequential recurrence.  The in-place listing of the paper is not used: x
// and y are never written.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "hc_common.cuh"
#include "hc_profile.cuh"
#include "hc_forward.cuh"
#include "hc_kernels.cuh"
#include "hc_tile.cuh"
#include <type_traits>

namespace hc {

// ---------------------------------------------------------------------------
// K2 kernel: one tile per outer index alpha (grid-stride over tiles).
template <class In>
struct RowLoader {
  const In* x;
  const In* y;
  __device__ __forceinline__ In operator()(int op, int i) const { return op ? y[i] : x[i]; }
};

template <class M, int C, bool FINAL>
__global__ void __launch_bounds__(256) tile_conv_kernel(const typename M::In* __restrict__ X,
                                                        const typename M::In* __restrict__ Y,
                                                        void* __restrict__ out_, long long ntiles) {
  typedef typename M::In In;
  typedef typename std::conditional<FINAL, typename M::Out, typename M::W>::type O;
  extern __shared__ __align__(16) unsigned char smem[];
#pragma unroll 1
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    RowLoader<In> ld{X + t * p2(C), Y + t * p2(C)};
    tile_body<M, C, FINAL>(ld, reinterpret_cast<O*>(out_) + t * p3(C), smem);
  }
}

// D = 0: z[0] = x[0] * y[0].
template <class M>
__global__ void scalar_conv_kernel(const typename M::In* x, const typename M::In* y,
                                   typename M::Out* z) {
  if (threadIdx.x == 0 && blockIdx.x == 0) z[0] = M::out(M::mul(x[0], y[0]));
}

// ---------------------------------------------------------------------------
// K3 kernel: interpolate k = K1 + K2 consecutive axes of a [hi][3^k][lo]
// array; a CTA tile is all 3^k rows of L consecutive columns of one h.
// src and dst may be the same array (every tile reads its elements before
// writing any; tiles are disjoint).
template <class M, int K1, int K2, int L, bool FINAL>
__global__ void __launch_bounds__(256) interp_pass_kernel(const typename M::W* src, void* dst_,
                                                          long long hi, long long lo) {
  extern __shared__ __align__(16) unsigned char smem[];
  const long long ctiles = (lo + L - 1) / L;
  const long long ntiles = hi * ctiles;
#pragma unroll 1
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long h = tile / ctiles;
    const long long l0 = (tile - h * ctiles) * L;
    interp_tile_body<M, K1, K2, L, FINAL, false>(src, dst_, h * p3(K1 + K2) * lo + l0, l0, lo,
                                                 smem);
  }
}

// ---------------------------------------------------------------------------
// Host side.

template <class M>
struct ColsPerTile {
  static constexpr int L = (sizeof(typename M::W) == 4) ? 32 : 16;
};

template <class M>
static int max_tile_axes() {
  return sizeof(typename M::W) == 4 ? 9 : 8;
}

static int threads_for_tile(int C) { return C >= 6 ? 256 : (C >= 4 ? 128 : 32); }

template <class M, int C, bool FINAL>
static cudaError_t launch_tile_c(const typename M::In* X, const typename M::In* Y, void* out,
                                 long long ntiles, cudaStream_t st) {
  const size_t smem = TileSmem<M, C>::bytes;
  auto k = tile_conv_kernel<M, C, FINAL>;
  ProfileScope prof(st, "tile_conv");
  cudaError_t e = prep_kernel(k, smem);
  if (e != cudaSuccess) return e;
  const int threads = threads_for_tile(C);
  k<<<grid_for(k, threads, smem, ntiles), threads, smem, st>>>(X, Y, out, ntiles);
  return cudaGetLastError();
}

template <class M, bool FINAL>
static cudaError_t launch_tile(int C, const typename M::In* X, const typename M::In* Y, void* out,
                               long long ntiles, cudaStream_t st) {
  switch (C) {
    case 1: return launch_tile_c<M, 1, FINAL>(X, Y, out, ntiles, st);
    case 2: return launch_tile_c<M, 2, FINAL>(X, Y, out, ntiles, st);
    case 3: return launch_tile_c<M, 3, FINAL>(X, Y, out, ntiles, st);
    case 4: return launch_tile_c<M, 4, FINAL>(X, Y, out, ntiles, st);
    case 5: return launch_tile_c<M, 5, FINAL>(X, Y, out, ntiles, st);
    case 6: return launch_tile_c<M, 6, FINAL>(X, Y, out, ntiles, st);
    case 7: return launch_tile_c<M, 7, FINAL>(X, Y, out, ntiles, st);
    case 8: return launch_tile_c<M, 8, FINAL>(X, Y, out, ntiles, st);
    case 9:
      if constexpr (sizeof(typename M::W) == 4) return launch_tile_c<M, 9, FINAL>(X, Y, out, ntiles, st);
      return cudaErrorInvalidValue;
  }
  return cudaErrorInvalidValue;
}

template <class M, int K1, int K2, bool FINAL>
static cudaError_t launch_interp_k(const typename M::W* src, void* dst, long long hi, long long lo,
                                   cudaStream_t st) {
  constexpr int L = ColsPerTile<M>::L;
  const size_t smem = K1 > 0 ? sizeof(typename M::W) * (size_t)p3(K1 + K2) * L : 0;
  auto k = interp_pass_kernel<M, K1, K2, L, FINAL>;
  ProfileScope prof(st, "interp_pass");
  cudaError_t e = prep_kernel(k, smem);
  if (e != cudaSuccess) return e;
  int threads = K1 > 0 ? 256 : L;
  if (K1 > 0 && p3(K1) * L < 256 && p3(K2) * L < 256) threads = 128;
  const long long ntiles = hi * ((lo + L - 1) / L);
  k<<<grid_for(k, threads, smem, ntiles), threads, smem, st>>>(src, dst, hi, lo);
  return cudaGetLastError();
}

template <class M, bool FINAL>
static cudaError_t launch_interp(int k, const typename M::W* src, void* dst, long long hi,
                                 long long lo, cudaStream_t st) {
  switch (k) {
    case 1: return launch_interp_k<M, 0, 1, FINAL>(src, dst, hi, lo, st);
    case 2: return launch_interp_k<M, 0, 2, FINAL>(src, dst, hi, lo, st);
    case 3: return launch_interp_k<M, 0, 3, FINAL>(src, dst, hi, lo, st);
    case 4: return launch_interp_k<M, 1, 3, FINAL>(src, dst, hi, lo, st);
    case 5: return launch_interp_k<M, 2, 3, FINAL>(src, dst, hi, lo, st);
    case 6: return launch_interp_k<M, 3, 3, FINAL>(src, dst, hi, lo, st);
  }
  return cudaErrorInvalidValue;
}

// The plan: which axes go where, and the workspace layout.
FwdPlan make_fwd_plan(int D, hc_dtype dt, int c_req, int kmax_req) {
  FwdPlan p;
  memset(&p, 0, sizeof(p));
  p.D = D;
  p.dtype = dt;
  const int cmax = (dt == HC_FP32) ? 9 : 8;
  int C = c_req > 0 ? c_req : cmax;
  if (C > cmax) C = cmax;
  if (C > D) C = D;
  p.C = C;
  p.a = D - C;
  int kmax = kmax_req > 0 ? kmax_req : 6;
  if (kmax > 6) kmax = 6;
  const size_t in_sz = (dt == HC_INT64 || dt == HC_FP64) ? 8 : 4;
  const size_t w_sz = (dt == HC_FP32) ? 4 : 8;
  // K1 passes: groups of <= 3 outer axes, outer first.
  for (int d = 0; d < p.a; d += 3) {
    const int k = (p.a - d) < 3 ? (p.a - d) : 3;
    p.eval_d0[p.n_eval] = d;
    p.eval_k[p.n_eval] = k;
    ++p.n_eval;
  }
  // Eval buffers: the last pass lands in Xo/Yo, earlier passes alternate.
  size_t xo = p.a > 0 ? pow3z(p.a) << C : 0;
  size_t tmax = 0;
  for (int i = 0; i < p.n_eval; ++i) {
    const int done = p.eval_d0[i] + p.eval_k[i];
    const size_t n = pow3z(done) << (D - done);
    const bool to_final = ((p.n_eval - 1 - i) % 2) == 0;
    p.eval_to_final[i] = to_final;
    if (!to_final && n > tmax) tmax = n;
  }
  // K3 passes: ceil(a / kmax) balanced groups, innermost first.
  if (p.a > 0) {
    const int np = (p.a + kmax - 1) / kmax;
    int end = p.a;
    for (int i = 0; i < np; ++i) {
      const int rem_groups = np - i;
      const int k = (end + rem_groups - 1) / rem_groups;  // ceil(end / rem)
      p.interp_d0[i] = end - k;
      p.interp_k[i] = k;
      end -= k;
    }
    p.n_interp = np;
  }
  size_t off = kWsHeader;
  p.off_xo = off;
  off = align_up(off + xo * in_sz, 256);
  p.off_yo = off;
  off = align_up(off + xo * in_sz, 256);
  p.off_tx = off;
  off = align_up(off + tmax * in_sz, 256);
  p.off_ty = off;
  off = align_up(off + tmax * in_sz, 256);
  p.off_w = off;
  if (dt == HC_FP32_MIXED && p.a > 0) off = align_up(off + pow3z(D) * w_sz, 256);
  p.ws_bytes = off;
  return p;
}

template <class M>
static cudaError_t run_forward(const FwdPlan& p, const void* x, const void* y, void* z,
                               unsigned char* ws, cudaStream_t st) {
  typedef typename M::In In;
  typedef typename M::W W;
  const int D = p.D, C = p.C, a = p.a;
  if (D == 0) {
    ProfileScope prof(st, "scalar_conv");
    scalar_conv_kernel<M><<<1, 32, 0, st>>>((const In*)x, (const In*)y, (typename M::Out*)z);
    return cudaGetLastError();
  }
  const In* X = (const In*)x;
  const In* Y = (const In*)y;
  In* Xo = (In*)(ws + p.off_xo);
  In* Yo = (In*)(ws + p.off_yo);
  In* Tx = (In*)(ws + p.off_tx);
  In* Ty = (In*)(ws + p.off_ty);
  cudaError_t e;
  // K1
  for (int i = 0; i < p.n_eval; ++i) {
    const int d0 = p.eval_d0[i], k = p.eval_k[i];
    const long long hi = (long long)pow3z(d0);
    const long long lo = (long long)1 << (D - d0 - k);
    In* dx = p.eval_to_final[i] ? Xo : Tx;
    In* dy = p.eval_to_final[i] ? Yo : Ty;
    e = launch_eval<M>(k, X, Y, dx, dy, hi, lo, st);
    if (e != cudaSuccess) return e;
    X = dx;
    Y = dy;
  }
  // K2
  const long long ntiles = (long long)pow3z(a);
  const bool mixed_ws = (sizeof(W) != sizeof(typename M::Out)) && a > 0;
  W* Wbuf = mixed_ws ? (W*)(ws + p.off_w) : (W*)z;
  if (a == 0)
    e = launch_tile<M, true>(C, X, Y, z, ntiles, st);
  else
    e = launch_tile<M, false>(C, X, Y, Wbuf, ntiles, st);
  if (e != cudaSuccess) return e;
  // K3
  for (int i = 0; i < p.n_interp; ++i) {
    const int d0 = p.interp_d0[i], k = p.interp_k[i];
    const long long hi = (long long)pow3z(d0);
    const long long lo = (long long)pow3z(a - d0 - k) * (long long)pow3z(C);
    const bool last = (i == p.n_interp - 1);
    if (last && mixed_ws)
      e = launch_interp<M, true>(k, Wbuf, z, hi, lo, st);
    else
      e = launch_interp<M, false>(k, Wbuf, Wbuf, hi, lo, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t forward_dispatch(const FwdPlan& p, const void* x, const void* y, void* z,
                             unsigned char* ws, cudaStream_t st) {
  switch (p.dtype) {
    case HC_INT64: return run_forward<ModeI64>(p, x, y, z, ws, st);
    case HC_FP64: return run_forward<ModeF64>(p, x, y, z, ws, st);
    case HC_FP32: return run_forward<ModeF32>(p, x, y, z, ws, st);
    case HC_FP32_MIXED: return run_forward<ModeMixed>(p, x, y, z, ws, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hc

// ---------------------------------------------------------------------------
// C ABI

extern "C" size_t hc_workspace_size(int D, hc_dtype dtype) {
  if (D < 0 || D > HC_MAX_D || hc::elem_size(dtype) == 0) return 0;
  return hc::make_fwd_plan(D, dtype, 0, 0).ws_bytes;
}

namespace hc {

hc_status convolve_checked(const void* x, const void* y, void* z, int D, hc_dtype dtype,
                           void* workspace, size_t ws_bytes, cudaStream_t stream, int c_req,
                           int kmax_req) {
  if (D < 0 || D > HC_MAX_D) return HC_ERR_ARG;
  const size_t es = elem_size(dtype);
  if (es == 0) return HC_ERR_DTYPE;
  if (!x || !y || !z) return HC_ERR_ARG;
  if (!aligned(x, 16) || !aligned(y, 16) || !aligned(z, 16)) return HC_ERR_ALIGN;
  const FwdPlan p = make_fwd_plan(D, dtype, c_req, kmax_req);
  if (ws_bytes < p.ws_bytes) return HC_ERR_WORKSPACE;
  if (p.ws_bytes > 0 && !workspace) return HC_ERR_ARG;
  if (workspace && !aligned(workspace, 256)) return HC_ERR_ALIGN;
  const size_t nx = es << D, nz = es * pow3z(D);
  if (overlaps(z, nz, x, nx) || overlaps(z, nz, y, nx)) return HC_ERR_ALIAS;
  if (workspace && p.ws_bytes > 0 &&
      (overlaps(workspace, p.ws_bytes, z, nz) || overlaps(workspace, p.ws_bytes, x, nx) ||
       overlaps(workspace, p.ws_bytes, y, nx)))
    return HC_ERR_ALIAS;
  return record_cuda_error(forward_dispatch(p, x, y, z, (unsigned char*)workspace, stream));
}

}  // namespace hc

extern "C" size_t hc_workspace_size_config(int D, hc_dtype dtype, int c, int kmax) {
  if (D < 0 || D > HC_MAX_D || hc::elem_size(dtype) == 0) return 0;
  return hc::make_fwd_plan(D, dtype, c, kmax).ws_bytes;
}

extern "C" hc_status hc_convolve_config(const void* x, const void* y, void* z, int D,
                                        hc_dtype dtype, int c, int kmax, void* workspace,
                                        size_t ws_bytes, hc_stream_t stream) {
  if (c < 0 || c > (dtype == HC_FP32 ? 9 : 8) || kmax < 0 || kmax > 6) return HC_ERR_ARG;
  return hc::convolve_checked(x, y, z, D, dtype, workspace, ws_bytes, (cudaStream_t)stream, c,
                              kmax);
}

extern "C" hc_status hc_convolve(const void* x, const void* y, void* z, int D, hc_dtype dtype,
                                 void* workspace, size_t ws_bytes, hc_stream_t stream) {
  return hc::convolve_checked(x, y, z, D, dtype, workspace, ws_bytes, (cudaStream_t)stream, 0, 0);
}
