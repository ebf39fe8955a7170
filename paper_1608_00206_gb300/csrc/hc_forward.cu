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
#include "hc_forward.cuh"
#include "hc_kernels.cuh"

namespace hc {

// ---------------------------------------------------------------------------
// K2: the fused tile.  C inner axes, split into G = ceil(C/3) groups of at
// most 3 axes (the outermost group takes the remainder).  Per tile alpha:
//   stage 0      : global Xo[alpha], Yo[alpha] -> evaluate group 0 -> smem
//   stage 1      : (G = 3) evaluate group 1 in smem
//   fused stage  : evaluate the innermost group, multiply, interpolate the
//                  innermost group, all in registers -> W tile in smem
//   interp stages: interpolate group G-2 .. 1 in smem, then group 0 from smem
//                  straight to global memory
// Every stage gives consecutive threads consecutive innermost indices, so
// shared-memory accesses are bank-conflict free (odd strides) and global
// accesses are contiguous per warp.  The buffer feeding the fused stage is
// stored transposed ([2^g][3^(C-g)]) so that its pencils, which are
// contiguous in the natural layout, are read with unit stride across threads.
template <int C>
struct TileShape {
  static constexpr int G = (C + 2) / 3;
  static constexpr int g0 = C - 3 * (G - 1);          // outermost group
  static constexpr int gL = (G == 1) ? C : 3;         // innermost group
  static constexpr int nLastPencils = p3(C - gL);     // pencils of the fused stage
};

template <class M, int C>
struct TileSmem {
  typedef typename M::In In;
  typedef typename M::W W;
  // W tile; the stage-0 buffer of a 3-group tile lives inside it.
  static constexpr size_t kW = sizeof(W) * (size_t)p3(C);
  // transposed buffer feeding the fused stage, per operand
  static constexpr size_t kLast = sizeof(In) * (size_t)p2(TileShape<C>::gL) * p3(C - TileShape<C>::gL);
  static constexpr size_t kS1 = TileShape<C>::G == 3 ? 2 * sizeof(In) * (size_t)p3(TileShape<C>::g0) * p2(C - TileShape<C>::g0) : 0;
  static_assert(kS1 <= kW, "stage-0 buffer must fit inside the W tile");
  static constexpr size_t bytes = kW + (TileShape<C>::G >= 2 ? 2 * kLast : 0);
};

template <class M, int C, bool FINAL>
__global__ void __launch_bounds__(256) tile_conv_kernel(const typename M::In* __restrict__ X,
                                                        const typename M::In* __restrict__ Y,
                                                        void* __restrict__ out_, long long ntiles) {
  typedef typename M::In In;
  typedef typename M::W W;
  typedef typename M::Out Out;
  typedef TileShape<C> S;
  extern __shared__ __align__(16) unsigned char smem[];
  W* Ws = reinterpret_cast<W*>(smem);
  In* LastX = reinterpret_cast<In*>(smem + TileSmem<M, C>::kW);
  In* LastY = LastX + p2(S::gL) * p3(C - S::gL);
  In* S1 = reinterpret_cast<In*>(smem);  // G == 3 only; aliases the W tile
  const int tid = threadIdx.x;
  const int nt = blockDim.x;

#pragma unroll 1
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const In* xr = X + t * p2(C);
    const In* yr = Y + t * p2(C);
    if constexpr (S::G == 1) {
      // C <= 3: one pencil, straight from global to global.
      if (tid == 0) {
        In a[p3(C)], b[p3(C)];
#pragma unroll
        for (int i = 0; i < p2(C); ++i) {
          a[i] = xr[i];
          b[i] = yr[i];
        }
        eval_pencil<M, C>(a);
        eval_pencil<M, C>(b);
        W w[p3(C)];
#pragma unroll
        for (int j = 0; j < p3(C); ++j) w[j] = M::mul(a[j], b[j]);
        interp_pencil<M, C>(w);
        if constexpr (FINAL) {
          Out* o = reinterpret_cast<Out*>(out_) + t * p3(C);
#pragma unroll
          for (int j = 0; j < p3(C); ++j) o[j] = M::out(w[j]);
        } else {
          W* o = reinterpret_cast<W*>(out_) + t * p3(C);
#pragma unroll
          for (int j = 0; j < p3(C); ++j) o[j] = w[j];
        }
      }
    } else {
      // ---- stage 0: evaluate group 0 (g0 axes) from global memory.
      {
        constexpr int R = p2(C - S::g0);  // pencils per operand
        #pragma unroll 1
        for (int p = tid; p < 2 * R; p += nt) {
          const int op = p / R, r = p - op * R;
          const In* src = op ? yr : xr;
          In v[p3(S::g0)];
#pragma unroll
          for (int b = 0; b < p2(S::g0); ++b) v[b] = src[b * R + r];
          eval_pencil<M, S::g0>(v);
          if constexpr (S::G == 2) {
            // next is the fused stage: transposed [2^gL][3^g0], r = last-group bits
            In* d = op ? LastY : LastX;
#pragma unroll
            for (int j = 0; j < p3(S::g0); ++j) d[r * p3(S::g0) + j] = v[j];
          } else {
            In* d = S1 + op * (p3(S::g0) * R);
#pragma unroll
            for (int j = 0; j < p3(S::g0); ++j) d[j * R + r] = v[j];
          }
        }
      }
      __syncthreads();
      // ---- stage 1 (G == 3): evaluate group 1 (3 axes) in shared memory.
      if constexpr (S::G == 3) {
        constexpr int O = p3(S::g0);
        constexpr int R = p2(S::gL);  // remaining binary axes (innermost group)
        constexpr int NP = O * R;
        #pragma unroll 1
        for (int p = tid; p < 2 * NP; p += nt) {
          const int op = p / NP, q = p - op * NP;
          const int o = q / R, r = q - o * R;
          const In* s = S1 + op * (O * 8 * R);
          In v[27];
#pragma unroll
          for (int b = 0; b < 8; ++b) v[b] = s[(o * 8 + b) * R + r];
          eval_pencil<M, 3>(v);
          In* d = op ? LastY : LastX;
#pragma unroll
          for (int j = 0; j < 27; ++j) d[r * (O * 27) + o * 27 + j] = v[j];
        }
        __syncthreads();
      }
      // ---- fused stage: evaluate innermost group, multiply, interpolate it.
      {
        constexpr int NO = S::nLastPencils;
        #pragma unroll 1
        for (int o = tid; o < NO; o += nt) {
          In a[27], b[27];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            a[q] = LastX[q * NO + o];
            b[q] = LastY[q * NO + o];
          }
          eval_pencil<M, 3>(a);
          eval_pencil<M, 3>(b);
          W w[27];
#pragma unroll
          for (int j = 0; j < 27; ++j) w[j] = M::mul(a[j], b[j]);
          interp_pencil<M, 3>(w);
#pragma unroll
          for (int j = 0; j < 27; ++j) Ws[o * 27 + j] = w[j];
        }
      }
      __syncthreads();
      // ---- interpolate group 1 (G == 3) in shared memory.
      if constexpr (S::G == 3) {
        constexpr int O = p3(S::g0), R = 27;
        #pragma unroll 1
        for (int p = tid; p < O * R; p += nt) {
          const int o = p / R, r = p - o * R;
          W v[27];
#pragma unroll
          for (int j = 0; j < 27; ++j) v[j] = Ws[(o * 27 + j) * R + r];
          interp_pencil<M, 3>(v);
#pragma unroll
          for (int j = 0; j < 27; ++j) Ws[(o * 27 + j) * R + r] = v[j];
        }
        __syncthreads();
      }
      // ---- interpolate group 0 and write the tile to global memory.
      {
        constexpr int R = p3(C - S::g0);
        #pragma unroll 1
        for (int r = tid; r < R; r += nt) {
          W v[p3(S::g0)];
#pragma unroll
          for (int j = 0; j < p3(S::g0); ++j) v[j] = Ws[j * R + r];
          interp_pencil<M, S::g0>(v);
          if constexpr (FINAL) {
            Out* o = reinterpret_cast<Out*>(out_) + t * p3(C);
#pragma unroll
            for (int j = 0; j < p3(S::g0); ++j) o[j * R + r] = M::out(v[j]);
          } else {
            W* o = reinterpret_cast<W*>(out_) + t * p3(C);
#pragma unroll
            for (int j = 0; j < p3(S::g0); ++j) o[j * R + r] = v[j];
          }
        }
      }
      __syncthreads();  // the next tile reuses shared memory
    }
  }
}

// D = 0: z[0] = x[0] * y[0].
template <class M>
__global__ void scalar_conv_kernel(const typename M::In* x, const typename M::In* y,
                                   typename M::Out* z) {
  if (threadIdx.x == 0 && blockIdx.x == 0) z[0] = M::out(M::mul(x[0], y[0]));
}

// ---------------------------------------------------------------------------
// K3: interpolate k = K1 + K2 consecutive axes of a [hi][3^k][lo] array.
// A CTA tile is all 3^k rows of L consecutive columns of one h.  Round 1
// interpolates the inner K2 axes in registers (pencils read straight from
// global memory, stride lo), round 2 the outer K1 axes after a pass through
// shared memory.  Consecutive threads take consecutive columns.  src and dst
// may be the same array (in place) -- every tile reads all its elements
// before writing any, and tiles are disjoint.
template <class M, int K1, int K2, int L, bool FINAL>
__global__ void __launch_bounds__(256) interp_pass_kernel(const typename M::W* src, void* dst_,
                                                          long long hi, long long lo) {
  typedef typename M::W W;
  typedef typename M::Out Out;
  constexpr int K = K1 + K2;
  constexpr int ROWS = p3(K);
  extern __shared__ __align__(16) unsigned char smem[];
  W* T = reinterpret_cast<W*>(smem);
  const long long ctiles = (lo + L - 1) / L;
  const long long ntiles = hi * ctiles;
  const int tid = threadIdx.x, nt = blockDim.x;

#pragma unroll 1
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long h = tile / ctiles;
    const long long l0 = (tile - h * ctiles) * L;
    const long long base = h * ROWS * lo + l0;
    if constexpr (K1 == 0) {
#pragma unroll 1
      for (int l = tid; l < L; l += nt) {
        if (l0 + l >= lo) continue;
        W v[p3(K2)];
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) v[j] = src[base + j * lo + l];
        interp_pencil<M, K2>(v);
        if constexpr (FINAL) {
          Out* d = reinterpret_cast<Out*>(dst_);
#pragma unroll
          for (int j = 0; j < p3(K2); ++j) d[base + j * lo + l] = M::out(v[j]);
        } else {
          W* d = reinterpret_cast<W*>(dst_);
#pragma unroll
          for (int j = 0; j < p3(K2); ++j) d[base + j * lo + l] = v[j];
        }
      }
    } else {
      // round 1: inner K2 axes, global -> registers -> shared
      #pragma unroll 1
      for (int p = tid; p < p3(K1) * L; p += nt) {
        const int o = p / L, l = p - o * L;
        if (l0 + l >= lo) continue;
        W v[p3(K2)];
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) v[j] = src[base + (long long)(o * p3(K2) + j) * lo + l];
        interp_pencil<M, K2>(v);
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) T[(o * p3(K2) + j) * L + l] = v[j];
      }
      __syncthreads();
      // round 2: outer K1 axes, shared -> registers -> global
      #pragma unroll 1
      for (int p = tid; p < p3(K2) * L; p += nt) {
        const int r = p / L, l = p - r * L;
        if (l0 + l >= lo) continue;
        W v[p3(K1)];
#pragma unroll
        for (int j = 0; j < p3(K1); ++j) v[j] = T[(j * p3(K2) + r) * L + l];
        interp_pencil<M, K1>(v);
        if constexpr (FINAL) {
          Out* d = reinterpret_cast<Out*>(dst_);
#pragma unroll
          for (int j = 0; j < p3(K1); ++j)
            d[base + (long long)(j * p3(K2) + r) * lo + l] = M::out(v[j]);
        } else {
          W* d = reinterpret_cast<W*>(dst_);
#pragma unroll
          for (int j = 0; j < p3(K1); ++j) d[base + (long long)(j * p3(K2) + r) * lo + l] = v[j];
        }
      }
      __syncthreads();  // shared tile reused by the next tile
    }
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
