// The hybrid schedule: the 4-way direct form on the top `mt` axes, the
// Karatsuba form on the others (Methods: the direct form z[1] = x[0]*y[1] +
// x[1]*y[0] needs no interpolation on its axis, at the price of four
// sub-products instead of three).  For every top digit string a:
//   P_a = sum over the sub-cube pairs (b, c) with b + c = a of
//         (E^{(x)n} x_b) (.) (E^{(x)n} y_c),      z_a = I^{(x)n} P_a,
// n = D - mt.  The top axes therefore need no whole-array interpolation pass:
// trading (4/3)^mt times the evaluation and product work for fewer passes
// over the 3^D array.  Schedule, with a = D - mt - C middle axes:
//   eval_pass   : the a middle axes of each of the 2^mt top sub-cubes
//                 (<= 3 per pass): [2^mt][2^a][2^C] -> [2^mt][3^a][2^C]
//   hybrid_tile : per (a_top, a_mid), the pairs' C-axis tiles evaluated and
//                 multiplied, their products summed in registers in the
//                 pairs' order, then the C inner axes interpolated
//   interp_pass : the a middle axes, <= k per pass, innermost pass first
// Per element this is the order of the oracle's hybrid form (evaluation
// outermost axis first, pairs in increasing x index, interpolation innermost
// axis first), so results are bitwise those of that form in every dtype.
#include <cstring>

#include "hc_common.cuh"
#include "hc_forward.cuh"
#include "hc_kernels.cuh"
#include "hc_profile.cuh"
#include "hc_tile.cuh"

namespace hc {

constexpr int kHybMaxTop = 6;

// Rows of pair s of tile t: the x and y sub-cubes of the top bit strings
// (b, c) with b + c = the tile's top digits, at the tile's middle index.
// Digit 0 gives bits (0, 0), 2 gives (1, 1); for the digit-1 axes, taken
// outermost first, bit (m1 - 1 - q) of s set gives x the 1.
struct HybRows {
  long long p3a;  // 3^a
  int mt, C;
  __device__ __forceinline__ int npairs(long long t) const {
    long long at = t / p3a;
    int n = 0;
    for (int d = 0; d < mt; ++d) {
      if (at % 3 == 1) ++n;
      at /= 3;
    }
    return 1 << n;
  }
  __device__ __forceinline__ void rows(long long t, int s, long long& rx, long long& ry) const {
    long long at = t / p3a;
    const long long am = t - at * p3a;
    int dig[kHybMaxTop];
    for (int d = mt - 1; d >= 0; --d) {
      dig[d] = (int)(at % 3);
      at /= 3;
    }
    int m1 = 0;
    for (int d = 0; d < mt; ++d) m1 += dig[d] == 1;
    long long bx = 0, by = 0;
    int q = 0;
    for (int d = 0; d < mt; ++d) {
      const long long bit = 1ll << (mt - 1 - d);
      if (dig[d] == 2) {
        bx |= bit;
        by |= bit;
      } else if (dig[d] == 1) {
        if ((s >> (m1 - 1 - q)) & 1) bx |= bit; else by |= bit;
        ++q;
      }
    }
    rx = (bx * p3a + am) << C;
    ry = (by * p3a + am) << C;
  }
};

// One tile per (a_top, a_mid) (grid-stride).  Requires C >= 4 and at most one
// fused pencil per thread (the stage buffers inside the W tile), which holds
// for C <= 8.  The pairs' rows are double-buffered with cp.async: the next
// pair's (or the next tile's first pair's) rows load while this pair runs.
template <class M, int C, bool FINAL>
__global__ void __launch_bounds__(256) hybrid_tile_kernel(const typename M::In* __restrict__ X,
                                                          const typename M::In* __restrict__ Y,
                                                          void* __restrict__ out_, HybRows hr,
                                                          long long ntiles) {
  typedef typename M::In In;
  typedef typename M::W W;
  typedef TileShape<C> S;
  typedef TileStages<M, C> St;
  static_assert(S::G >= 2 && TileSmem<M, C>::kAlias, "hybrid tiles: C >= 4, one pencil per thread");
  typedef typename std::conditional<FINAL, typename M::Out, W>::type O;
  extern __shared__ __align__(16) unsigned char smem[];
  In* rowbuf = reinterpret_cast<In*>(smem + TileRows<M, C>::kOff);  // [buffer][operand][2^C]
  const int tid = threadIdx.x, nt = blockDim.x;
  auto prefetch = [&](long long t, int s, int b) {
    long long rx, ry;
    hr.rows(t, s, rx, ry);
#pragma unroll 1
    for (int e = tid; e < 2 * p2(C); e += nt) {
      const int op = e >> C, i = e & (p2(C) - 1);
      cp_async<sizeof(In)>(rowbuf + (b * 2 + op) * p2(C) + i, (op ? Y + ry : X + rx) + i);
    }
    cp_async_commit();
  };
  constexpr int NO = S::nLastPencils;
  const int LP = TileSmem<M, C>::LP;
  int b = 0;
  long long t = blockIdx.x;
  if (t < ntiles) prefetch(t, 0, 0);
#pragma unroll 1
  for (; t < ntiles; t += gridDim.x) {
    const int np = hr.npairs(t);
    W acc[27];
#pragma unroll 1
    for (int s = 0; s < np; ++s, b ^= 1) {
      cp_async_wait<0>();
      __syncthreads();  // pair s's rows are in buffer b; the last pair's reads are done
      if (s + 1 < np)
        prefetch(t, s + 1, b ^ 1);
      else if (t + gridDim.x < ntiles)
        prefetch(t + gridDim.x, 0, b ^ 1);
      RowLoader<In> ld{rowbuf + (b * 2) * p2(C), rowbuf + (b * 2 + 1) * p2(C)};
#pragma unroll 1
      for (int p = tid; p < St::kStage0; p += nt) St::stage0(ld, smem, p);
      __syncthreads();
      if constexpr (S::G == 3) {
        St::stage1(smem);
        __syncthreads();
      }
      // evaluate the innermost group of both operands, multiply, add into
      // this thread's accumulator pencil (pairs in order)
      if (tid < NO) {
        const In* LastX = St::last_x(smem);
        const In* LastY = LastX + p2(S::gL) * LP;
        In xa[27], ya[27];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          xa[q] = LastX[q * LP + tid];
          ya[q] = LastY[q * LP + tid];
        }
        eval_pencil<M, 3>(xa);
        eval_pencil<M, 3>(ya);
#pragma unroll
        for (int j = 0; j < 27; ++j) {
          const W pj = M::mul(xa[j], ya[j]);
          acc[j] = s == 0 ? pj : M::wadd(acc[j], pj);
        }
      }
    }
    __syncthreads();  // every read of the stage buffers (inside the W tile) is done
    W* Ws = reinterpret_cast<W*>(smem);
    if (tid < NO) {
      interp_pencil<M, 3>(acc);
#pragma unroll
      for (int j = 0; j < 27; ++j) Ws[tid * 27 + j] = acc[j];
    }
    __syncthreads();
    if constexpr (S::G == 3) {
      St::interp1(smem);
      __syncthreads();
    }
    O* out_tile = reinterpret_cast<O*>(out_) + t * p3(C);
#pragma unroll 1
    for (int r = tid; r < St::kInterp0; r += nt) St::template interp0<FINAL, false>(out_tile, smem, r);
    // the next tile's first barrier orders these reads before its writes
  }
}


// Plan: mt top axes (1..6), C tile axes (4..8, clamped to D - mt; 0 = 8),
// a = D - mt - C middle axes through passes of <= kmax axes (0 = 6).  ok is
// false when D - mt < 4 or mt is out of range.
HybPlan make_hybrid_plan(int D, hc_dtype dt, int mt, int c_req, int kmax_req) {
  HybPlan p;
  memset(&p, 0, sizeof(p));
  p.D = D;
  p.dtype = dt;
  p.mt = mt;
  int C = c_req > 0 ? (c_req < 8 ? c_req : 8) : 8;
  if (C > D - mt) C = D - mt;
  p.C = C;
  p.a = D - mt - C;
  p.ok = mt >= 1 && mt <= kHybMaxTop && C >= 4;
  if (!p.ok) return p;
  int kmax = kmax_req > 0 ? (kmax_req < 6 ? kmax_req : 6) : 6;
  const size_t in_sz = in_size(dt);
  for (int d = 0; d < p.a; d += 3) {
    const int k = (p.a - d) < 3 ? (p.a - d) : 3;
    p.eval_d0[p.n_eval] = d;
    p.eval_k[p.n_eval] = k;
    ++p.n_eval;
  }
  const size_t top = (size_t)1 << mt;
  const size_t xo = p.a > 0 ? (top * pow3z(p.a)) << C : 0;
  size_t tmax = 0;
  for (int i = 0; i < p.n_eval; ++i) {
    const int done = p.eval_d0[i] + p.eval_k[i];
    const bool to_final = ((p.n_eval - 1 - i) % 2) == 0;
    p.eval_to_final[i] = to_final;
    const size_t n = (top * pow3z(done)) << (D - mt - done);
    if (!to_final && n > tmax) tmax = n;
  }
  if (p.a > 0) {
    const int np = (p.a + kmax - 1) / kmax;
    int end = p.a;
    for (int i = 0; i < np; ++i) {
      const int rem = np - i;
      const int k = (end + rem - 1) / rem;
      p.interp_d0[i] = end - k;
      p.interp_k[i] = k;
      end -= k;
    }
    p.n_interp = np;
  }
  size_t off = kWsHeader;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  p.off_xo = take(xo * in_sz);
  p.off_yo = take(xo * in_sz);
  p.off_tx = take(tmax * in_sz);
  p.off_ty = take(tmax * in_sz);
  p.ws_bytes = off;
  return p;
}

template <class M, int C, bool FINAL>
static cudaError_t launch_hybrid_tile_c(const typename M::In* X, const typename M::In* Y,
                                        void* out, const HybRows& hr, long long ntiles,
                                        cudaStream_t st) {
  ProfileScope prof(st, "hybrid_tile");
  const size_t smem = TileRows<M, C>::bytes;
  auto k = hybrid_tile_kernel<M, C, FINAL>;
  cudaError_t e = prep_kernel(k, smem);
  if (e != cudaSuccess) return e;
  k<<<grid_for(k, 256, smem, ntiles), 256, smem, st>>>(X, Y, out, hr, ntiles);
  return cudaGetLastError();
}

template <class M, bool FINAL>
static cudaError_t launch_hybrid_tile(int C, const typename M::In* X, const typename M::In* Y,
                                      void* out, const HybRows& hr, long long ntiles,
                                      cudaStream_t st) {
  switch (C) {
    case 4: return launch_hybrid_tile_c<M, 4, FINAL>(X, Y, out, hr, ntiles, st);
    case 5: return launch_hybrid_tile_c<M, 5, FINAL>(X, Y, out, hr, ntiles, st);
    case 6: return launch_hybrid_tile_c<M, 6, FINAL>(X, Y, out, hr, ntiles, st);
    case 7: return launch_hybrid_tile_c<M, 7, FINAL>(X, Y, out, hr, ntiles, st);
    case 8: return launch_hybrid_tile_c<M, 8, FINAL>(X, Y, out, hr, ntiles, st);
  }
  return cudaErrorInvalidValue;
}

// w: the caller's array for the intermediate (hc_convolve_out), z then
// written only by the final stores; nullptr: the intermediate lives in z.
template <class M>
static cudaError_t run_hybrid(const HybPlan& p, const void* x, const void* y, void* z,
                              unsigned char* ws, cudaStream_t st, void* w) {
  typedef typename M::In In;
  typedef typename M::W W;
  W* Wbuf = w ? (W*)w : (W*)z;
  const int D = p.D, C = p.C, a = p.a, mt = p.mt;
  const In* X = (const In*)x;
  const In* Y = (const In*)y;
  cudaError_t e;
  for (int i = 0; i < p.n_eval; ++i) {
    const int d0 = p.eval_d0[i], k = p.eval_k[i];
    const long long hi = ((long long)1 << mt) * (long long)pow3z(d0);
    const long long lo = (long long)1 << (D - mt - d0 - k);
    In* dx = (In*)(ws + (p.eval_to_final[i] ? p.off_xo : p.off_tx));
    In* dy = (In*)(ws + (p.eval_to_final[i] ? p.off_yo : p.off_ty));
    e = launch_eval<M>(k, X, Y, dx, dy, hi, lo, st);
    if (e != cudaSuccess) return e;
    X = dx;
    Y = dy;
  }
  HybRows hr;
  hr.p3a = (long long)pow3z(a);
  hr.mt = mt;
  hr.C = C;
  const long long ntiles = (long long)pow3z(mt) * hr.p3a;
  e = a == 0 ? launch_hybrid_tile<M, true>(C, X, Y, z, hr, ntiles, st)
             : launch_hybrid_tile<M, false>(C, X, Y, Wbuf, hr, ntiles, st);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < p.n_interp; ++i) {
    const int d0 = p.interp_d0[i], k = p.interp_k[i];
    const long long hi = (long long)pow3z(mt) * (long long)pow3z(d0);
    const long long lo = (long long)pow3z(a - d0 - k) * (long long)pow3z(C);
    const bool last = i == p.n_interp - 1;
    const int cols = last && p.cols_outer ? p.cols_outer : p.cols;
    if (last && w)
      e = launch_interp<M, true>(k, cols, Wbuf, z, hi, lo, st);
    else
      e = launch_interp<M, false>(k, cols, Wbuf, Wbuf, hi, lo, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

bool hybrid_dtype_ok(hc_dtype dt) { return dt == HC_INT64 || dt == HC_FP64 || dt == HC_FP32; }

cudaError_t hybrid_dispatch(const HybPlan& p, const void* x, const void* y, void* z,
                            unsigned char* ws, cudaStream_t st, void* w) {
  switch (p.dtype) {
    case HC_INT64: return run_hybrid<ModeI64>(p, x, y, z, ws, st, w);
    case HC_FP64: return run_hybrid<ModeF64>(p, x, y, z, ws, st, w);
    case HC_FP32: return run_hybrid<ModeF32>(p, x, y, z, ws, st, w);
    default: break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace hc
