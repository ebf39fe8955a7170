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
#include <vector>

#include "hc_common.cuh"
#include "hc_profile.cuh"
#include "hc_forward.cuh"
#include "hc_kernels.cuh"
#include "hc_tile.cuh"
#include <type_traits>

namespace hc {

// ---------------------------------------------------------------------------
// K2 kernel: one tile per outer index alpha (grid-stride over tiles).

// pitch: elements between consecutive tiles' outputs (3^C, or more for the
// padded intermediate of HC_SCHED_PADDED).
template <class M, int C, bool FINAL>
__global__ void __launch_bounds__(256) tile_conv_kernel(const typename M::In* __restrict__ X,
                                                        const typename M::In* __restrict__ Y,
                                                        void* __restrict__ out_, long long ntiles,
                                                        long long pitch) {
  typedef typename M::In In;
  typedef typename std::conditional<FINAL, typename M::Out, typename M::W>::type O;
  extern __shared__ __align__(16) unsigned char smem[];
  In* rows = reinterpret_cast<In*>(smem + TileRows<M, C>::kOff);  // [buffer][operand][2^C]
  auto prefetch = [&](long long t, int b) {
#pragma unroll 1
    for (int e = threadIdx.x; e < 2 * p2(C); e += blockDim.x) {
      const int op = e >> C, i = e & (p2(C) - 1);
      cp_async<sizeof(In)>(rows + (b * 2 + op) * p2(C) + i, (op ? Y : X) + t * p2(C) + i);
    }
    cp_async_commit();
  };
  if ((long long)blockIdx.x < ntiles) prefetch(blockIdx.x, 0);
  int it = 0;
#pragma unroll 1
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, it ^= 1) {
    if (t + gridDim.x < ntiles) {
      prefetch(t + gridDim.x, it ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // this tile's rows are in buffer `it`
    RowLoader<In> ld{rows + (it * 2 + 0) * p2(C), rows + (it * 2 + 1) * p2(C)};
    tile_body<M, C, FINAL>(ld, reinterpret_cast<O*>(out_) + t * pitch, smem);
    if constexpr (TileShape<C>::G == 1) __syncthreads();  // buffer reuse (larger tiles end with one)
  }
}

// K2 with bulk stores (tile_loop_bulk): intermediate tiles into a plain
// device allocation.
// T44: the two four-axis groups of C = 8 binary32 tiles (TileStages44,
// 128 threads).
template <class M, int C, bool T44 = false>
__global__ void __launch_bounds__(T44 ? 128 : 256) tile_conv_bulk_kernel(
    const typename M::In* __restrict__ X, const typename M::In* __restrict__ Y,
    typename M::W* __restrict__ out, long long ntiles, long long pitch) {
  typedef typename M::In In;
  extern __shared__ __align__(16) unsigned char smem[];
  auto src = [&](long long t, int op) -> const In* { return (op ? Y : X) + t * p2(C); };
  auto dst = [&](long long t) { return out + t * pitch; };
  if constexpr (T44)
    tile_loop_bulk<M, C, decltype(src), decltype(dst), TileStages44<M>>(src, dst, ntiles, smem);
  else
    tile_loop_bulk<M, C>(src, dst, ntiles, smem);
}

// HC_FP32_FF: the binary32 inputs as float-float pairs (x, 0), written once
// before the first pass (blockIdx.y selects the operand).
__global__ void __launch_bounds__(256) widen_ff_kernel(const float* __restrict__ x,
                                                       const float* __restrict__ y,
                                                       ffv* __restrict__ xw, ffv* __restrict__ yw,
                                                       long long n) {
  const float* s = blockIdx.y ? y : x;
  ffv* d = blockIdx.y ? yw : xw;
#pragma unroll 1
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = ffv{s[i], 0.0f};
}

// D = 0: z[0] = x[0] * y[0].
template <class M>
__global__ void scalar_conv_kernel(const typename M::In* x, const typename M::In* y,
                                   typename M::Out* z) {
  if (threadIdx.x == 0 && blockIdx.x == 0) z[0] = M::out(M::mul(x[0], y[0]));
}

// ---------------------------------------------------------------------------
// Host side.

template <class M>
static int max_tile_axes() {
  return sizeof(typename M::W) == 4 ? 9 : 8;
}

static int threads_for_tile(int C) { return C >= 4 ? 256 : 32; }

template <class M, int C, bool FINAL>
static cudaError_t launch_tile_c(const typename M::In* X, const typename M::In* Y, void* out,
                                 long long ntiles, cudaStream_t st, long long pitch) {
  ProfileScope prof(st, "tile_conv");
  if constexpr (use_bulk_tiles<M, C, FINAL>()) {
    if (is_device_allocation(out)) {
      const size_t smem = TileBulk<M, C>::bytes;
      constexpr bool t44 = use_tile44<M, C>();
      constexpr int threads = t44 ? 128 : 256;
      auto k = tile_conv_bulk_kernel<M, C, t44>;
      cudaError_t e = prep_kernel(k, smem);
      if (e != cudaSuccess) return e;
      k<<<grid_for(k, threads, smem, ntiles), threads, smem, st>>>(X, Y, (typename M::W*)out,
                                                                   ntiles, pitch);
      return cudaGetLastError();
    }
  }
  const size_t smem = TileRows<M, C>::bytes;
  auto k = tile_conv_kernel<M, C, FINAL>;
  cudaError_t e = prep_kernel(k, smem);
  if (e != cudaSuccess) return e;
  const int threads = threads_for_tile(C);
  k<<<grid_for(k, threads, smem, ntiles), threads, smem, st>>>(X, Y, out, ntiles, pitch);
  return cudaGetLastError();
}

template <class M, bool FINAL>
static cudaError_t launch_tile(int C, const typename M::In* X, const typename M::In* Y, void* out,
                               long long ntiles, cudaStream_t st, long long pitch = 0) {
  if (pitch == 0) pitch = (long long)pow3z(C);
  switch (C) {
    case 1: return launch_tile_c<M, 1, FINAL>(X, Y, out, ntiles, st, pitch);
    case 2: return launch_tile_c<M, 2, FINAL>(X, Y, out, ntiles, st, pitch);
    case 3: return launch_tile_c<M, 3, FINAL>(X, Y, out, ntiles, st, pitch);
    case 4: return launch_tile_c<M, 4, FINAL>(X, Y, out, ntiles, st, pitch);
    case 5: return launch_tile_c<M, 5, FINAL>(X, Y, out, ntiles, st, pitch);
    case 6: return launch_tile_c<M, 6, FINAL>(X, Y, out, ntiles, st, pitch);
    case 7: return launch_tile_c<M, 7, FINAL>(X, Y, out, ntiles, st, pitch);
    case 8: return launch_tile_c<M, 8, FINAL>(X, Y, out, ntiles, st, pitch);
    case 9:
      if constexpr (sizeof(typename M::W) == 4) return launch_tile_c<M, 9, FINAL>(X, Y, out, ntiles, st, pitch);
      return cudaErrorInvalidValue;
  }
  return cudaErrorInvalidValue;
}

// The plan: which axes go where, and the workspace layout.
FwdPlan make_fwd_plan(int D, hc_dtype dt, int c_req, int kmax_req, bool padded) {
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
  const size_t in_sz = in_size(dt);
  const size_t w_sz = w_size(dt);
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
  p.padded = padded && p.a > 0;
  if (p.padded) {
    // tile pitch: 3^C rounded up to 128 bytes of intermediate elements
    const long long q = (long long)(128 / w_sz);
    p.pitch = ((long long)pow3z(C) + q - 1) / q * q;
    off = align_up(off + pow3z(p.a) * (size_t)p.pitch * w_sz, 256);
  } else {
    p.pitch = (long long)pow3z(C);
    if (wide_intermediate(dt) && p.a > 0) off = align_up(off + pow3z(D) * w_sz, 256);
  }
  p.ws_bytes = off;
  return p;
}

template <class M>
static cudaError_t run_forward(const FwdPlan& p, const void* x, const void* y, void* z,
                               unsigned char* ws, cudaStream_t st, void* w_user) {
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
  if (p.padded) {
    // the intermediate in the workspace, tile t at t * pitch (every row of
    // every pass 128-byte aligned); the last pass writes z's own layout
    W* Pw = (W*)(ws + p.off_w);
    e = launch_tile<M, false>(C, X, Y, Pw, ntiles, st, p.pitch);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < p.n_interp; ++i) {
      const int d0 = p.interp_d0[i], k = p.interp_k[i];
      const long long hi = (long long)pow3z(d0);
      const long long lo = (long long)pow3z(a - d0 - k) * p.pitch;
      const bool last = (i == p.n_interp - 1);  // d0 = 0: the outermost axes, hi = 1
      const int cols = last && p.cols_outer ? p.cols_outer : p.cols;
      if (last)
        e = launch_interp_remap<M>(k, cols, Pw, (typename M::Out*)z, lo, p.pitch,
                                   (long long)pow3z(C), st);
      else
        e = launch_interp<M, false>(k, cols, Pw, Pw, hi, lo, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const bool mixed_ws = (sizeof(W) != sizeof(typename M::Out)) && a > 0;
  // split: the caller's array holds the intermediate, z only the final stores
  const bool split = !mixed_ws && w_user != nullptr && sizeof(W) == sizeof(typename M::Out);
  W* Wbuf = mixed_ws ? (W*)(ws + p.off_w) : (split ? (W*)w_user : (W*)z);
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
    // the last pass is the one over the outermost axes (hi = 1)
    const int cols = last && p.cols_outer ? p.cols_outer : p.cols;
    if (last && (mixed_ws || split))
      e = launch_interp<M, true>(k, cols, Wbuf, z, hi, lo, st);
    else
      e = launch_interp<M, false>(k, cols, Wbuf, Wbuf, hi, lo, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

ChunkPlan make_chunk_plan(int D, hc_dtype dt, int c_req, int m_req, bool bulk) {
  ChunkPlan p;
  memset(&p, 0, sizeof(p));
  p.D = D;
  p.dtype = dt;
  const int cmax = (dt == HC_FP32) ? 9 : 8;
  int C = c_req > 0 ? (c_req < cmax ? c_req : cmax) : cmax;
  if (C > D) C = D;
  const int mmax = m_req > 0 ? (m_req < 6 ? m_req : 6) : 6;
  p.C = C;
  p.m = (D - C) < mmax ? (D - C) : mmax;
  p.ap = D - C - p.m;
  const size_t es = in_size(dt);  // evaluated-operand elements
  const size_t wsz = w_size(dt);
  // The first m - 3 middle axes are evaluated together with the a' outer
  // axes, leaving at most 3 to evaluate on the fly inside the tiles.
  p.bulk = bulk;
  p.m_pre = bulk ? p.m : (p.m > 3 ? p.m - 3 : 0);
  const int ev = p.ap + p.m_pre;  // axes evaluated by whole-array passes
  // whole-array evaluation passes (<= 3 axes each, outer first)
  for (int d = 0; d < ev; d += 3) {
    const int k = (ev - d) < 3 ? (ev - d) : 3;
    p.eval_d0[p.n_eval] = d;
    p.eval_k[p.n_eval] = k;
    ++p.n_eval;
  }
  size_t xo = ev > 0 ? pow3z(ev) << (D - ev) : 0, tmax = 0;
  for (int i = 0; i < p.n_eval; ++i) {
    const int done = p.eval_d0[i] + p.eval_k[i];
    const bool to_final = ((p.n_eval - 1 - i) % 2) == 0;
    p.eval_to_final[i] = to_final;
    const size_t n = pow3z(done) << (D - done);
    if (!to_final && n > tmax) tmax = n;
  }
  // whole-array interpolation passes over the a' outer axes (<= 6, innermost first)
  if (p.ap > 0) {
    const int np = (p.ap + 5) / 6;
    int end = p.ap;
    for (int i = 0; i < np; ++i) {
      const int rem = np - i;
      const int k = (end + rem - 1) / rem;
      p.interp_d0[i] = end - k;
      p.interp_k[i] = k;
      end -= k;
    }
    p.n_interp = np;
  }
  p.L = kPersistCols;
  p.units = (long long)pow3z(p.ap);
  p.n_tiles = (int)pow3z(p.m);
  if (p.m > 0) {
    const long long coltiles = ((long long)pow3z(C) + p.L - 1) / p.L;
    long long cpt = 32768 / ((long long)pow3z(p.m) * p.L);
    if (cpt < 1) cpt = 1;
    if (bulk && (cpt & 1)) ++cpt;  // the slab kernel's column tiles are 2 * L wide
    p.cpt = (int)cpt;
    p.n_cols = (int)((coltiles + cpt - 1) / cpt);
  } else {
    p.cpt = 1;
    p.n_cols = 0;
  }
  p.per_unit = p.n_tiles + p.n_cols;
  p.total = p.units * p.per_unit;
  size_t smem = tile_smem_bytes(dt, C);
  const size_t ismem = p.m >= 4 ? 2 * wsz * pow3z(p.m) * p.L : 0;  // two column tiles in flight
  p.smem = smem > ismem ? smem : ismem;
  size_t off = kWsHeader;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  p.off_ctr = take(8 * (size_t)(p.units + 1));
  p.off_xo = take(xo * es);
  p.off_yo = take(xo * es);
  p.off_tx = take(tmax * es);
  p.off_ty = take(tmax * es);
  p.off_w = take((wide_intermediate(dt) && (p.m > 0 || p.ap > 0)) ? pow3z(D) * wsz : 0);
  p.ws_bytes = off;
  return p;
}

cudaError_t chunk_dispatch(const ChunkPlan& p, const void* x, const void* y, void* z,
                           unsigned char* ws, cudaStream_t st, void* w) {
  switch (p.dtype) {
    case HC_INT64: return chunk_forward_i64(p, x, y, z, ws, st, w);
    case HC_FP64: return chunk_forward_f64(p, x, y, z, ws, st, w);
    case HC_FP32: return chunk_forward_f32(p, x, y, z, ws, st, w);
    case HC_FP32_MIXED: return chunk_forward_mix(p, x, y, z, ws, st, w);
    case HC_FP32_FF: return chunk_forward_ff(p, x, y, z, ws, st, w);
  }
  return cudaErrorInvalidValue;
}

cudaError_t forward_dispatch(const FwdPlan& p, const void* x, const void* y, void* z,
                             unsigned char* ws, cudaStream_t st, void* w) {
  switch (p.dtype) {
    case HC_INT64: return run_forward<ModeI64>(p, x, y, z, ws, st, w);
    case HC_FP64: return run_forward<ModeF64>(p, x, y, z, ws, st, w);
    case HC_FP32: return run_forward<ModeF32>(p, x, y, z, ws, st, w);
    case HC_FP32_MIXED: return run_forward<ModeMixed>(p, x, y, z, ws, st, w);
    case HC_FP32_FF: return run_forward<ModeFF>(p, x, y, z, ws, st, w);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hc

// ---------------------------------------------------------------------------
// Schedules, the default-schedule table and the C ABI

namespace hc {

static std::mutex g_sched_mu;
constexpr int kNumDtypes = 5;  // HC_INT64 .. HC_FP32_FF
static hc_schedule g_default[HC_MAX_D + 1][kNumDtypes];
static bool g_has_default[HC_MAX_D + 1][kNumDtypes];

bool schedule_valid(const hc_schedule& s, hc_dtype dtype) {
  const int cmax = dtype == HC_FP32 ? 9 : 8;
  if (s.kind < HC_SCHED_DEFAULT || s.kind > HC_SCHED_PADDED) return false;
  if (s.c < 0 || s.c > cmax || s.k < 0 || s.k > 6) return false;
  if (s.kind == HC_SCHED_HYBRID) {
    if (s.top < 1 || s.top > 6 || s.c > 8 || !hybrid_dtype_ok(dtype)) return false;
  } else if (s.kind == HC_SCHED_LOWMEM) {
    if (s.top < 1 || s.top > 6 || !hybrid_dtype_ok(dtype)) return false;
  } else if (s.top != 0) {
    return false;
  }
  auto width_ok = [](int w) {
    return w == 0 || w == 8 || w == 16 || w == 32 || w == -16 || w == -32;
  };
  return width_ok(s.cols) && width_ok(s.cols_outer);
}

hc_schedule resolve_schedule(int D, hc_dtype dtype, const hc_schedule* s) {
  if (s && s->kind != HC_SCHED_DEFAULT) return *s;
  hc_schedule r = {HC_SCHED_CHUNKED, 0, 0, 0, 0, 0};
  if (D >= 0 && D <= HC_MAX_D && dtype >= 0 && dtype < kNumDtypes) {
    std::lock_guard<std::mutex> g(g_sched_mu);
    if (g_has_default[D][dtype]) r = g_default[D][dtype];
  }
  if (s) {  // a DEFAULT schedule may still fix the column widths
    if (s->cols) r.cols = s->cols;
    if (s->cols_outer) r.cols_outer = s->cols_outer;
  }
  return r;
}

static FwdPlan passes_plan(int D, hc_dtype dt, const hc_schedule& s) {
  FwdPlan p = make_fwd_plan(D, dt, s.c, s.k, s.kind == HC_SCHED_PADDED);
  p.cols = s.cols;
  p.cols_outer = s.cols_outer;
  return p;
}

static ChunkPlan chunked_plan(int D, hc_dtype dt, const hc_schedule& s) {
  ChunkPlan p = make_chunk_plan(D, dt, s.c, s.k, s.kind == HC_SCHED_CHUNKED_BULK);
  p.cols = s.cols;
  p.cols_outer = s.cols_outer;
  return p;
}

// HC_FP32_FF: the widened inputs, two arrays of 2^D float-float pairs after
// the plan's own workspace.
static size_t widen_bytes(int D, hc_dtype dtype) {
  return dtype == HC_FP32_FF ? 2 * align_up(sizeof(ffv) << D, 256) : 0;
}

static HybPlan hybrid_plan(int D, hc_dtype dt, const hc_schedule& s) {
  HybPlan p = make_hybrid_plan(D, dt, s.top, s.c, s.k);
  p.cols = s.cols;
  p.cols_outer = s.cols_outer;
  return p;
}

static LowPlan lowmem_plan(int D, hc_dtype dt, const hc_schedule& s) {
  return make_lowmem_plan(D, dt, s.top, s.c, s.k, s.cols, s.cols_outer);
}

static size_t plan_ws(int D, hc_dtype dtype, const hc_schedule& s) {
  if (s.kind == HC_SCHED_PASSES || s.kind == HC_SCHED_PADDED || D == 0)
    return passes_plan(D, dtype, s).ws_bytes;
  if (s.kind == HC_SCHED_LOWMEM) {
    const LowPlan l = lowmem_plan(D, dtype, s);
    return l.ok ? l.ws_bytes : 0;
  }
  if (s.kind == HC_SCHED_HYBRID) {
    const HybPlan h = hybrid_plan(D, dtype, s);
    return h.ok ? h.ws_bytes : 0;
  }
  return chunked_plan(D, dtype, s).ws_bytes;
}

size_t schedule_ws(int D, hc_dtype dtype, const hc_schedule& s) {
  if (D < 0 || D > HC_MAX_D || elem_size(dtype) == 0) return 0;
  return plan_ws(D, dtype, s) + widen_bytes(D, dtype);
}

hc_status convolve_checked(const void* x, const void* y, void* z, int D, hc_dtype dtype,
                           void* workspace, size_t ws_bytes, cudaStream_t stream,
                           const hc_schedule* sched, void* w) {
  if (D < 0 || D > HC_MAX_D) return HC_ERR_ARG;
  const size_t es = elem_size(dtype);
  if (es == 0) return HC_ERR_DTYPE;
  if (sched && !schedule_valid(*sched, dtype)) return HC_ERR_ARG;
  if (!x || !y || !z) return HC_ERR_ARG;
  if (!aligned(x, 16) || !aligned(y, 16) || !aligned(z, 16)) return HC_ERR_ALIGN;
  const hc_schedule s = resolve_schedule(D, dtype, sched);
  if (s.kind == HC_SCHED_HYBRID && D > 0 && !hybrid_plan(D, dtype, s).ok)
    return HC_ERR_ARG;  // fewer than 4 tile axes below the direct ones
  if (s.kind == HC_SCHED_LOWMEM && D > 0 && !lowmem_plan(D, dtype, s).ok)
    return HC_ERR_ARG;  // no axis left below the top ones
  const size_t need = schedule_ws(D, dtype, s);
  if (ws_bytes < need) return HC_ERR_WORKSPACE;
  if (need > 0 && !workspace) return HC_ERR_ARG;
  if (workspace && !aligned(workspace, 256)) return HC_ERR_ALIGN;
  const size_t nx = es << D, nz = es * pow3z(D);
  if (overlaps(z, nz, x, nx) || overlaps(z, nz, y, nx)) return HC_ERR_ALIAS;
  if (workspace && need > 0 &&
      (overlaps(workspace, need, z, nz) || overlaps(workspace, need, x, nx) ||
       overlaps(workspace, need, y, nx)))
    return HC_ERR_ALIAS;
  if (w) {
    if (!aligned(w, 16)) return HC_ERR_ALIGN;
    if (overlaps(w, nz, z, nz) || overlaps(w, nz, x, nx) || overlaps(w, nz, y, nx) ||
        (workspace && need > 0 && overlaps(w, nz, workspace, need)))
      return HC_ERR_ALIAS;
  }
  if (dtype == HC_FP32_FF) {
    // widen x, y into the workspace's tail; the passes then read pairs
    unsigned char* tail = (unsigned char*)workspace + plan_ws(D, dtype, s);
    ffv* xw = (ffv*)tail;
    ffv* yw = (ffv*)(tail + align_up(sizeof(ffv) << D, 256));
    const long long n = 1ll << D;
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)device_caps().sms * 8;
    if (blocks > cap) blocks = cap;
    {
      ProfileScope prof(stream, "widen");
      widen_ff_kernel<<<dim3((unsigned)blocks, 2), 256, 0, stream>>>((const float*)x,
                                                                    (const float*)y, xw, yw, n);
    }
    const hc_status wst = record_cuda_error(cudaGetLastError());
    if (wst != HC_OK) return wst;
    x = xw;
    y = yw;
  }
  if (s.kind == HC_SCHED_PASSES || s.kind == HC_SCHED_PADDED || D == 0)
    return record_cuda_error(forward_dispatch(passes_plan(D, dtype, s), x, y, z,
                                              (unsigned char*)workspace, stream, w));
  if (s.kind == HC_SCHED_HYBRID)
    return record_cuda_error(hybrid_dispatch(hybrid_plan(D, dtype, s), x, y, z,
                                             (unsigned char*)workspace, stream, w));
  if (s.kind == HC_SCHED_LOWMEM)
    return record_cuda_error(lowmem_dispatch(lowmem_plan(D, dtype, s), x, y, z,
                                             (unsigned char*)workspace, stream, w));
  return record_cuda_error(chunk_dispatch(chunked_plan(D, dtype, s), x, y, z,
                                          (unsigned char*)workspace, stream, w));
}

// Candidate schedules of the autotuner for (D, dtype).
static std::vector<hc_schedule> tune_candidates(int D, hc_dtype dtype) {
  std::vector<hc_schedule> v;
  const int cmax = dtype == HC_FP32 ? 9 : 8;
  if (D <= cmax) {
    v.push_back({HC_SCHED_CHUNKED, 0, 0, 0, 0});
    return v;
  }
  const int cols[5] = {8, 16, 32, -16, -32};
  for (int c = cmax - 1; c <= cmax; ++c) {
    for (int k = 3; k <= 6; ++k)
      for (int ci = 0; ci < 5; ++ci) {
        v.push_back({HC_SCHED_PASSES, c, k, cols[ci], 0});
        v.push_back({HC_SCHED_CHUNKED, c, k, cols[ci], 0});
        v.push_back({HC_SCHED_CHUNKED_BULK, c, k, cols[ci], 0});
      }
  }
  // the hybrid form (2..4 direct top axes, 8-axis tiles, the middle axes in
  // passes of 5 or 6) only where it gives the same bits as the recurrence:
  // int64.  A default schedule never changes a floating-point result's
  // rounding; the hybrid form stays available by explicit request.
  if (dtype == HC_INT64) {
    for (int top = 2; top <= 4; ++top)
      for (int k = 5; k <= 6; ++k)
        for (int w : {32, -32}) {
          const hc_schedule h = {HC_SCHED_HYBRID, 8, k, w, 0, top};
          if (D - top >= 4) v.push_back(h);
        }
  }
  return v;
}

}  // namespace hc

extern "C" size_t hc_workspace_size(int D, hc_dtype dtype) {
  return hc::schedule_ws(D, dtype, hc::resolve_schedule(D, dtype, nullptr));
}

extern "C" size_t hc_workspace_size_schedule(int D, hc_dtype dtype, const hc_schedule* s) {
  if (s && !hc::schedule_valid(*s, dtype)) return 0;
  return hc::schedule_ws(D, dtype, hc::resolve_schedule(D, dtype, s));
}

extern "C" hc_status hc_convolve(const void* x, const void* y, void* z, int D, hc_dtype dtype,
                                 void* workspace, size_t ws_bytes, hc_stream_t stream) {
  return hc::convolve_checked(x, y, z, D, dtype, workspace, ws_bytes, (cudaStream_t)stream,
                              nullptr);
}

extern "C" hc_status hc_convolve_schedule(const void* x, const void* y, void* z, int D,
                                          hc_dtype dtype, const hc_schedule* s, void* workspace,
                                          size_t ws_bytes, hc_stream_t stream) {
  if (!s) return HC_ERR_ARG;
  return hc::convolve_checked(x, y, z, D, dtype, workspace, ws_bytes, (cudaStream_t)stream, s);
}

extern "C" hc_status hc_convolve_out(const void* x, const void* y, void* w, void* z, int D,
                                     hc_dtype dtype, void* workspace, size_t ws_bytes,
                                     hc_stream_t stream) {
  if (hc::wide_intermediate(dtype)) {
    if (w) return HC_ERR_ARG;  // its intermediate lives in the workspace
  } else if (!w) {
    return HC_ERR_ARG;
  }
  // The kernels store to z and w at these addresses: z must be device,
  // managed or page-locked host memory mapped at the same address, w device
  // or managed memory.  Checked on the host, before any launch.
  if (!x || !y || !z) return HC_ERR_ARG;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, z) != cudaSuccess) {
    cudaGetLastError();
    return HC_ERR_ARG;
  }
  if (a.type == cudaMemoryTypeUnregistered ||
      (a.type == cudaMemoryTypeHost && a.devicePointer != z))
    return HC_ERR_ARG;
  if (w) {
    if (cudaPointerGetAttributes(&a, w) != cudaSuccess) {
      cudaGetLastError();
      return HC_ERR_ARG;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return HC_ERR_ARG;
  }
  return hc::convolve_checked(x, y, z, D, dtype, workspace, ws_bytes, (cudaStream_t)stream,
                              nullptr, w);
}

extern "C" hc_status hc_set_default_schedule(int D, hc_dtype dtype, const hc_schedule* s) {
  if (D < 0 || D > HC_MAX_D || hc::elem_size(dtype) == 0) return HC_ERR_ARG;
  if (s && (!hc::schedule_valid(*s, dtype) || s->kind == HC_SCHED_DEFAULT)) return HC_ERR_ARG;
  // a default keeps the recurrence's bits: no hybrid form for floating point
  if (s && s->kind == HC_SCHED_HYBRID && dtype != HC_INT64) return HC_ERR_ARG;
  std::lock_guard<std::mutex> g(hc::g_sched_mu);
  hc::g_has_default[D][dtype] = s != nullptr;
  if (s) hc::g_default[D][dtype] = *s;
  return HC_OK;
}

extern "C" hc_status hc_get_default_schedule(int D, hc_dtype dtype, hc_schedule* s) {
  if (D < 0 || D > HC_MAX_D || hc::elem_size(dtype) == 0 || !s) return HC_ERR_ARG;
  *s = hc::resolve_schedule(D, dtype, nullptr);
  return HC_OK;
}

extern "C" size_t hc_autotune_workspace_size(int D, hc_dtype dtype) {
  if (D < 0 || D > HC_MAX_D || hc::elem_size(dtype) == 0) return 0;
  size_t m = hc::schedule_ws(D, dtype, hc::resolve_schedule(D, dtype, nullptr));
  for (const hc_schedule& s : hc::tune_candidates(D, dtype)) {
    const size_t w = hc::schedule_ws(D, dtype, s);
    if (w > m) m = w;
  }
  return m;
}

extern "C" hc_status hc_autotune(const void* x, const void* y, void* z, int D, hc_dtype dtype,
                                 void* workspace, size_t ws_bytes, int reps, hc_stream_t stream,
                                 hc_schedule* best, double* best_ms) {
  using namespace hc;
  if (D < 0 || D > HC_MAX_D || elem_size(dtype) == 0 || reps < 1) return HC_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) return record_cuda_error(ce);
  hc_schedule win = {HC_SCHED_CHUNKED, 0, 0, 0, 0};
  double win_ms = -1.0;
  hc_status status = HC_OK;
  for (const hc_schedule& s : tune_candidates(D, dtype)) {
    if (schedule_ws(D, dtype, s) > ws_bytes) continue;
    status = convolve_checked(x, y, z, D, dtype, workspace, ws_bytes, st, &s);  // warm-up
    if (status != HC_OK) break;
    double t_min = -1.0;
    for (int r = 0; r < reps && status == HC_OK; ++r) {
      cudaEventRecord(e0, st);
      status = convolve_checked(x, y, z, D, dtype, workspace, ws_bytes, st, &s);
      cudaEventRecord(e1, st);
      ce = cudaEventSynchronize(e1);
      if (ce != cudaSuccess) {
        status = record_cuda_error(ce);
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (t_min < 0.0 || ms < t_min) t_min = ms;
    }
    if (status != HC_OK) break;
    if (win_ms < 0.0 || t_min < win_ms) {
      win_ms = t_min;
      win = s;
    }
  }
  // second stage: the winner's (kind, c, k) with every pair of widths for the
  // inner passes and the pass over the outermost axes (meaningful when its
  // plan has two or more whole-array passes)
  if (status == HC_OK && win_ms >= 0.0 && win.kind == HC_SCHED_PASSES &&
      passes_plan(D, dtype, win).n_interp >= 2) {
    const int widths[5] = {8, 16, 32, -16, -32};
    const hc_schedule base = win;
    for (int wi = 0; wi < 25 && status == HC_OK; ++wi) {
      hc_schedule s = base;
      s.cols = widths[wi / 5];
      s.cols_outer = widths[wi % 5];
      if (s.cols == s.cols_outer) continue;  // a single width was timed already
      status = convolve_checked(x, y, z, D, dtype, workspace, ws_bytes, st, &s);  // warm-up
      double t_min = -1.0;
      for (int r = 0; r < reps && status == HC_OK; ++r) {
        cudaEventRecord(e0, st);
        status = convolve_checked(x, y, z, D, dtype, workspace, ws_bytes, st, &s);
        cudaEventRecord(e1, st);
        ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) {
          status = record_cuda_error(ce);
          break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (t_min < 0.0 || ms < t_min) t_min = ms;
      }
      if (status == HC_OK && t_min >= 0.0 && t_min < win_ms) {
        win_ms = t_min;
        win = s;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != HC_OK) return status;
  if (win_ms < 0.0) return HC_ERR_WORKSPACE;  // no candidate fitted the workspace
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms;
  return HC_OK;
}
