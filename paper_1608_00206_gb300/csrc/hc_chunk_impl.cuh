// The chunked forward schedule for one arithmetic mode (included by one
// translation unit per mode).
#pragma once

#include "hc_common.cuh"
#include "hc_forward.cuh"
#include "hc_kernels.cuh"
#include "hc_persist.cuh"
#include "hc_profile.cuh"
#include "hc_slab.cuh"
#include "hc_tile.cuh"

namespace hc {

template <class M, int C, bool FIN>
__global__ void __launch_bounds__(256, (sizeof(typename M::W) == 4 ? 3 : 2)) chunk_kernel(UniformUnits uu, long long total,
                                                    unsigned long long* counters, WsHeader* hdr) {
  extern __shared__ __align__(16) unsigned char smem[];
  // L2 priorities: tiles kept for their unit's columns, finished columns
  // streamed out (2% on GB300 against plain accesses, same bits)
  persistent_loop<M, C, true, FIN, true>(nullptr, nullptr, uu, total, counters, hdr, smem);
}

template <class M, int C, bool FIN>
static cudaError_t launch_chunk_c(const ChunkPlan& p, const UniformUnits& uu,
                                  unsigned long long* ctr, WsHeader* hdr, cudaStream_t st) {
  auto k = chunk_kernel<M, C, FIN>;
  ProfileScope prof(st, "chunk");
  cudaError_t e = prep_kernel(k, p.smem);
  if (e != cudaSuccess) return e;
  const int grid = grid_for(k, 256, p.smem, p.total);
  UniformUnits u2 = uu;
  u2.lag = grid < p.n_tiles ? grid : p.n_tiles;  // one wave of CTAs (see uniform_ticket)
  k<<<grid, 256, p.smem, st>>>(u2, p.total, ctr, hdr);
  return cudaGetLastError();
}

template <class M, bool FIN>
static cudaError_t launch_chunk(const ChunkPlan& p, const UniformUnits& uu,
                                unsigned long long* ctr, WsHeader* hdr, cudaStream_t st) {
  switch (p.C) {
    case 1: return launch_chunk_c<M, 1, FIN>(p, uu, ctr, hdr, st);
    case 2: return launch_chunk_c<M, 2, FIN>(p, uu, ctr, hdr, st);
    case 3: return launch_chunk_c<M, 3, FIN>(p, uu, ctr, hdr, st);
    case 4: return launch_chunk_c<M, 4, FIN>(p, uu, ctr, hdr, st);
    case 5: return launch_chunk_c<M, 5, FIN>(p, uu, ctr, hdr, st);
    case 6: return launch_chunk_c<M, 6, FIN>(p, uu, ctr, hdr, st);
    case 7: return launch_chunk_c<M, 7, FIN>(p, uu, ctr, hdr, st);
    case 8: return launch_chunk_c<M, 8, FIN>(p, uu, ctr, hdr, st);
    case 9:
      if constexpr (sizeof(typename M::W) == 4) return launch_chunk_c<M, 9, FIN>(p, uu, ctr, hdr, st);
      return cudaErrorInvalidValue;
  }
  return cudaErrorInvalidValue;
}

// The slab kernel of the chunked-bulk schedule, for a compile-time tile C and
// m middle axes.
template <class M, int C, int MM, bool FIN>
static cudaError_t launch_slab_cm(const ChunkPlan& p, const SlabArgs& a0, cudaStream_t st) {
  auto k = slab_kernel<M, C, MM, FIN>;
  ProfileScope prof(st, "slab");
  const size_t smem = SlabSmem<M, C, MM>::bytes;
  cudaError_t e = prep_kernel(k, smem);
  if (e != cudaSuccess) return e;
  const int grid = grid_for(k, 256, smem, p.total);
  SlabArgs a = a0;
  a.uu.lag = grid < p.n_tiles ? grid : p.n_tiles;  // one wave of CTAs (see uniform_ticket)
  k<<<grid, 256, smem, st>>>(a);
  return cudaGetLastError();
}

template <class M, int C, bool FIN>
static cudaError_t launch_slab_c(const ChunkPlan& p, const SlabArgs& a, cudaStream_t st) {
  switch (p.m) {
    case 1: return launch_slab_cm<M, C, 1, FIN>(p, a, st);
    case 2: return launch_slab_cm<M, C, 2, FIN>(p, a, st);
    case 3: return launch_slab_cm<M, C, 3, FIN>(p, a, st);
    case 4: return launch_slab_cm<M, C, 4, FIN>(p, a, st);
    case 5: return launch_slab_cm<M, C, 5, FIN>(p, a, st);
    case 6: return launch_slab_cm<M, C, 6, FIN>(p, a, st);
  }
  return cudaErrorInvalidValue;
}

// Tile sizes the slab kernel is built for: C = 7 and 8, whose two W tiles
// and rows fit one CTA's shared memory for every dtype (a 9-axis float32
// tile does not: the chunked-bulk plan then runs on the generic engine).
template <class M>
static bool slab_supported(int C, int m) {
  return m >= 1 && m <= 6 && (C == 7 || C == 8);
}

template <class M, bool FIN>
static cudaError_t launch_slab(const ChunkPlan& p, const SlabArgs& a, cudaStream_t st) {
  static_assert(SlabSmem<M, 8, 6>::bytes <= 227 * 1024, "slab tiles fit one CTA");
  if (p.C == 8) return launch_slab_c<M, 8, FIN>(p, a, st);
  if (p.C == 7) return launch_slab_c<M, 7, FIN>(p, a, st);
  return cudaErrorInvalidValue;
}

template <class M>
static cudaError_t chunk_forward_m(const ChunkPlan& p, const void* x, const void* y, void* z,
                                   unsigned char* ws, cudaStream_t st, void* w_user) {
  typedef typename M::In In;
  typedef typename M::W W;
  constexpr bool kMixed = !std::is_same<typename M::W, typename M::Out>::value;
  const int D = p.D;
  cudaError_t e;
  // whole-array evaluation of the a' outer axes
  const In* X = (const In*)x;
  const In* Y = (const In*)y;
  for (int i = 0; i < p.n_eval; ++i) {
    const int d0 = p.eval_d0[i], k = p.eval_k[i];
    In* ox = (In*)(ws + (p.eval_to_final[i] ? p.off_xo : p.off_tx));
    In* oy = (In*)(ws + (p.eval_to_final[i] ? p.off_yo : p.off_ty));
    e = launch_eval<M>(k, X, Y, ox, oy, (long long)pow3z(d0), (long long)1 << (D - d0 - k), st);
    if (e != cudaSuccess) return e;
    X = ox;
    Y = oy;
  }
  // status word and counters start at zero
  e = cudaMemsetAsync(ws, 0, p.off_ctr + 8 * (size_t)(p.units + 1), st);
  if (e != cudaSuccess) return e;
  const bool w_in_ws = kMixed && (p.m > 0 || p.ap > 0);
  // split: the caller's array holds the intermediate and z only receives the
  // final stores
  const bool split = !kMixed && w_user != nullptr;
  W* wbuf = w_in_ws ? (W*)(ws + p.off_w) : (split ? (W*)w_user : (W*)z);
  const bool fin = (kMixed || split) && p.ap == 0;  // the columns finish the result
  UniformUnits uu;
  uu.x = X;
  uu.y = Y;
  uu.w = wbuf;
  uu.z = (fin || p.m == 0) ? z : (void*)wbuf;
  uu.in_stride = (long long)pow3z(p.m_pre) << (p.C + p.m - p.m_pre);
  uu.m_pre = p.m_pre;
  uu.units = (int)p.units;
  uu.out_stride = (long long)pow3z(p.C + p.m);
  uu.per_unit = p.per_unit;
  uu.C = p.C;
  uu.m = p.m;
  uu.n_tiles = p.n_tiles;
  uu.n_cols = p.n_cols;
  uu.cpt = p.cpt;
  uu.need = p.n_tiles;
  unsigned long long* ctr = (unsigned long long*)(ws + p.off_ctr);
  // The chunked-bulk schedule (every middle axis evaluated above) runs the
  // slab kernel where its bulk tile copies apply: a tile size it is built
  // for and an intermediate in a plain device allocation.  Otherwise the
  // generic engine runs the same plan (its on-the-fly evaluation then has no
  // axis left to evaluate), with the same bits.
  if (p.bulk && p.m_pre == p.m && slab_supported<M>(p.C, p.m) && is_device_allocation(wbuf)) {
    SlabArgs a;
    a.x = X;
    a.y = Y;
    a.w = wbuf;
    a.z = fin ? z : (void*)wbuf;
    a.ctr = ctr;
    a.hdr = (WsHeader*)ws;
    a.uu = uu;
    a.total = p.total;
    e = fin ? launch_slab<M, true>(p, a, st) : launch_slab<M, false>(p, a, st);
  } else if (fin) {
    e = launch_chunk<M, true>(p, uu, ctr, (WsHeader*)ws, st);
  } else {
    e = launch_chunk<M, false>(p, uu, ctr, (WsHeader*)ws, st);
  }
  if (e != cudaSuccess) return e;
  // whole-array interpolation of the a' outer axes, innermost pass first
  for (int i = 0; i < p.n_interp; ++i) {
    const int d0 = p.interp_d0[i], k = p.interp_k[i];
    const long long hi = (long long)pow3z(d0);
    const long long lo = (long long)pow3z(p.ap - d0 - k) * (long long)pow3z(p.C + p.m);
    const bool last = i == p.n_interp - 1;
    const int cols = last && p.cols_outer ? p.cols_outer : p.cols;  // outermost axes: hi = 1
    if (last && (kMixed || split))
      e = launch_interp<M, true>(k, cols, wbuf, z, hi, lo, st);
    else
      e = launch_interp<M, false>(k, cols, wbuf, wbuf, hi, lo, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace hc
