// Batching form: many independent hypercube convolutions of uneven D.
//
// Two ways to run an instance, both launched by hc_batched_launch (so one
// CUDA graph replays the whole batch):
//   fused   -- one unit of the persistent ticket engine (hc_persist.cuh):
//              C = min(D, tile axes), m = D - C <= 6 middle axes evaluated on
//              the fly; 3^m tile tickets, then column tickets interpolating
//              the middle axes while the instance's 3^D intermediate is in
//              L2.  All fused instances share one persistent launch; the
//              host builds one descriptor per instance and a ticket ->
//              (instance, local ticket) table in the interleaved order of
//              hc_persist.cuh, so a CTA finds its work with a single load.
//   grouped -- the instances of one D run as whole passes over all of them
//              (the PASSES schedule with an instance index): evaluation of
//              the a = D - C outer axes into one array per group, one tile
//              launch over every tile of the group, one interpolation pass
//              of the a outer axes over every instance.
// Instances with D <= fused_max_d are fused, the others grouped; the split
// (the fusion depth) is the batched autotuner's choice.
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "hc_common.cuh"
#include "hc_profile.cuh"
#include "hc_kernels.cuh"
#include "hc_persist.cuh"
#include "hc_tile.cuh"

namespace hc {

// counters[0]: ticket counter; counters[1 + i]: finished tiles of instance i.
template <class M>
__global__ void __launch_bounds__(256, (sizeof(typename M::W) == 4 ? 2 : 1)) batched_kernel(const UnitDesc* __restrict__ desc,
                                                      const int2* __restrict__ ticket_map,
                                                      long long total,
                                                      unsigned long long* counters,
                                                      WsHeader* hdr) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr bool kFin = !std::is_same<typename M::W, typename M::Out>::value;
  UniformUnits none;
  persistent_loop<M, -1, false, kFin>(desc, ticket_map, none, total, counters, hdr, smem);
}

// ---------------------------------------------------------------------------
// Grouped form: per-instance pointers of one group.
struct GroupPtrs {
  const void* x;
  const void* y;
  void* w;  // intermediate (the output array itself unless mixed precision)
  void* z;  // output
};

// First evaluation pass of a group: K outer axes of every instance, read from
// its own x, y ([2^K][lo] each), written to dx, dy ([n][3^K][lo]).
template <class M, int K>
__global__ void __launch_bounds__(256) group_eval_kernel(const GroupPtrs* __restrict__ tab, int n,
                                                         long long lo,
                                                         typename M::In* __restrict__ dx,
                                                         typename M::In* __restrict__ dy) {
  typedef typename M::In T;
  const long long cols = (long long)n * lo;
#pragma unroll 1
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < cols;
       c += (long long)gridDim.x * blockDim.x) {
    const long long i = c / lo, l = c - i * lo;
    const T* src = reinterpret_cast<const T*>(blockIdx.y ? tab[i].y : tab[i].x) + l;
    T v[p3(K)];
#pragma unroll
    for (int b = 0; b < p2(K); ++b) v[b] = src[b * lo];
    eval_pencil<M, K>(v);
    T* d = (blockIdx.y ? dy : dx) + i * p3(K) * lo + l;
#pragma unroll
    for (int j = 0; j < p3(K); ++j) d[j * lo] = v[j];
  }
}

// Tiles of a group: tile t belongs to instance t / per (local tile t % per);
// its rows come from the evaluated operands X, Y ([n * per][2^C]) or, when
// X is null (every instance is one tile), from the instance's own x, y.
// The next tile's rows are prefetched with cp.async as in tile_conv_kernel.
template <class M, int C, bool FINAL>
__global__ void __launch_bounds__(256) group_tile_kernel(const GroupPtrs* __restrict__ tab,
                                                         const typename M::In* __restrict__ X,
                                                         const typename M::In* __restrict__ Y,
                                                         long long per, long long ntiles) {
  typedef typename M::In In;
  typedef typename std::conditional<FINAL, typename M::Out, typename M::W>::type O;
  extern __shared__ __align__(16) unsigned char smem[];
  In* rows = reinterpret_cast<In*>(smem + TileRows<M, C>::kOff);  // [buffer][operand][2^C]
  auto src = [&](long long t, int op) -> const In* {
    if (X) return (op ? Y : X) + t * p2(C);
    return reinterpret_cast<const In*>(op ? tab[t].y : tab[t].x);
  };
  auto prefetch = [&](long long t, int b) {
#pragma unroll 1
    for (int e = threadIdx.x; e < 2 * p2(C); e += blockDim.x) {
      const int op = e >> C, i = e & (p2(C) - 1);
      cp_async<sizeof(In)>(rows + (b * 2 + op) * p2(C) + i, src(t, op) + i);
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
    const long long i = t / per, local = t - i * per;
    O* out = reinterpret_cast<O*>(FINAL ? tab[i].z : tab[i].w) + local * p3(C);
    RowLoader<In> ld{rows + (it * 2 + 0) * p2(C), rows + (it * 2 + 1) * p2(C)};
    tile_body<M, C, FINAL>(ld, out, smem);
    if constexpr (TileShape<C>::G == 1) __syncthreads();  // buffer reuse
  }
}

// The same group tiles (intermediate only) stored with bulk copies
// (tile_loop_bulk), when every instance's intermediate array of the group is
// a plain device allocation.
// T44: the two four-axis groups of C = 8 binary32 tiles (TileStages44,
// 128 threads).
template <class M, int C, bool T44 = false>
__global__ void __launch_bounds__(T44 ? 128 : 256) group_tile_bulk_kernel(
    const GroupPtrs* __restrict__ tab, const typename M::In* __restrict__ X,
    const typename M::In* __restrict__ Y, long long per, long long ntiles) {
  typedef typename M::In In;
  typedef typename M::W W;
  extern __shared__ __align__(16) unsigned char smem[];
  auto src = [&](long long t, int op) -> const In* { return (op ? Y : X) + t * p2(C); };
  auto dst = [&](long long t) {
    const long long i = t / per, local = t - i * per;
    return reinterpret_cast<W*>(tab[i].w) + local * p3(C);
  };
  if constexpr (T44)
    tile_loop_bulk<M, C, decltype(src), decltype(dst), TileStages44<M>>(src, dst, ntiles, smem);
  else
    tile_loop_bulk<M, C>(src, dst, ntiles, smem);
}

// Interpolation of the a = K1 + K2 outer axes of every instance of a group,
// in place on its [3^a][lo] intermediate (FINAL: written to its output in
// the output type).  Tile t: instance t / per, columns (t % per) * L ...;
// the same three tile loops as interp_pass_kernel (double-buffered cp.async,
// register prefetch, or one tile at a time), each tile on its instance's
// arrays.
template <class M, int K1, int K2, int L, bool FINAL>
__global__ void __launch_bounds__(K1 > 0 ? ((p3(K2) * L + 31) / 32 * 32 < 1024
                                                 ? (p3(K2) * L + 31) / 32 * 32 : 1024)
                                          : 256)
    group_interp_kernel(const GroupPtrs* __restrict__ tab, long long lo, long long per,
                        long long ntiles) {
  typedef typename M::W W;
  extern __shared__ __align__(16) unsigned char smem[];
  if constexpr (K1 > 0 && (InterpPipe<M, K1, K2, L>::kOn || InterpPipe<M, K1, K2, L>::kReg)) {
    const long long first = blockIdx.x, step = gridDim.x;
    const int n = first < ntiles ? (int)((ntiles - 1 - first) / step + 1) : 0;
    auto tile = [&](int i, long long& base, long long& l0) {
      const long long t = first + (long long)i * step;
      l0 = (t - t / per * per) * L;
      base = l0;
    };
    auto ptrs = [&](int i, const W*& s, void*& d) {
      const long long inst = (first + (long long)i * step) / per;
      s = reinterpret_cast<const W*>(tab[inst].w);
      d = FINAL ? tab[inst].z : tab[inst].w;
    };
    if constexpr (InterpPipe<M, K1, K2, L>::kOn)
      interp_tiles_pipelined<M, K1, K2, L, FINAL, decltype(tile), false, decltype(ptrs)>(
          nullptr, nullptr, lo, n, tile, smem, ptrs);
    else
      interp_tiles_regpipe<M, K1, K2, L, FINAL, decltype(tile), false, decltype(ptrs)>(
          nullptr, nullptr, lo, n, tile, smem, ptrs);
  } else {
#pragma unroll 1
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const long long i = t / per, l0 = (t - i * per) * L;
      interp_tile_body<M, K1, K2, L, FINAL, false>(reinterpret_cast<const W*>(tab[i].w),
                                                   FINAL ? tab[i].z : tab[i].w, l0, l0, lo, smem);
    }
  }
}

// ---------------------------------------------------------------------------
// Host side.

// One group of the grouped form: the instances with one D.
struct GroupPlan {
  int D, C, a, n;
  bool bulk = false;  // every intermediate array is a plain device allocation
  size_t off_tab;           // GroupPtrs[n]
  size_t off_xo, off_yo;    // operands evaluated on the a outer axes, [n][3^a][2^C]
  size_t off_tx, off_ty;    // first evaluation pass when a > 3, [n][3^3][2^(D-3)]
};

struct BatchPlan {
  hc_dtype dtype;
  int fused_max_d;
  // fused part (persistent engine)
  int n;  // fused instances
  long long total;
  size_t smem;
  size_t off_ctr, off_desc, off_tab, off_w;
  std::vector<int> fused_index;  // instance -> fused unit, or -1 (grouped)
  // grouped part
  std::vector<GroupPlan> groups;
  size_t ws_bytes;
};

static std::mutex g_plans_mu;
static std::map<const void*, BatchPlan> g_plans;  // prepared workspaces

static int batch_cmax(hc_dtype dt) { return dt == HC_FP32 ? 9 : 8; }

// Fusion depth used when the caller does not choose one (measured on GB300:
// 4096 float32 instances with D in 6..14).
constexpr int kDefaultFusedMaxD = 9;

// Tile axes of an instance: 8-axis tiles keep the persistent kernel at
// several CTAs per SM (a 9-axis float32 tile needs 126 KB of shared memory);
// 9 only when D = 15.
static int batch_tile_axes(int D, hc_dtype dt) {
  const int ctile = D > 8 + 6 ? batch_cmax(dt) : 8;
  return D < ctile ? D : ctile;
}

static hc_status build_batch(const hc_instance* inst, int n, hc_dtype dt, int fused_max_d,
                             BatchPlan* plan, std::vector<UnitDesc>* descs,
                             std::vector<int2>* table,
                             std::vector<std::vector<GroupPtrs>>* gtabs, void* workspace) {
  if (n < 0 || (n > 0 && !inst)) return HC_ERR_ARG;
  const size_t es = elem_size(dt);
  if (es == 0 || dt == HC_FP32_FF) return HC_ERR_DTYPE;  // FF: plain form only
  const int cmax = batch_cmax(dt);
  const size_t wsz = (dt == HC_FP32_MIXED) ? 8 : es;
  const bool mixed = dt == HC_FP32_MIXED;
  const int L = kPersistCols;
  if (fused_max_d < 0) fused_max_d = 0;  // D = 0 instances always run fused
  BatchPlan p;
  p.dtype = dt;
  p.fused_max_d = fused_max_d;
  p.n = 0;
  p.total = 0;
  p.smem = 0;
  p.fused_index.assign(n, -1);
  long long ticket = 0;
  size_t smem = 0, wbytes = 0;
  std::vector<UnitDesc> fd;
  std::vector<int> by_d[HC_MAX_D + 1];
  for (int i = 0; i < n; ++i) {
    const hc_instance& q = inst[i];
    if (q.D < 0 || q.D > cmax + 6) return HC_ERR_ARG;
    if (!q.x || !q.y || !q.z) return HC_ERR_ARG;
    if (!aligned(q.x, 16) || !aligned(q.y, 16) || !aligned(q.z, 16)) return HC_ERR_ALIGN;
    const size_t nx = es << q.D, nz = es * pow3z(q.D);
    if (overlaps(q.z, nz, q.x, nx) || overlaps(q.z, nz, q.y, nx)) return HC_ERR_ALIAS;
    if (q.D > fused_max_d) {
      by_d[q.D].push_back(i);
      continue;
    }
    UnitDesc d;
    memset(&d, 0, sizeof(d));
    d.x = q.x;
    d.y = q.y;
    d.z = q.z;
    d.w = q.z;
    d.C = batch_tile_axes(q.D, dt);
    d.m = q.D - d.C;
    d.n_tiles = (int)pow3z(d.m);
    if (d.m > 0) {
      const long long coltiles = ((long long)pow3z(d.C) + L - 1) / L;
      long long cpt = 32768 / ((long long)pow3z(d.m) * L);
      if (cpt < 1) cpt = 1;
      d.cpt = (int)cpt;
      d.n_cols = (int)((coltiles + cpt - 1) / cpt);
    } else {
      d.cpt = 1;
      d.n_cols = 0;
    }
    d.need = d.n_tiles;
    d.first = ticket;
    ticket += d.n_tiles + d.n_cols;
    if (mixed && d.m > 0) {
      d.w = (void*)(uintptr_t)wbytes;  // offset for now; rebased below
      wbytes = align_up(wbytes + 8 * pow3z(q.D), 256);
    }
    size_t sm = d.C > 0 ? tile_smem_bytes(dt, d.C) : 0;
    const size_t ism = d.m >= 4 ? 2 * wsz * pow3z(d.m) * L : 0;
    if (ism > sm) sm = ism;
    if (sm > smem) smem = sm;
    p.fused_index[i] = (int)fd.size();
    fd.push_back(d);
  }
  p.n = (int)fd.size();
  p.total = ticket;
  p.smem = smem;
  size_t off = kWsHeader;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  p.off_ctr = take(8 * (size_t)(p.n + 1));
  p.off_desc = take(sizeof(UnitDesc) * (size_t)p.n);
  p.off_tab = take(sizeof(int2) * (size_t)ticket);
  p.off_w = take(wbytes);
  for (auto& d : fd)
    if (mixed && d.m > 0) d.w = workspace ? (unsigned char*)workspace + p.off_w + (uintptr_t)d.w : nullptr;
  // grouped part
  if (gtabs) gtabs->clear();
  for (int D = 0; D <= HC_MAX_D; ++D) {
    if (by_d[D].empty()) continue;
    GroupPlan g;
    g.D = D;
    g.C = batch_tile_axes(D, dt);
    g.a = D - g.C;
    g.n = (int)by_d[D].size();
    g.off_tab = take(sizeof(GroupPtrs) * (size_t)g.n);
    const size_t rows = (size_t)g.n * pow3z(g.a) << g.C;
    g.off_xo = g.a > 0 ? take(rows * es) : 0;
    g.off_yo = g.a > 0 ? take(rows * es) : 0;
    const size_t trows = (size_t)g.n * 27 << (D > 3 ? D - 3 : 0);
    g.off_tx = g.a > 3 ? take(trows * es) : 0;
    g.off_ty = g.a > 3 ? take(trows * es) : 0;
    std::vector<GroupPtrs> tab(g.n);
    for (int k = 0; k < g.n; ++k) {
      const hc_instance& q = inst[by_d[D][k]];
      tab[k].x = q.x;
      tab[k].y = q.y;
      tab[k].z = q.z;
      tab[k].w = q.z;
      if (mixed && g.a > 0) {
        const size_t wo = take(8 * pow3z(D));
        tab[k].w = workspace ? (unsigned char*)workspace + wo : nullptr;
      }
    }
    if (gtabs) gtabs->push_back(std::move(tab));
    p.groups.push_back(g);
  }
  p.ws_bytes = off;
  if (descs) *descs = fd;
  if (table) {
    // tiles(0), tiles(1), cols(0), tiles(2), cols(1), ..., cols(n - 1)
    table->clear();
    table->reserve((size_t)ticket);
    const int nf = p.n;
    if (nf > 0)
      for (int t = 0; t < fd[0].n_tiles; ++t) table->push_back(make_int2(0, t));
    for (int i = 0; i < nf; ++i) {
      if (i + 1 < nf)
        for (int t = 0; t < fd[i + 1].n_tiles; ++t) table->push_back(make_int2(i + 1, t));
      for (int c = 0; c < fd[i].n_cols; ++c) table->push_back(make_int2(i, fd[i].n_tiles + c));
    }
  }
  *plan = std::move(p);
  return HC_OK;
}

template <class M>
static cudaError_t launch_fused_m(const BatchPlan& p, unsigned char* ws, cudaStream_t st) {
  auto k = batched_kernel<M>;
  ProfileScope prof(st, "batched");
  cudaError_t e = prep_kernel(k, p.smem);
  if (e != cudaSuccess) return e;
  k<<<grid_for(k, 256, p.smem, p.total), 256, p.smem, st>>>(
      (const UnitDesc*)(ws + p.off_desc), (const int2*)(ws + p.off_tab), p.total,
      (unsigned long long*)(ws + p.off_ctr), (WsHeader*)ws);
  return cudaGetLastError();
}

template <class M, int K>
static cudaError_t launch_group_eval_k(const GroupPtrs* tab, int n, long long lo,
                                       typename M::In* dx, typename M::In* dy, cudaStream_t st) {
  ProfileScope prof(st, "batched_eval");
  const long long cols = (long long)n * lo;
  long long blocks = (cols + 255) / 256;
  const long long cap = (long long)device_caps().sms * 8;
  if (blocks > cap) blocks = cap;
  group_eval_kernel<M, K><<<dim3((unsigned)blocks, 2), 256, 0, st>>>(tab, n, lo, dx, dy);
  return cudaGetLastError();
}

template <class M, int C, bool FINAL>
static cudaError_t launch_group_tile_c(const GroupPtrs* tab, const typename M::In* X,
                                       const typename M::In* Y, long long per, long long ntiles,
                                       bool bulk, cudaStream_t st) {
  ProfileScope prof(st, "batched_tile");
  if constexpr (use_bulk_tiles<M, C, FINAL>()) {
    if (bulk) {
      const size_t smem = TileBulk<M, C>::bytes;
      constexpr bool t44 = use_tile44<M, C>();
      constexpr int threads = t44 ? 128 : 256;
      auto k = group_tile_bulk_kernel<M, C, t44>;
      cudaError_t e = prep_kernel(k, smem);
      if (e != cudaSuccess) return e;
      k<<<grid_for(k, threads, smem, ntiles), threads, smem, st>>>(tab, X, Y, per, ntiles);
      return cudaGetLastError();
    }
  }
  const size_t smem = TileRows<M, C>::bytes;
  auto k = group_tile_kernel<M, C, FINAL>;
  cudaError_t e = prep_kernel(k, smem);
  if (e != cudaSuccess) return e;
  const int threads = C >= 4 ? 256 : 32;
  k<<<grid_for(k, threads, smem, ntiles), threads, smem, st>>>(tab, X, Y, per, ntiles);
  return cudaGetLastError();
}

template <class M, bool FINAL>
static cudaError_t launch_group_tile(int C, const GroupPtrs* tab, const typename M::In* X,
                                     const typename M::In* Y, long long per, long long ntiles,
                                     bool bulk, cudaStream_t st) {
  switch (C) {
    case 1: return launch_group_tile_c<M, 1, FINAL>(tab, X, Y, per, ntiles, bulk, st);
    case 2: return launch_group_tile_c<M, 2, FINAL>(tab, X, Y, per, ntiles, bulk, st);
    case 3: return launch_group_tile_c<M, 3, FINAL>(tab, X, Y, per, ntiles, bulk, st);
    case 4: return launch_group_tile_c<M, 4, FINAL>(tab, X, Y, per, ntiles, bulk, st);
    case 5: return launch_group_tile_c<M, 5, FINAL>(tab, X, Y, per, ntiles, bulk, st);
    case 6: return launch_group_tile_c<M, 6, FINAL>(tab, X, Y, per, ntiles, bulk, st);
    case 7: return launch_group_tile_c<M, 7, FINAL>(tab, X, Y, per, ntiles, bulk, st);
    case 8: return launch_group_tile_c<M, 8, FINAL>(tab, X, Y, per, ntiles, bulk, st);
    case 9:
      if constexpr (sizeof(typename M::W) == 4)
        return launch_group_tile_c<M, 9, FINAL>(tab, X, Y, per, ntiles, bulk, st);
      return cudaErrorInvalidValue;
  }
  return cudaErrorInvalidValue;
}

template <class M, int K1, int K2, bool FINAL>
static cudaError_t launch_group_interp_k(const GroupPtrs* tab, int n, long long lo,
                                         cudaStream_t st) {
  // columns per tile: 32, except 16 for 8-byte intermediates below 6 axes
  // (two 16-column buffers double-buffer at two CTAs per SM) and 64 for
  // 4-byte ones over 4 axes (81-row tiles: 32 columns leave each CTA only
  // 10 KB in flight; the 4096-instance float32 batch 9.60 -> 9.47 ms; 16
  // columns over 6 axes measured 9.49 -> 10.21 ms and are not used)
  constexpr int L = K1 == 0 ? 256
                    : (sizeof(typename M::W) == 8 && K1 + K2 < 6
                           ? 16
                           : (sizeof(typename M::W) == 4 && K1 + K2 == 4 ? 64 : 32));
  constexpr size_t smem = K1 > 0 ? InterpPipe<M, K1, K2, L>::kSmem : 0;
  constexpr int tw = (p3(K2) * L + 31) / 32 * 32;
  constexpr int threads = K1 > 0 ? (tw < 1024 ? tw : 1024) : 256;
  auto k = group_interp_kernel<M, K1, K2, L, FINAL>;
  ProfileScope prof(st, "batched_interp");
  cudaError_t e = prep_kernel(k, smem);
  if (e != cudaSuccess) return e;
  const long long per = (lo + L - 1) / L, ntiles = (long long)n * per;
  k<<<grid_for(k, threads, smem, ntiles), threads, smem, st>>>(tab, lo, per, ntiles);
  return cudaGetLastError();
}

template <class M, bool FINAL>
static cudaError_t launch_group_interp(int a, const GroupPtrs* tab, int n, long long lo,
                                       cudaStream_t st) {
  switch (a) {
    case 1: return launch_group_interp_k<M, 0, 1, FINAL>(tab, n, lo, st);
    case 2: return launch_group_interp_k<M, 0, 2, FINAL>(tab, n, lo, st);
    case 3: return launch_group_interp_k<M, 0, 3, FINAL>(tab, n, lo, st);
    // balanced splits: the round-1 pencils (3^K2 elements, 3^K1 * L of them)
    // and the round-2 pencils (3^K1 elements, 3^K2 * L of them) keep every
    // one of the 3^K2 * L threads busy in both rounds (K2 = 3 left two
    // thirds of them idle in round 1 at 5 axes and eight ninths at 4): the
    // 4096-instance float32 batch 9.41 -> 9.25 ms on GB300, same bits
    case 4: return launch_group_interp_k<M, 2, 2, FINAL>(tab, n, lo, st);
    case 5: return launch_group_interp_k<M, 3, 2, FINAL>(tab, n, lo, st);
    case 6: return launch_group_interp_k<M, 3, 3, FINAL>(tab, n, lo, st);
  }
  return cudaErrorInvalidValue;
}

template <class M>
static cudaError_t launch_groups_m(const BatchPlan& p, unsigned char* ws, cudaStream_t st) {
  typedef typename M::In In;
  constexpr bool kMixed = !std::is_same<typename M::W, typename M::Out>::value;
  cudaError_t e = cudaSuccess;
  for (const GroupPlan& g : p.groups) {
    const GroupPtrs* tab = (const GroupPtrs*)(ws + g.off_tab);
    In* X = nullptr;
    In* Y = nullptr;
    if (g.a > 0) {
      // evaluate the a outer axes: the first <= 3 from the instances, the rest
      // on the group's array
      In* xo = (In*)(ws + g.off_xo);
      In* yo = (In*)(ws + g.off_yo);
      const int k1 = g.a < 3 ? g.a : 3;
      In* dx = g.a > 3 ? (In*)(ws + g.off_tx) : xo;
      In* dy = g.a > 3 ? (In*)(ws + g.off_ty) : yo;
      const long long lo1 = 1ll << (g.D - k1);
      switch (k1) {
        case 1: e = launch_group_eval_k<M, 1>(tab, g.n, lo1, dx, dy, st); break;
        case 2: e = launch_group_eval_k<M, 2>(tab, g.n, lo1, dx, dy, st); break;
        case 3: e = launch_group_eval_k<M, 3>(tab, g.n, lo1, dx, dy, st); break;
      }
      if (e != cudaSuccess) return e;
      if (g.a > 3) {
        e = launch_eval<M>(g.a - 3, dx, dy, xo, yo, (long long)g.n * 27, 1ll << g.C, st);
        if (e != cudaSuccess) return e;
      }
      X = xo;
      Y = yo;
    }
    const long long per = (long long)pow3z(g.a), ntiles = (long long)g.n * per;
    if (g.a == 0)
      e = launch_group_tile<M, true>(g.C, tab, nullptr, nullptr, 1, ntiles, false, st);
    else
      e = launch_group_tile<M, false>(g.C, tab, X, Y, per, ntiles, g.bulk, st);
    if (e != cudaSuccess) return e;
    if (g.a > 0) {
      e = launch_group_interp<M, kMixed>(g.a, tab, g.n, (long long)pow3z(g.C), st);
      if (e != cudaSuccess) return e;
    }
  }
  return e;
}

static hc_status batched_launch_plan(const BatchPlan& p, void* workspace, cudaStream_t st) {
  unsigned char* ws = (unsigned char*)workspace;
  cudaError_t e = cudaSuccess;
  if (p.n > 0 && p.total > 0) {
    // status word and counters are contiguous from the start of the workspace
    e = cudaMemsetAsync(ws, 0, p.off_ctr + 8 * (size_t)(p.n + 1), st);
    if (e != cudaSuccess) return record_cuda_error(e);
    switch (p.dtype) {
      case HC_INT64: e = launch_fused_m<ModeI64>(p, ws, st); break;
      case HC_FP64: e = launch_fused_m<ModeF64>(p, ws, st); break;
      case HC_FP32: e = launch_fused_m<ModeF32>(p, ws, st); break;
      case HC_FP32_MIXED: e = launch_fused_m<ModeMixed>(p, ws, st); break;
    }
    if (e != cudaSuccess) return record_cuda_error(e);
  }
  if (!p.groups.empty()) {
    switch (p.dtype) {
      case HC_INT64: e = launch_groups_m<ModeI64>(p, ws, st); break;
      case HC_FP64: e = launch_groups_m<ModeF64>(p, ws, st); break;
      case HC_FP32: e = launch_groups_m<ModeF32>(p, ws, st); break;
      case HC_FP32_MIXED: e = launch_groups_m<ModeMixed>(p, ws, st); break;
    }
  }
  return record_cuda_error(e);
}

static hc_status prepare(const hc_instance* inst, int n, hc_dtype dtype, int fused_max_d,
                         void* workspace, size_t ws_bytes, cudaStream_t stream) {
  BatchPlan p;
  hc_status s = build_batch(inst, n, dtype, fused_max_d, &p, nullptr, nullptr, nullptr, nullptr);
  if (s != HC_OK) return s;
  if (!workspace) return HC_ERR_ARG;
  if (!aligned(workspace, 256)) return HC_ERR_ALIGN;
  if (ws_bytes < p.ws_bytes) return HC_ERR_WORKSPACE;
  const size_t es = elem_size(dtype);
  for (int i = 0; i < n; ++i) {
    const size_t nx = es << inst[i].D, nz = es * pow3z(inst[i].D);
    if (overlaps(workspace, p.ws_bytes, inst[i].z, nz) ||
        overlaps(workspace, p.ws_bytes, inst[i].x, nx) ||
        overlaps(workspace, p.ws_bytes, inst[i].y, nx))
      return HC_ERR_ALIAS;
  }
  std::vector<UnitDesc> descs;
  std::vector<int2> table;
  std::vector<std::vector<GroupPtrs>> gtabs;
  s = build_batch(inst, n, dtype, fused_max_d, &p, &descs, &table, &gtabs, workspace);
  if (s != HC_OK) return s;
  // groups whose intermediate arrays are all plain device allocations store
  // their tiles with bulk copies (checked once here, not at every launch)
  for (size_t g = 0; g < p.groups.size(); ++g) {
    bool all = p.groups[g].a > 0;
    for (size_t k = 0; all && k < gtabs[g].size(); ++k) all = is_device_allocation(gtabs[g][k].w);
    p.groups[g].bulk = all;
  }
  unsigned char* ws = (unsigned char*)workspace;
  cudaError_t e = cudaSuccess;
  if (p.n > 0)
    e = cudaMemcpyAsync(ws + p.off_desc, descs.data(), sizeof(UnitDesc) * (size_t)p.n,
                        cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess && !table.empty())
    e = cudaMemcpyAsync(ws + p.off_tab, table.data(), sizeof(int2) * table.size(),
                        cudaMemcpyHostToDevice, stream);
  for (size_t g = 0; e == cudaSuccess && g < p.groups.size(); ++g)
    e = cudaMemcpyAsync(ws + p.groups[g].off_tab, gtabs[g].data(),
                        sizeof(GroupPtrs) * gtabs[g].size(), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return record_cuda_error(e);
  std::lock_guard<std::mutex> g(g_plans_mu);
  g_plans[workspace] = std::move(p);
  return HC_OK;
}

static bool lookup_plan(const void* workspace, BatchPlan* p) {
  std::lock_guard<std::mutex> g(g_plans_mu);
  auto it = g_plans.find(workspace);
  if (it == g_plans.end()) return false;
  *p = it->second;
  return true;
}

// Fusion depths the batched autotuner tries: everything fused, nothing fused
// (but D = 0), and every split in between that separates the batch.
static std::vector<int> split_candidates(const hc_instance* inst, int n, hc_dtype dt) {
  int dmax = 0;
  bool have[HC_MAX_D + 1] = {false};
  for (int i = 0; i < n; ++i)
    if (inst[i].D >= 0 && inst[i].D <= HC_MAX_D) {
      have[inst[i].D] = true;
      if (inst[i].D > dmax) dmax = inst[i].D;
    }
  std::vector<int> v;
  v.push_back(-1);
  for (int d = 0; d < dmax; ++d)
    if (have[d]) v.push_back(d);
  v.push_back(batch_cmax(dt) + 6);
  return v;
}

}  // namespace hc

extern "C" size_t hc_batched_workspace_size(const hc_instance* inst, int n, hc_dtype dtype) {
  // the largest over every fusion depth, so that one workspace serves any
  // split (and the autotuner)
  size_t best = 0;
  for (int split : hc::split_candidates(inst, n, dtype)) {
    hc::BatchPlan p;
    if (hc::build_batch(inst, n, dtype, split, &p, nullptr, nullptr, nullptr, nullptr) != HC_OK)
      return 0;
    if (p.ws_bytes > best) best = p.ws_bytes;
  }
  return best;
}

extern "C" hc_status hc_batched_prepare(const hc_instance* inst, int n, hc_dtype dtype,
                                        void* workspace, size_t ws_bytes, hc_stream_t stream) {
  return hc::prepare(inst, n, dtype, hc::kDefaultFusedMaxD, workspace, ws_bytes,
                     (cudaStream_t)stream);
}

extern "C" hc_status hc_batched_prepare_split(const hc_instance* inst, int n, hc_dtype dtype,
                                              int fused_max_d, void* workspace, size_t ws_bytes,
                                              hc_stream_t stream) {
  if (fused_max_d < -1) return HC_ERR_ARG;
  return hc::prepare(inst, n, dtype, fused_max_d, workspace, ws_bytes, (cudaStream_t)stream);
}

extern "C" hc_status hc_batched_launch(void* workspace, size_t ws_bytes, hc_stream_t stream) {
  using namespace hc;
  if (!workspace) return HC_ERR_ARG;
  BatchPlan p;
  if (!lookup_plan(workspace, &p)) return HC_ERR_ARG;
  if (ws_bytes < p.ws_bytes) return HC_ERR_WORKSPACE;
  return batched_launch_plan(p, workspace, (cudaStream_t)stream);
}

extern "C" hc_status hc_batched_autotune(const hc_instance* inst, int n, hc_dtype dtype,
                                         void* workspace, size_t ws_bytes, int reps,
                                         hc_stream_t stream, int* best_fused_max_d,
                                         double* best_ms) {
  using namespace hc;
  if (!best_fused_max_d || reps < 1) return HC_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return record_cuda_error(cudaGetLastError());
  int best = -2;
  float best_t = 0;
  hc_status s = HC_OK;
  for (int split : split_candidates(inst, n, dtype)) {
    s = prepare(inst, n, dtype, split, workspace, ws_bytes, st);
    if (s != HC_OK) break;
    s = hc_batched_launch(workspace, ws_bytes, stream);  // warm-up
    if (s != HC_OK) break;
    float ms = 0;
    cudaError_t e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && s == HC_OK; ++r) s = hc_batched_launch(workspace, ws_bytes, stream);
    if (s != HC_OK) break;
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      s = record_cuda_error(e);
      break;
    }
    ms /= reps;
    if (best == -2 || ms < best_t) {
      best = split;
      best_t = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != HC_OK) return s;
  if (best == -2) return HC_ERR_ARG;
  *best_fused_max_d = best;
  if (best_ms) *best_ms = best_t;
  return prepare(inst, n, dtype, best, workspace, ws_bytes, st);  // leave the winner prepared
}

extern "C" hc_status hc_batched_inject_stall(void* workspace, int instance) {
  using namespace hc;
  if (!workspace) return HC_ERR_ARG;
  BatchPlan p;
  if (!lookup_plan(workspace, &p)) return HC_ERR_ARG;
  if (instance < 0 || instance >= (int)p.fused_index.size()) return HC_ERR_ARG;
  const int u = p.fused_index[instance];
  if (u < 0) return HC_OK;  // a grouped instance has no waits
  unsigned char* d = (unsigned char*)workspace + p.off_desc + sizeof(UnitDesc) * (size_t)u;
  UnitDesc desc;
  cudaError_t e = cudaMemcpy(&desc, d, sizeof(desc), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return record_cuda_error(e);
  desc.need = desc.n_tiles + 1;  // one more finished tile than the instance has
  e = cudaMemcpy(d, &desc, sizeof(desc), cudaMemcpyHostToDevice);
  return record_cuda_error(e);
}

extern "C" hc_status hc_convolve_batched(const hc_instance* inst, int n, hc_dtype dtype,
                                         void* workspace, size_t ws_bytes, hc_stream_t stream) {
  hc_status s = hc_batched_prepare(inst, n, dtype, workspace, ws_bytes, stream);
  if (s != HC_OK) return s;
  return hc_batched_launch(workspace, ws_bytes, stream);
}
