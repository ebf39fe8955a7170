// Kernels and launch helpers shared by the forward, backward and batched
// translation units.
#pragma once

#include "hc_common.cuh"
#include "hc_tile.cuh"
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

// Bulk tile stores where they apply: intermediate tiles (a final-tile
// launch is a single tile, D <= C), C >= 4, and two CTAs with two W buffers
// each still fit one SM's shared memory.
template <class M, int C, bool FINAL>
constexpr bool use_bulk_tiles() {
  return !FINAL && C >= 4 && 2 * (TileBulk<M, C>::bytes + 1024) <= 228 * 1024;
}

// Bulk copies are issued only into plain device allocations (not managed or
// host-mapped memory, which the per-thread stores handle).
inline bool is_device_allocation(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice;
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

// ---------------------------------------------------------------------------
// K3 kernel: interpolate k = K1 + K2 consecutive axes of a [hi][3^k][lo]
// array; a CTA tile is all 3^k rows of L consecutive columns of one h.
// src and dst may be the same array (every tile reads its elements before
// writing any; tiles are disjoint).
// Whether the pass double-buffers its tiles: only when two buffers still let
// two CTAs share an SM (otherwise the lost occupancy costs more than the
// overlap gains; measured on GB300).
// Otherwise, when the next tile's round-1 pencil fits in registers beside
// the current round-2 pencil (estimated 2 pencils + 24 registers a thread,
// one CTA per SM), it is prefetched into registers (interp_tiles_regpipe).
template <class M, int K1, int K2, int L>
struct InterpPipe {
  static constexpr size_t kBuf = sizeof(typename M::W) * (size_t)p3(K1 + K2) * L;
  static constexpr bool kOn = K1 > 0 && 2 * kBuf <= 113 * 1024;
  static constexpr int kThreads = (p3(K2) * L + 31) / 32 * 32;
  // registers a thread needs: two pencils plus addressing (16 for 4-byte
  // values: the 27-row, 32-column binary32 pass fits 864 threads in 72
  // registers without spills, which lets its tiles be register-prefetched;
  // GB300: 4096-instance batch 8.74 -> 8.42 ms, D = 19 float32 passes 4.43
  // -> 4.34 ms)
  static constexpr int kRegs =
      2 * p3(K2) * (int)(sizeof(typename M::W) / 4) + (sizeof(typename M::W) == 4 ? 16 : 24);
  static constexpr bool kReg = K1 > 0 && K1 <= K2 && !kOn && kThreads * kRegs <= 65536;
  static constexpr size_t kSmem = K1 == 0 ? 0 : (kOn ? 2 * kBuf : kBuf);
};

template <class M, int K1, int K2, int L, bool FINAL, bool TR>
__global__ void __launch_bounds__(K1 > 0 ? (p3(K2) * L + 31) / 32 * 32 : 256) interp_pass_kernel(const typename M::W* src, void* dst_,
                                                          long long hi, long long lo) {
  extern __shared__ __align__(16) unsigned char smem[];
  const long long ctiles = (lo + L - 1) / L;
  const long long ntiles = hi * ctiles;
  if constexpr (InterpPipe<M, K1, K2, L>::kOn) {
    // this CTA's tiles blockIdx.x, blockIdx.x + gridDim.x, ... double-buffered
    const long long first = blockIdx.x, step = gridDim.x;
    const int n = first < ntiles ? (int)((ntiles - 1 - first) / step + 1) : 0;
    auto tile = [&](int i, long long& base, long long& l0) {
      const long long t = first + (long long)i * step;
      const long long h = t / ctiles;
      l0 = (t - h * ctiles) * L;
      base = h * p3(K1 + K2) * lo + l0;
    };
    interp_tiles_pipelined<M, K1, K2, L, FINAL, decltype(tile), TR>(src, dst_, lo, n, tile, smem);
  } else if constexpr (InterpPipe<M, K1, K2, L>::kReg) {
    const long long first = blockIdx.x, step = gridDim.x;
    const int n = first < ntiles ? (int)((ntiles - 1 - first) / step + 1) : 0;
    auto tile = [&](int i, long long& base, long long& l0) {
      const long long t = first + (long long)i * step;
      const long long h = t / ctiles;
      l0 = (t - h * ctiles) * L;
      base = h * p3(K1 + K2) * lo + l0;
    };
    interp_tiles_regpipe<M, K1, K2, L, FINAL, decltype(tile), TR>(src, dst_, lo, n, tile, smem);
  } else {
#pragma unroll 1
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const long long h = tile / ctiles;
      const long long l0 = (tile - h * ctiles) * L;
      interp_tile_body<M, K1, K2, L, FINAL, false, TR>(src, dst_, h * p3(K1 + K2) * lo + l0, l0,
                                                       lo, smem);
    }
  }
}

// K3 with 16-byte row copies (interp_tiles_wide).
template <class M, int K1, int K2, int L, bool FINAL, bool TR>
__global__ void __launch_bounds__((p3(K2) * L + 31) / 32 * 32) interp_wide_kernel(const typename M::W* src, void* dst_,
                                                          long long hi, long long lo) {
  extern __shared__ __align__(16) unsigned char smem[];
  const long long ctiles = (lo + L - 1) / L;
  const long long ntiles = hi * ctiles;
  const long long first = blockIdx.x, step = gridDim.x;
  const int n = first < ntiles ? (int)((ntiles - 1 - first) / step + 1) : 0;
  auto tile = [&](int i, long long& base, long long& l0) {
    const long long t = first + (long long)i * step;
    const long long h = t / ctiles;
    l0 = (t - h * ctiles) * L;
    base = h * p3(K1 + K2) * lo + l0;
  };
  interp_tiles_wide<M, K1, K2, L, FINAL, decltype(tile), TR>(src, dst_, lo, hi * p3(K1 + K2) * lo, n,
                                                             tile, smem);
}

// Columns per whole-array interpolation tile (the schedule's `cols`).
template <class M>
inline int default_cols() {
  return sizeof(typename M::W) == 4 ? 32 : 16;
}

// k = K1 + K2 axes per pass; K1 > 0: a CTA of 27 * L threads (one pencil per
// thread and round) owns an L-column tile; K1 == 0: 256 columns per CTA, one
// column per thread.
template <class M, int K1, int K2, int L, bool FINAL, bool TR>
inline cudaError_t launch_interp_kl(const typename M::W* src, void* dst, long long hi,
                                    long long lo, cudaStream_t st) {
  constexpr int LT = K1 > 0 ? L : 256;
  const size_t smem = InterpPipe<M, K1, K2, LT>::kSmem;
  auto k = interp_pass_kernel<M, K1, K2, LT, FINAL, TR>;
  ProfileScope prof(st, TR ? "interp_t_pass" : "interp_pass");
  cudaError_t e = prep_kernel(k, smem);
  if (e != cudaSuccess) return e;
  int threads = K1 > 0 ? (p3(K2) * L + 31) / 32 * 32 : 256;
  if (threads > 1024) threads = 1024;
  const long long ntiles = hi * ((lo + LT - 1) / LT);
  k<<<grid_for(k, threads, smem, ntiles), threads, smem, st>>>(src, dst, hi, lo);
  return cudaGetLastError();
}

// The same pass with 16-byte row copies (interp_wide_kernel).
template <class M, int K1, int K2, int L, bool FINAL, bool TR>
inline cudaError_t launch_wide_kl(const typename M::W* src, void* dst, long long hi, long long lo,
                                  cudaStream_t st) {
  typedef WideRows<M, K1, K2, L> WR;
  auto k = interp_wide_kernel<M, K1, K2, L, FINAL, TR>;
  ProfileScope prof(st, TR ? "interp_t_pass" : "interp_pass");
  cudaError_t e = prep_kernel(k, WR::kSmem);
  if (e != cudaSuccess) return e;
  const int threads = (p3(K2) * L + 31) / 32 * 32;
  const long long ntiles = hi * ((lo + L - 1) / L);
  k<<<grid_for(k, threads, WR::kSmem, ntiles), threads, WR::kSmem, st>>>(src, dst, hi, lo);
  return cudaGetLastError();
}

// cols: 8, 16, 32 columns per tile with per-element copies; -16, -32: 16 or
// 32 columns with 16-byte row copies.
template <class M, int K1, int K2, bool FINAL, bool TR>
inline cudaError_t launch_interp_k(int cols, const typename M::W* src, void* dst, long long hi,
                                   long long lo, cudaStream_t st) {
  if constexpr (K1 == 0) return launch_interp_kl<M, 0, K2, 256, FINAL, TR>(src, dst, hi, lo, st);
  switch (cols) {
    case 8: return launch_interp_kl<M, K1, K2, 8, FINAL, TR>(src, dst, hi, lo, st);
    case 16: return launch_interp_kl<M, K1, K2, 16, FINAL, TR>(src, dst, hi, lo, st);
    case 32: return launch_interp_kl<M, K1, K2, 32, FINAL, TR>(src, dst, hi, lo, st);
    case -16: return launch_wide_kl<M, K1, K2, 16, FINAL, TR>(src, dst, hi, lo, st);
    case -32: return launch_wide_kl<M, K1, K2, 32, FINAL, TR>(src, dst, hi, lo, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// The last pass of the padded schedule: interpolate the k outermost axes of
// the padded intermediate [3^k][lo] (lo = 3^(a-k) * pitch: blocks of `pitch`
// columns of which the first cn = 3^C are real) and store the results in z's
// own layout [3^k][lo / pitch * cn].  The reads are 128-byte aligned rows;
// padding columns are read and interpolated but never stored.  K1 > 0: one
// round-1 pencil per thread prefetched into registers for the next tile
// while round 2 of this one runs (as interp_tiles_regpipe); K1 == 0: whole
// columns per thread, no shared memory.
template <class M, int K1, int K2, int L>
__global__ void __launch_bounds__(K1 > 0 ? p3(K2) * L : 256)
    interp_remap_kernel(const typename M::W* __restrict__ src, typename M::Out* __restrict__ dst,
                        long long lo, long long pitch, long long cn) {
  typedef typename M::W W;
  extern __shared__ __align__(16) unsigned char smem[];
  const long long lo_z = lo / pitch * cn;
  auto zcol = [&](long long c, long long& zc) -> bool {  // false: a padding column
    const long long q = c / pitch, r = c - q * pitch;
    zc = q * cn + r;
    return c < lo && r < cn;
  };
  if constexpr (K1 == 0) {
#pragma unroll 1
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < lo;
         c += (long long)gridDim.x * blockDim.x) {
      long long zc;
      if (!zcol(c, zc)) continue;
      W v[p3(K2)];
#pragma unroll
      for (int j = 0; j < p3(K2); ++j) v[j] = src[j * lo + c];
      interp_pencil<M, K2>(v);
#pragma unroll
      for (int j = 0; j < p3(K2); ++j) dst[j * lo_z + zc] = M::out(v[j]);
    }
  } else {
    W* T = reinterpret_cast<W*>(smem);
    const long long ntiles = (lo + L - 1) / L;
    const int tid = threadIdx.x;
    const int a1 = tid / L, l1 = tid - a1 * L;  // round 1: outer index a1, column l1
    constexpr int N1 = p3(K1) * L;
    W pre[p3(K2)];
    auto fetch = [&](long long t) {
      const long long c = t * L + l1;
      if (tid < N1 && c < lo) {
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) pre[j] = src[(long long)(a1 * p3(K2) + j) * lo + c];
      }
    };
    long long t = blockIdx.x;
    if (t < ntiles) fetch(t);
#pragma unroll 1
    for (; t < ntiles; t += gridDim.x) {
      const long long l0 = t * L;
      if (tid < N1 && l0 + l1 < lo) {
        W v[p3(K2)];
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) v[j] = pre[j];
        interp_pencil<M, K2>(v);
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) T[(a1 * p3(K2) + j) * L + l1] = v[j];
      }
      __syncthreads();
      if (t + gridDim.x < ntiles) fetch(t + gridDim.x);
      {  // round 2: inner index r = tid / L, column l = tid % L (all p3(K2) * L threads)
        const int r = tid / L, l = tid - r * L;
        long long zc;
        if (zcol(l0 + l, zc)) {
          W v[p3(K1)];
#pragma unroll
          for (int j = 0; j < p3(K1); ++j) v[j] = T[(j * p3(K2) + r) * L + l];
          interp_pencil<M, K1>(v);
#pragma unroll
          for (int j = 0; j < p3(K1); ++j)
            dst[(long long)(j * p3(K2) + r) * lo_z + zc] = M::out(v[j]);
        }
      }
      __syncthreads();  // T is rewritten by the next tile's round 1
    }
  }
}

template <class M, int K1, int K2, int L>
inline cudaError_t launch_remap_kl(const typename M::W* src, typename M::Out* dst, long long lo,
                                   long long pitch, long long cn, cudaStream_t st) {
  auto k = interp_remap_kernel<M, K1, K2, L>;
  ProfileScope prof(st, "interp_remap");
  constexpr size_t smem = K1 > 0 ? sizeof(typename M::W) * (size_t)p3(K1 + K2) * L : 0;
  cudaError_t e = prep_kernel(k, smem);
  if (e != cudaSuccess) return e;
  constexpr int threads = K1 > 0 ? p3(K2) * L : 256;
  const long long work = K1 > 0 ? (lo + L - 1) / L : (lo + 255) / 256;
  k<<<grid_for(k, threads, smem, work), threads, smem, st>>>(src, dst, lo, pitch, cn);
  return cudaGetLastError();
}

// The padded schedule's last pass over k = 1..6 outermost axes; cols: 16 or
// 32 columns per tile (the sign of a 16-byte-copy width is ignored).
template <class M>
inline cudaError_t launch_interp_remap(int k, int cols, const typename M::W* src,
                                       typename M::Out* dst, long long lo, long long pitch,
                                       long long cn, cudaStream_t st) {
  const bool wide = (cols < 0 ? -cols : cols) >= 32;
  switch (k) {
    case 1: return launch_remap_kl<M, 0, 1, 256>(src, dst, lo, pitch, cn, st);
    case 2: return launch_remap_kl<M, 0, 2, 256>(src, dst, lo, pitch, cn, st);
    case 3: return launch_remap_kl<M, 0, 3, 256>(src, dst, lo, pitch, cn, st);
    case 4:
      return wide ? launch_remap_kl<M, 1, 3, 32>(src, dst, lo, pitch, cn, st)
                  : launch_remap_kl<M, 1, 3, 16>(src, dst, lo, pitch, cn, st);
    case 5:
      return wide ? launch_remap_kl<M, 2, 3, 32>(src, dst, lo, pitch, cn, st)
                  : launch_remap_kl<M, 2, 3, 16>(src, dst, lo, pitch, cn, st);
    case 6:
      return wide ? launch_remap_kl<M, 3, 3, 32>(src, dst, lo, pitch, cn, st)
                  : launch_remap_kl<M, 3, 3, 16>(src, dst, lo, pitch, cn, st);
  }
  return cudaErrorInvalidValue;
}

// Interpolation (TR = false) or its transpose (TR = true) of k consecutive
// axes of a [hi][3^k][lo] array, src -> dst (may be the same array).
template <class M, bool FINAL, bool TR = false>
inline cudaError_t launch_interp(int k, int cols, const typename M::W* src, void* dst,
                                 long long hi, long long lo, cudaStream_t st) {
  if (cols == 0) cols = default_cols<M>();
  switch (k) {
    case 1: return launch_interp_k<M, 0, 1, FINAL, TR>(cols, src, dst, hi, lo, st);
    case 2: return launch_interp_k<M, 0, 2, FINAL, TR>(cols, src, dst, hi, lo, st);
    case 3: return launch_interp_k<M, 0, 3, FINAL, TR>(cols, src, dst, hi, lo, st);
    // K2 = 3: round 1 over 27-element pencils of the inner axes.  The
    // balanced splits (2, 2) and (3, 2) -- fewer threads, every thread busy
    // in both rounds -- measured slower here on GB300 (D = 18 float32 passes
    // 1.57 -> 1.61 ms, D = 18 int64 2.38 -> 2.50 ms, adjoint I^T 1.50 ->
    // 1.65 ms) and faster for the batched group passes, which use them.
    case 4: return launch_interp_k<M, 1, 3, FINAL, TR>(cols, src, dst, hi, lo, st);
    case 5: return launch_interp_k<M, 2, 3, FINAL, TR>(cols, src, dst, hi, lo, st);
    case 6: return launch_interp_k<M, 3, 3, FINAL, TR>(cols, src, dst, hi, lo, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hc
