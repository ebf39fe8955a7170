// Tile bodies shared by the plain kernels (one launch per pass) and the
// persistent batched kernel.
#pragma once

#include <type_traits>

#include "hc_common.cuh"

namespace hc {

// Asynchronous global -> shared copies (cp.async, sm_80+), 4 or 8 bytes.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <bool CG, class T>
__device__ __forceinline__ T ldw(const T* p) {
  if constexpr (CG) {
    if constexpr (sizeof(T) == 8) {
      unsigned long long v = __ldcg(reinterpret_cast<const unsigned long long*>(p));
      T r;
      memcpy(&r, &v, 8);
      return r;
    } else {
      unsigned int v = __ldcg(reinterpret_cast<const unsigned int*>(p));
      T r;
      memcpy(&r, &v, 4);
      return r;
    }
  } else {
    return *p;
  }
}

// L2 eviction priority of a global access (createpolicy, .L2::cache_hint).
// kPolNone: a plain access.  kPolKeep (evict_last): data that other CTAs of
// the same launch read back soon, e.g. a chunk's tiles before its column
// tickets; kept in L2 ahead of other lines.  kPolStream (evict_first): data
// the launch does not touch again, e.g. a chunk's finished columns; the
// first to leave L2, so they do not push out the lines still in use.
enum : int { kPolNone = 0, kPolKeep = 1, kPolStream = 2 };

template <int POL>
__device__ __forceinline__ unsigned long long l2_policy() {
  unsigned long long p = 0;
  if constexpr (POL == kPolKeep)
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  else if constexpr (POL == kPolStream)
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// *p = v with the L2 priority POL (p: global memory).
template <int POL, class T>
__device__ __forceinline__ void st_pol(T* p, const T& v) {
  if constexpr (POL == kPolNone) {
    *p = v;
  } else {
    static_assert(sizeof(T) == 8 || sizeof(T) == 4, "4- or 8-byte elements");
    const unsigned long long pol = l2_policy<POL>();
    if constexpr (sizeof(T) == 8) {
      unsigned long long b;
      memcpy(&b, &v, 8);
      asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"(b), "l"(pol)
                   : "memory");
    } else {
      unsigned b;
      memcpy(&b, &v, 4);
      asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(b), "l"(pol)
                   : "memory");
    }
  }
}

// cp.async of 4 or 8 bytes with the L2 priority POL on the global read.
template <int BYTES, int POL>
__device__ __forceinline__ void cp_async_pol(void* smem, const void* gmem) {
  if constexpr (POL == kPolNone) {
    cp_async<BYTES>(smem, gmem);
  } else {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const unsigned long long pol = l2_policy<POL>();
    if constexpr (BYTES == 8)
      asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;\n" ::"r"(s),
                   "l"(gmem), "l"(pol)
                   : "memory");
    else
      asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2;\n" ::"r"(s),
                   "l"(gmem), "l"(pol)
                   : "memory");
  }
}

// A load through L2 only (as ldw<true>) with the L2 priority POL.
template <int POL, class T>
__device__ __forceinline__ T ld_cg_pol(const T* p) {
  if constexpr (POL == kPolNone) {
    return ldw<true>(p);
  } else {
    const unsigned long long pol = l2_policy<POL>();
    T r;
    if constexpr (sizeof(T) == 8) {
      unsigned long long b;
      asm volatile("ld.global.cg.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(b) : "l"(p), "l"(pol));
      memcpy(&r, &b, 8);
    } else {
      unsigned b;
      asm volatile("ld.global.cg.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(b) : "l"(p), "l"(pol));
      memcpy(&r, &b, 4);
    }
    return r;
  }
}

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

// Row stride (elements) of a transposed [2^gL][n] buffer written by stage 1:
// the smallest stride >= n whose byte size is 16 modulo 32, so that the
// stage's writes (8 consecutive lanes on 8 rows) fall in distinct banks.
constexpr int padded_rows(int n, int elem_bytes) {
  return (n * elem_bytes) % 32 == 16 ? n : padded_rows(n + 1, elem_bytes);
}

template <class M, int C>
struct TileSmem {
  typedef typename M::In In;
  typedef typename M::W W;
  // W tile; the stage-0 buffer of a 3-group tile lives inside it.
  static constexpr size_t kW = sizeof(W) * (size_t)p3(C);
  // transposed buffer feeding the fused stage, per operand: [2^gL][LP]
  static constexpr int LP = TileShape<C>::G == 3
                                ? padded_rows(TileShape<C>::nLastPencils, (int)sizeof(In))
                                : TileShape<C>::nLastPencils;
  static constexpr size_t kLast = sizeof(In) * (size_t)p2(TileShape<C>::gL) * LP;
  // stage-0 output [operand][3^g0][S1R]: rows padded so that the stage-1
  // reads of two neighbouring rows fall in different banks
  static constexpr int S1R = p2(C - TileShape<C>::g0) + (p2(C - TileShape<C>::g0) % 16 == 0 ? 8 : 0);
  static constexpr size_t kS1 = TileShape<C>::G == 3 ? 2 * sizeof(In) * (size_t)p3(TileShape<C>::g0) * S1R : 0;
  static_assert(kS1 <= kW, "stage-0 buffer must fit inside the W tile");
  // With at most 256 fused pencils (one per thread of a 256-thread CTA) the
  // fused stage reads all its inputs before any thread writes W, so the
  // stage buffers live inside the W tile too: [S1 | LastX | LastY | ...].
  static constexpr bool kAlias =
      TileShape<C>::G >= 2 && TileShape<C>::nLastPencils <= 256 && kS1 + 2 * kLast <= kW;
  static constexpr size_t kLastOff = kAlias ? kS1 : kW;
  static constexpr size_t bytes = kAlias ? kW : kW + (TileShape<C>::G >= 2 ? 2 * kLast : 0);
};

// Loader of a tile whose two operand rows are plain arrays (global or shared).
template <class In>
struct RowLoader {
  const In* x;
  const In* y;
  __device__ __forceinline__ In operator()(int op, int i) const { return op ? y[i] : x[i]; }
};

// Shared memory of a tile kernel whose input rows come from a double buffer
// that cp.async fills with the next tile's rows while the current tile is
// being computed: the tile's own smem, then [buffer][operand][2^C] rows.
template <class M, int C>
struct TileRows {
  static constexpr size_t kOff = (TileSmem<M, C>::bytes + 15) / 16 * 16;
  static constexpr size_t bytes = kOff + 2 * 2 * sizeof(typename M::In) * (size_t)p2(C);
};

// Bulk (TMA engine) shared -> global store of `bytes` bytes; both addresses
// 16-byte aligned, bytes a multiple of 16.  One thread issues it; the shared
// source must have been fenced for the async proxy (fence.proxy.async).
__device__ __forceinline__ void bulk_store(void* gmem, const void* smem, unsigned bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gmem), "r"(s),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// Wait until at most N of this thread's bulk groups are still reading their
// shared source (READ) or still in flight at all.
template <int N, bool READ>
__device__ __forceinline__ void bulk_wait() {
  if constexpr (READ)
    asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
  else
    asm volatile("cp.async.bulk.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared memory of the tile kernel that stores its tiles with bulk copies:
// two W tiles (tile t computes in buffer t & 1 while the copy of tile t - 1
// drains the other), each with 16 spare bytes so the tile can be placed at
// its output's address modulo 16, then the [buffer][operand][2^C] rows.
template <class M, int C>
struct TileBulk {
  static constexpr size_t kWB = (TileSmem<M, C>::bytes + 15) / 16 * 16 + 16;
  static constexpr size_t kOff = 2 * kWB;
  static constexpr size_t bytes = kOff + 2 * 2 * sizeof(typename M::In) * (size_t)p2(C);
};

// Loader: ld(op, i) returns element i of the tile's operand row (op 0 = x,
// 1 = y), already evaluated on the outer axes.  out_tile: the tile's 3^C
// outputs.  smem: TileSmem<M, C>::bytes of shared memory.
template <class M>
inline size_t tile_smem_bytes_m(int C) {
  switch (C) {
    case 1: return TileSmem<M, 1>::bytes;
    case 2: return TileSmem<M, 2>::bytes;
    case 3: return TileSmem<M, 3>::bytes;
    case 4: return TileSmem<M, 4>::bytes;
    case 5: return TileSmem<M, 5>::bytes;
    case 6: return TileSmem<M, 6>::bytes;
    case 7: return TileSmem<M, 7>::bytes;
    case 8: return TileSmem<M, 8>::bytes;
    case 9: return TileSmem<M, 9>::bytes;
  }
  return 0;
}

// Shared memory of tile_body for a dtype and tile size C.
inline size_t tile_smem_bytes(hc_dtype dt, int C) {
  switch (dt) {
    case HC_INT64: return tile_smem_bytes_m<ModeI64>(C);
    case HC_FP64: return tile_smem_bytes_m<ModeF64>(C);
    case HC_FP32: return tile_smem_bytes_m<ModeF32>(C);
    case HC_FP32_MIXED: return tile_smem_bytes_m<ModeMixed>(C);
    case HC_FP32_FF: return tile_smem_bytes_m<ModeFF>(C);
  }
  return 0;
}

// The stages of a tile of G >= 2 groups, one pencil per call (tile_body and
// the pipelined bulk loop run them; see tile_body for the order).  smem: the
// tile's TileSmem<M, C>::bytes.
template <class M, int C>
struct TileStages {
  typedef typename M::In In;
  typedef typename M::W W;
  typedef typename M::Out Out;
  typedef TileShape<C> S;
  static constexpr int G = S::G;
  static constexpr int LP = TileSmem<M, C>::LP;  // row stride of LastX, LastY
  static constexpr int kStage0 = 2 * p2(C - S::g0);   // stage-0 pencils
  static constexpr int kInterp0 = p3(C - S::g0);      // last-stage pencils
  static __device__ __forceinline__ In* last_x(unsigned char* smem) {
    return reinterpret_cast<In*>(smem + TileSmem<M, C>::kLastOff);
  }

  // stage 0, pencil p: evaluate group 0 (g0 axes) from the operand rows
  template <class Loader>
  static __device__ __forceinline__ void stage0(const Loader& ld, unsigned char* smem, int p) {
    constexpr int R = p2(C - S::g0);  // pencils per operand
    const int op = p / R, r = p - op * R;
    In v[p3(S::g0)];
#pragma unroll
    for (int b = 0; b < p2(S::g0); ++b) v[b] = ld(op, b * R + r);
    eval_pencil<M, S::g0>(v);
    if constexpr (S::G == 2) {
      // next is the fused stage: transposed [2^gL][3^g0], r = last-group bits
      In* d = last_x(smem) + op * (p2(S::gL) * LP);
#pragma unroll
      for (int j = 0; j < p3(S::g0); ++j) d[r * p3(S::g0) + j] = v[j];
    } else {
      constexpr int S1R = TileSmem<M, C>::S1R;
      In* d = reinterpret_cast<In*>(smem) + op * (p3(S::g0) * S1R);  // S1 aliases the W tile
#pragma unroll
      for (int j = 0; j < p3(S::g0); ++j) d[j * S1R + r] = v[j];
    }
  }

  // stage 1 (G == 3): evaluate group 1 (3 axes) in shared memory, all pencils
  static __device__ __forceinline__ void stage1(unsigned char* smem) {
    constexpr int O = p3(S::g0);
    constexpr int R = p2(S::gL);  // remaining binary axes (innermost group)
    constexpr int NP = O * R;
    constexpr int S1R = TileSmem<M, C>::S1R;  // = 8 * R + padding
    const In* S1 = reinterpret_cast<const In*>(smem);
    In* LastX = last_x(smem);
    In* LastY = LastX + p2(S::gL) * LP;
#pragma unroll 1
    for (int p = threadIdx.x; p < 2 * NP; p += blockDim.x) {
      const int op = p / NP, q = p - op * NP;
      const int o = q / R, r = q - o * R;
      const In* s = S1 + op * (O * S1R);
      In v[27];
#pragma unroll
      for (int b = 0; b < 8; ++b) v[b] = s[o * S1R + b * R + r];
      eval_pencil<M, 3>(v);
      In* d = op ? LastY : LastX;
#pragma unroll
      for (int j = 0; j < 27; ++j) d[r * LP + o * 27 + j] = v[j];
    }
  }

  // fused stage: evaluate the innermost group, multiply, interpolate it.
  // With the stage buffers inside the W tile (kAlias) every thread reads its
  // one pencil's inputs, a barrier follows, then W is written.
  static __device__ __forceinline__ void fused(unsigned char* smem) {
    constexpr int NO = S::nLastPencils;
    W* Ws = reinterpret_cast<W*>(smem);
    const In* LastX = last_x(smem);
    const In* LastY = LastX + p2(S::gL) * LP;
    if constexpr (TileSmem<M, C>::kAlias) {
      const int o = threadIdx.x;
      In a[27], b[27];
      if (o < NO) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          a[q] = LastX[q * LP + o];
          b[q] = LastY[q * LP + o];
        }
      }
      __syncthreads();
      if (o < NO) {
        eval_pencil<M, 3>(a);
        eval_pencil<M, 3>(b);
        W w[27];
#pragma unroll
        for (int j = 0; j < 27; ++j) w[j] = M::mul(a[j], b[j]);
        interp_pencil<M, 3>(w);
#pragma unroll
        for (int j = 0; j < 27; ++j) Ws[o * 27 + j] = w[j];
      }
    } else {
#pragma unroll 1
      for (int o = threadIdx.x; o < NO; o += blockDim.x) {
        In a[27], b[27];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          a[q] = LastX[q * LP + o];
          b[q] = LastY[q * LP + o];
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
  }

  // interpolate group 1 (G == 3) in shared memory, all pencils.  The group-0
  // digit o runs fastest across threads: lanes then never straddle two
  // 27-element runs of one o, whose banks would overlap.
  static __device__ __forceinline__ void interp1(unsigned char* smem) {
    constexpr int O = p3(S::g0), R = 27;
    W* Ws = reinterpret_cast<W*>(smem);
#pragma unroll 1
    for (int p = threadIdx.x; p < O * R; p += blockDim.x) {
      const int r = p / O, o = p - r * O;
      W v[27];
#pragma unroll
      for (int j = 0; j < 27; ++j) v[j] = Ws[(o * 27 + j) * R + r];
      interp_pencil<M, 3>(v);
#pragma unroll
      for (int j = 0; j < 27; ++j) Ws[(o * 27 + j) * R + r] = v[j];
    }
  }

  // last stage, pencil r: interpolate group 0 and write the outputs to
  // out_tile (global), or back into the W tile (SMEM_OUT)
  template <bool FINAL, bool SMEM_OUT, int POL = kPolNone>
  static __device__ __forceinline__ void interp0(void* __restrict__ out_tile, unsigned char* smem,
                                                 int r) {
    constexpr int R = p3(C - S::g0);
    W* Ws = reinterpret_cast<W*>(smem);
    W v[p3(S::g0)];
#pragma unroll
    for (int j = 0; j < p3(S::g0); ++j) v[j] = Ws[j * R + r];
    interp_pencil<M, S::g0>(v);
    if constexpr (SMEM_OUT) {
#pragma unroll
      for (int j = 0; j < p3(S::g0); ++j) Ws[j * R + r] = v[j];
    } else if constexpr (FINAL) {
      Out* o = reinterpret_cast<Out*>(out_tile);
#pragma unroll
      for (int j = 0; j < p3(S::g0); ++j) st_pol<POL>(o + j * R + r, M::out(v[j]));
    } else {
      W* o = reinterpret_cast<W*>(out_tile);
#pragma unroll
      for (int j = 0; j < p3(S::g0); ++j) st_pol<POL>(o + j * R + r, v[j]);
    }
  }
};

// The stages of a tile of C = 8 axes of 4-byte values split into two groups
// of four instead of 2 + 3 + 3: stage 0 evaluates the outer four axes of
// each operand row (16 -> 81 values per pencil) into a transposed
// [operand][2^4][81] buffer at the start of the W tile, the fused stage
// evaluates the inner four axes of both operands, multiplies and
// interpolates the inner four (81-value pencils), and the last stage
// interpolates the outer four.  The data pass through shared memory three
// times instead of five; every element sees the same operations in the same
// order (evaluation outer axes first, interpolation inner axes first).  One
// pencil per thread in the fused stage (at least 81 threads).  Every index
// pattern is conflict-free: 81 = 17 mod 32 words between the rows that
// neighbouring threads write.
template <class M>
struct TileStages44 {
  typedef typename M::In In;
  typedef typename M::W W;
  typedef typename M::Out Out;
  static_assert(sizeof(In) == 4 && sizeof(W) == 4, "four-axis pencils hold 4-byte values");
  static constexpr int G = 2;
  static constexpr int kStage0 = 2 * 16;  // pencils of stage 0, both operands
  static constexpr int kFused = 81;       // pencils of the fused stage
  static constexpr int kInterp0 = 81;     // pencils of the last stage
  static constexpr int LP = 81;           // row stride of the stage-0 output
  static_assert(2 * 16 * LP <= p3(8), "the stage-0 output fits inside the W tile");

  template <class Loader>
  static __device__ __forceinline__ void stage0(const Loader& ld, unsigned char* smem, int p) {
    const int op = p >> 4, r = p & 15;  // r: the inner group's four bits
    In v[81];
#pragma unroll
    for (int b = 0; b < 16; ++b) v[b] = ld(op, b * 16 + r);
    eval_pencil<M, 4>(v);
    In* d = reinterpret_cast<In*>(smem) + op * (16 * LP);
#pragma unroll
    for (int j = 0; j < 81; ++j) d[r * LP + j] = v[j];
  }

  // every thread reads its pencil's inputs, a barrier follows (the inputs
  // live inside the W tile), then the pencil's 81 outputs are written
  static __device__ __forceinline__ void fused(unsigned char* smem) {
    W* Ws = reinterpret_cast<W*>(smem);
    const In* LastX = reinterpret_cast<const In*>(smem);
    const In* LastY = LastX + 16 * LP;
    const int o = threadIdx.x;  // the outer group's digits
    In a[81], b[81];
    if (o < kFused) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        a[q] = LastX[q * LP + o];
        b[q] = LastY[q * LP + o];
      }
    }
    __syncthreads();
    if (o < kFused) {
      eval_pencil<M, 4>(a);
      eval_pencil<M, 4>(b);
      W w[81];
#pragma unroll
      for (int j = 0; j < 81; ++j) w[j] = M::mul(a[j], b[j]);
      interp_pencil<M, 4>(w);
#pragma unroll
      for (int j = 0; j < 81; ++j) Ws[o * 81 + j] = w[j];
    }
  }

  // last stage, pencil r (the inner group's digits): interpolate the outer
  // four axes; to out_tile (global) or back into the W tile (SMEM_OUT)
  template <bool FINAL, bool SMEM_OUT, int POL = kPolNone>
  static __device__ __forceinline__ void interp0(void* __restrict__ out_tile, unsigned char* smem,
                                                 int r) {
    W* Ws = reinterpret_cast<W*>(smem);
    W v[81];
#pragma unroll
    for (int j = 0; j < 81; ++j) v[j] = Ws[j * 81 + r];
    interp_pencil<M, 4>(v);
    if constexpr (SMEM_OUT) {
#pragma unroll
      for (int j = 0; j < 81; ++j) Ws[j * 81 + r] = v[j];
    } else if constexpr (FINAL) {
      Out* o = reinterpret_cast<Out*>(out_tile);
#pragma unroll
      for (int j = 0; j < 81; ++j) st_pol<POL>(o + j * 81 + r, M::out(v[j]));
    } else {
      W* o = reinterpret_cast<W*>(out_tile);
#pragma unroll
      for (int j = 0; j < 81; ++j) st_pol<POL>(o + j * 81 + r, v[j]);
    }
  }
};

// Whether the bulk-store tile loops of (M, C) use the two four-axis groups:
// C = 8 binary32 tiles (register pencils of 81 values, 127 registers, no
// spills), launched with 128 threads.  Measured on GB300 against the
// 2 + 3 + 3 split (same bits): D = 18 float32 tile 0.392 -> 0.325 ms, the
// 4096-instance float32 batch's tiles 3.44 -> 2.90 ms.
template <class M, int C>
constexpr bool use_tile44() {
  return C == 8 && std::is_same<M, ModeF32>::value;
}

// SMEM_OUT (intermediate tiles only, FINAL false): the last stage writes the
// finished tile back into the W tile in shared memory (in place, each thread
// its own pencils; out_tile unused) and fences it for the async proxy, so
// that the caller can store it with one bulk copy.
// POL: L2 priority of the tile's global stores.
template <class M, int C, bool FINAL, class Loader, bool SMEM_OUT = false, int POL = kPolNone>
__device__ __forceinline__ void tile_body(const Loader& ld, void* __restrict__ out_tile,
                                          unsigned char* smem) {
  typedef typename M::In In;
  typedef typename M::W W;
  typedef typename M::Out Out;
  typedef TileShape<C> S;
  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  if constexpr (S::G == 1) {
    // C <= 3: one pencil, straight from global to global.
    if (tid == 0) {
      In a[p3(C)], b[p3(C)];
#pragma unroll
      for (int i = 0; i < p2(C); ++i) {
        a[i] = ld(0, i);
        b[i] = ld(1, i);
      }
      eval_pencil<M, C>(a);
      eval_pencil<M, C>(b);
      W w[p3(C)];
#pragma unroll
      for (int j = 0; j < p3(C); ++j) w[j] = M::mul(a[j], b[j]);
      interp_pencil<M, C>(w);
      if constexpr (FINAL) {
        Out* o = reinterpret_cast<Out*>(out_tile);
#pragma unroll
        for (int j = 0; j < p3(C); ++j) st_pol<POL>(o + j, M::out(w[j]));
      } else {
        W* o = reinterpret_cast<W*>(out_tile);
#pragma unroll
        for (int j = 0; j < p3(C); ++j) st_pol<POL>(o + j, w[j]);
      }
    }
  } else {
    typedef TileStages<M, C> St;
#pragma unroll 1
    for (int p = tid; p < St::kStage0; p += nt) St::stage0(ld, smem, p);
    __syncthreads();
    if constexpr (S::G == 3) {
      St::stage1(smem);
      __syncthreads();
    }
    St::fused(smem);
    __syncthreads();
    if constexpr (S::G == 3) {
      St::interp1(smem);
      __syncthreads();
    }
#pragma unroll 1
    for (int r = tid; r < St::kInterp0; r += nt)
      St::template interp0<FINAL, SMEM_OUT, POL>(out_tile, smem, r);
    if constexpr (SMEM_OUT) {
      static_assert(!FINAL, "bulk tile stores write the intermediate W");
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();  // the caller's next tile reuses shared memory
  }
}

// Tile loop whose intermediate tiles are stored with bulk copies: each
// finished tile is written back into shared memory and stored by the TMA
// engine with one bulk copy, which drains while the CTA computes the next
// tile in the other W buffer (the per-thread stores of the last stage
// otherwise bunch up the tile's whole output at its end).  The W buffer is
// placed at the output's address modulo 16, so that shared and global
// addresses agree in their low bits; the elements before the output's first
// 16-byte boundary and after its last are stored by threads.  The tiles are
// pipelined one stage deep: the next tile's stage 0 (from its rows,
// prefetched with cp.async) runs in the other W buffer in the same barrier
// interval as this tile's last stage, which fills the threads stage 0 leaves
// idle and saves two barriers per tile.  src(t, op): tile t's operand row
// (op 0 = x, 1 = y), 2^C elements; out(t): tile t's 3^C outputs, in a plain
// device allocation.  smem: TileBulk<M, C>::bytes.  Tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...
template <class M, int C, class SrcFn, class OutFn, class St = TileStages<M, C>>
__device__ __forceinline__ void tile_loop_bulk(SrcFn src, OutFn out, long long ntiles,
                                               unsigned char* smem) {
  typedef typename M::In In;
  typedef typename M::W W;
  static_assert(St::G >= 2, "bulk tiles: C >= 4");
  typedef TileBulk<M, C> B;
  constexpr int N = p3(C);
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long step = gridDim.x;
  In* rows = reinterpret_cast<In*>(smem + B::kOff);  // [buffer][operand][2^C]
  auto prefetch = [&](long long t, int b) {
#pragma unroll 1
    for (int e = tid; e < 2 * p2(C); e += nt) {
      const int op = e >> C, i = e & (p2(C) - 1);
      cp_async<sizeof(In)>(rows + (b * 2 + op) * p2(C) + i, src(t, op) + i);
    }
    cp_async_commit();
  };
  // tile t's W tile in buffer b, at its output's address modulo 16
  auto wtile = [&](long long t, int b) {
    return smem + b * B::kWB + (unsigned)(reinterpret_cast<uintptr_t>(out(t)) & 15);
  };
  long long t = blockIdx.x;
  if (t >= ntiles) return;
  prefetch(t, 0);
  if (t + step < ntiles) {
    prefetch(t + step, 1);
    cp_async_wait<1>();
  } else {
    cp_async_wait<0>();
  }
  __syncthreads();  // the first tile's rows are in buffer 0
  {
    RowLoader<In> ld{rows, rows + p2(C)};
    unsigned char* w0 = wtile(t, 0);
#pragma unroll 1
    for (int p = tid; p < St::kStage0; p += nt) St::stage0(ld, w0, p);
  }
  __syncthreads();
  int b = 0;
#pragma unroll 1
  for (; t < ntiles; t += step, b ^= 1) {
    unsigned char* w = wtile(t, b);
    const long long tn = t + step;
    const bool next = tn < ntiles;
    if constexpr (St::G == 3) {
      St::stage1(w);
      __syncthreads();
    }
    St::fused(w);
    if constexpr (St::G == 3) {
      __syncthreads();
      St::interp1(w);
    }
    // before the barrier that opens the last stage: the next tile's rows have
    // landed, and the copy of tile t - step has read the other W buffer
    if (next) cp_async_wait<0>();
    if (tid == 0) bulk_wait<0, true>();
    __syncthreads();
    // last stage of tile t and stage 0 of tile tn, one barrier interval
    {
      RowLoader<In> ld{rows + ((b ^ 1) * 2) * p2(C), rows + ((b ^ 1) * 2 + 1) * p2(C)};
      unsigned char* wn = next ? wtile(tn, b ^ 1) : nullptr;
      const int items = St::kInterp0 + (next ? St::kStage0 : 0);
#pragma unroll 1
      for (int p = tid; p < items; p += nt) {
        if (p < St::kInterp0)
          St::template interp0<false, true>(nullptr, w, p);
        else
          St::stage0(ld, wn, p - St::kInterp0);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    // tile t is in w[0, N): head / body / tail split at 16-byte boundaries
    W* out_tile = out(t);
    const unsigned mis = (unsigned)(reinterpret_cast<uintptr_t>(out_tile) & 15);
    const int head = mis ? (int)((16 - mis) / sizeof(W)) : 0;
    const int body = (int)(((N - head) * sizeof(W)) / 16 * 16 / sizeof(W));
    const W* ws = reinterpret_cast<const W*>(w);
    if (tid == 0 && body > 0) bulk_store(out_tile + head, ws + head, (unsigned)(body * sizeof(W)));
    for (int e = tid; e < head; e += nt) out_tile[e] = ws[e];
    for (int e = head + body + tid; e < N; e += nt) out_tile[e] = ws[e];
    // rows buffer b was consumed by this tile's stage 0, one iteration ago
    if (tn + step < ntiles) prefetch(tn + step, b);
  }
  if (tid == 0) bulk_wait<0, false>();
}

// ---------------------------------------------------------------------------
// K3: interpolate k = K1 + K2 consecutive axes of a [hi][3^k][lo] array.
// A CTA tile is all 3^k rows of L consecutive columns of one h.  Round 1
// interpolates the inner K2 axes in registers (pencils read straight from
// global memory, stride lo), round 2 the outer K1 axes after a pass through
// shared memory.  Consecutive threads take consecutive columns.  src and dst
// may be the same array (in place) -- every tile reads all its elements
// before writing any, and tiles are disjoint.
// One tile: rows base + j * lo for j < 3^k, columns l0 + [0, L) clipped to
// lo (base already includes l0).  CG = read src through L2 only (data
// written by other CTAs of the same launch).
// TR: the transposed map I^T (outer K1 axes first, then the inner K2 axes,
// each pencil transformed outermost axis first) -- the adjoint's pass.
// LPOL / SPOL (non-transposed, K1 > 0): L2 priorities of the global loads
// (CG only) and of the stores.
template <class M, int K1, int K2, int L, bool FINAL, bool CG, bool TR = false,
          int LPOL = kPolNone, int SPOL = kPolNone>
__device__ __forceinline__ void interp_tile_body(const typename M::W* src, void* dst_,
                                                 long long base, long long l0, long long lo,
                                                 unsigned char* smem) {
  typedef typename M::W W;
  typedef typename M::Out Out;
  W* T = reinterpret_cast<W*>(smem);
  const int tid = threadIdx.x, nt = blockDim.x;
  {
    if constexpr (K1 == 0) {
#pragma unroll 1
      for (int l = tid; l < L; l += nt) {
        if (l0 + l >= lo) continue;
        W v[p3(K2)];
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) v[j] = ldw<CG>(src + base + j * lo + l);
        if constexpr (TR)
          interp_t_pencil<M, K2>(v);
        else
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
    } else if constexpr (TR) {
      // round 1: outer K1 axes (I^T), global -> registers -> shared
#pragma unroll 1
      for (int p = tid; p < p3(K2) * L; p += nt) {
        const int r = p / L, l = p - r * L;
        if (l0 + l >= lo) continue;
        W v[p3(K1)];
#pragma unroll
        for (int j = 0; j < p3(K1); ++j)
          v[j] = ldw<CG>(src + base + (long long)(j * p3(K2) + r) * lo + l);
        interp_t_pencil<M, K1>(v);
#pragma unroll
        for (int j = 0; j < p3(K1); ++j) T[(j * p3(K2) + r) * L + l] = v[j];
      }
      __syncthreads();
      // round 2: inner K2 axes (I^T), shared -> registers -> global
#pragma unroll 1
      for (int p = tid; p < p3(K1) * L; p += nt) {
        const int o = p / L, l = p - o * L;
        if (l0 + l >= lo) continue;
        W v[p3(K2)];
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) v[j] = T[(o * p3(K2) + j) * L + l];
        interp_t_pencil<M, K2>(v);
        W* d = reinterpret_cast<W*>(dst_);
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) d[base + (long long)(o * p3(K2) + j) * lo + l] = v[j];
      }
      __syncthreads();
    } else {
      // round 1: inner K2 axes, global -> registers -> shared
      #pragma unroll 1
      for (int p = tid; p < p3(K1) * L; p += nt) {
        const int o = p / L, l = p - o * L;
        if (l0 + l >= lo) continue;
        W v[p3(K2)];
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) {
          const W* a = src + base + (long long)(o * p3(K2) + j) * lo + l;
          if constexpr (CG)
            v[j] = ld_cg_pol<LPOL>(a);
          else
            v[j] = *a;
        }
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
            st_pol<SPOL>(d + base + (long long)(j * p3(K2) + r) * lo + l, M::out(v[j]));
        } else {
          W* d = reinterpret_cast<W*>(dst_);
#pragma unroll
          for (int j = 0; j < p3(K1); ++j)
            st_pol<SPOL>(d + base + (long long)(j * p3(K2) + r) * lo + l, v[j]);
        }
      }
      __syncthreads();  // shared tile reused by the caller's next tile
    }
  }
}

// Per-tile array pointers for the multi-tile interpolation loops: by default
// every tile uses the loop's src / dst; a PtrFn `ptrs(i, src, dst)` gives
// tile i its own arrays (the grouped batched form: one array per instance).
struct NoPtrs {};

// Pipelined interpolation of k = K1 + K2 axes (K1 > 0) over a sequence of
// column tiles.  Tile i is rows base_i + j * lo (j < 3^k), columns
// l0_i + [0, L) clipped to lo.  Its elements are copied into shared buffer
// i % 2 with cp.async while tile i - 1 is being interpolated; round 1
// interpolates the inner K2 axes in place in shared memory, round 2 the outer
// K1 axes from shared memory to dst.  smem: 2 * 3^k * L W elements.
// `tile(i, base, l0)` yields the position of tile i; n tiles in all.
// LPOL / SPOL: L2 priorities of the element copies in and of the stores out.
template <class M, int K1, int K2, int L, bool FINAL, class TileFn, bool TR = false,
          class PtrFn = NoPtrs, int LPOL = kPolNone, int SPOL = kPolNone>
__device__ __forceinline__ void interp_tiles_pipelined(const typename M::W* src0, void* dst0,
                                                       long long lo, int n, const TileFn& tile,
                                                       unsigned char* smem,
                                                       const PtrFn& ptrs = PtrFn()) {
  typedef typename M::W W;
  typedef typename M::Out Out;
  constexpr int ROWS = p3(K1 + K2);
  constexpr int NE = ROWS * L;
  W* buf0 = reinterpret_cast<W*>(smem);
  W* buf1 = buf0 + NE;
  const int tid = threadIdx.x, nt = blockDim.x;
  auto arrays = [&](int i, const W*& s, void*& d) {
    if constexpr (std::is_same<PtrFn, NoPtrs>::value) {
      s = src0;
      d = dst0;
    } else {
      ptrs(i, s, d);
    }
  };
  auto prefetch = [&](int i, W* b) {
    long long base, l0;
    tile(i, base, l0);
    const W* src;
    void* dd;
    arrays(i, src, dd);
#pragma unroll 1
    for (int e = tid; e < NE; e += nt) {
      const int row = e / L, l = e - row * L;
      if (l0 + l < lo) cp_async_pol<sizeof(W), LPOL>(b + e, src + base + (long long)row * lo + l);
    }
    cp_async_commit();
  };
  if (n > 0) prefetch(0, buf0);
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    W* b = (i & 1) ? buf1 : buf0;
    if (i + 1 < n) {
      prefetch(i + 1, (i & 1) ? buf0 : buf1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // tile i's elements are in b
    long long base, l0;
    tile(i, base, l0);
    const W* src_i;
    void* dst_;
    arrays(i, src_i, dst_);
    if constexpr (TR) {
      // I^T: round 1 the outer K1 axes in place, round 2 the inner K2 axes
#pragma unroll 1
      for (int p = tid; p < p3(K2) * L; p += nt) {
        const int r = p / L, l = p - r * L;
        if (l0 + l >= lo) continue;
        W v[p3(K1)];
#pragma unroll
        for (int j = 0; j < p3(K1); ++j) v[j] = b[(j * p3(K2) + r) * L + l];
        interp_t_pencil<M, K1>(v);
#pragma unroll
        for (int j = 0; j < p3(K1); ++j) b[(j * p3(K2) + r) * L + l] = v[j];
      }
      __syncthreads();
#pragma unroll 1
      for (int p = tid; p < p3(K1) * L; p += nt) {
        const int o = p / L, l = p - o * L;
        if (l0 + l >= lo) continue;
        W v[p3(K2)];
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) v[j] = b[(o * p3(K2) + j) * L + l];
        interp_t_pencil<M, K2>(v);
        W* d = reinterpret_cast<W*>(dst_);
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) d[base + (long long)(o * p3(K2) + j) * lo + l] = v[j];
      }
      __syncthreads();
    } else {
    // round 1: inner K2 axes, in place
#pragma unroll 1
    for (int p = tid; p < p3(K1) * L; p += nt) {
      const int o = p / L, l = p - o * L;
      if (l0 + l >= lo) continue;
      W v[p3(K2)];
#pragma unroll
      for (int j = 0; j < p3(K2); ++j) v[j] = b[(o * p3(K2) + j) * L + l];
      interp_pencil<M, K2>(v);
#pragma unroll
      for (int j = 0; j < p3(K2); ++j) b[(o * p3(K2) + j) * L + l] = v[j];
    }
    __syncthreads();
    // round 2: outer K1 axes, shared -> global
#pragma unroll 1
    for (int p = tid; p < p3(K2) * L; p += nt) {
      const int r = p / L, l = p - r * L;
      if (l0 + l >= lo) continue;
      W v[p3(K1)];
#pragma unroll
      for (int j = 0; j < p3(K1); ++j) v[j] = b[(j * p3(K2) + r) * L + l];
      interp_pencil<M, K1>(v);
      if constexpr (FINAL) {
        Out* d = reinterpret_cast<Out*>(dst_);
#pragma unroll
        for (int j = 0; j < p3(K1); ++j)
          st_pol<SPOL>(d + base + (long long)(j * p3(K2) + r) * lo + l, M::out(v[j]));
      } else {
        W* d = reinterpret_cast<W*>(dst_);
#pragma unroll
        for (int j = 0; j < p3(K1); ++j)
          st_pol<SPOL>(d + base + (long long)(j * p3(K2) + r) * lo + l, v[j]);
      }
    }
    __syncthreads();  // b is refilled two tiles later
    }
  }
}

// Interpolation of k = K1 + K2 axes (K1 > 0) over a sequence of column
// tiles with a register prefetch: each thread owns one round-1 pencil per
// tile and loads the next tile's pencil into registers right after the
// barrier that ends round 1, so those loads are in flight while round 2 of
// the current tile runs (one smem buffer of 3^k * L elements; the register
// copy doubles the bytes in flight without a second buffer).  Same
// arithmetic and per-element order as interp_tile_body; src may equal dst
// (tiles are disjoint, and a tile's elements are loaded before any of them
// is stored).  Needs blockDim.x >= 3^max(K1,K2) * L.
template <class M, int K1, int K2, int L, bool FINAL, class TileFn, bool TR = false,
          class PtrFn = NoPtrs>
__device__ __forceinline__ void interp_tiles_regpipe(const typename M::W* src0, void* dst0,
                                                     long long lo, int n, const TileFn& tile,
                                                     unsigned char* smem,
                                                     const PtrFn& ptrs = PtrFn()) {
  typedef typename M::W W;
  typedef typename M::Out Out;
  constexpr int P1 = TR ? p3(K1) : p3(K2);        // round-1 pencil length
  constexpr int N1 = (TR ? p3(K2) : p3(K1)) * L;  // round-1 pencils
  constexpr int P2 = TR ? p3(K2) : p3(K1);        // round-2 pencil length
  constexpr int N2 = (TR ? p3(K1) : p3(K2)) * L;  // round-2 pencils
  W* T = reinterpret_cast<W*>(smem);
  const int tid = threadIdx.x;
  // round-1 pencil of this thread: a1 = outer index o (I) or inner index r (I^T)
  const int a1 = tid / L, l1 = tid - a1 * L;
  const int a2 = tid / L, l2 = tid - a2 * L;
  auto row1 = [&](int j) { return TR ? j * p3(K2) + a1 : a1 * p3(K2) + j; };
  auto row2 = [&](int j) { return TR ? a2 * p3(K2) + j : j * p3(K2) + a2; };
  auto arrays = [&](int i, const W*& s, void*& d) {
    if constexpr (std::is_same<PtrFn, NoPtrs>::value) {
      s = src0;
      d = dst0;
    } else {
      ptrs(i, s, d);
    }
  };
  W pre[P1];
  auto fetch = [&](int i) {
    long long base, l0;
    tile(i, base, l0);
    const W* src;
    void* dd;
    arrays(i, src, dd);
    if (tid < N1 && l0 + l1 < lo) {
#pragma unroll
      for (int j = 0; j < P1; ++j) pre[j] = src[base + (long long)row1(j) * lo + l1];
    }
  };
  if (n > 0) fetch(0);
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    long long base, l0;
    tile(i, base, l0);
    const W* src_i;
    void* dst_;
    arrays(i, src_i, dst_);
    if (tid < N1 && l0 + l1 < lo) {
      W v[P1];
#pragma unroll
      for (int j = 0; j < P1; ++j) v[j] = pre[j];
      if constexpr (TR)
        interp_t_pencil<M, K1>(v);
      else
        interp_pencil<M, K2>(v);
#pragma unroll
      for (int j = 0; j < P1; ++j) T[row1(j) * L + l1] = v[j];
    }
    __syncthreads();
    if (i + 1 < n) fetch(i + 1);
    if (tid < N2 && l0 + l2 < lo) {
      W v[P2];
#pragma unroll
      for (int j = 0; j < P2; ++j) v[j] = T[row2(j) * L + l2];
      if constexpr (TR)
        interp_t_pencil<M, K2>(v);
      else
        interp_pencil<M, K1>(v);
      if constexpr (FINAL && !TR) {
        Out* d = reinterpret_cast<Out*>(dst_);
#pragma unroll
        for (int j = 0; j < P2; ++j) d[base + (long long)row2(j) * lo + l2] = M::out(v[j]);
      } else {
        W* d = reinterpret_cast<W*>(dst_);
#pragma unroll
        for (int j = 0; j < P2; ++j) d[base + (long long)row2(j) * lo + l2] = v[j];
      }
    }
    __syncthreads();  // T is rewritten by the next tile's round 1
  }
}

// 16-byte asynchronous copy global -> shared of `bytes` (<= 16) bytes, the
// rest of the 16 zero-filled.  Both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes)
               : "memory");
}

// Tiles of k = K1 + K2 rows loaded with 16-byte copies: a row segment of L
// columns starts at element base + j * lo, which for an odd lo is generally
// not 16-byte aligned, so each row is widened to the enclosing aligned range
// (row stride RS = L + A - 1 rounded up to A = 16 / s elements) and indexed
// from its own offset (base + j * lo) mod A.  One copy instruction moves A
// elements: a quarter (4-byte) or half (8-byte) of the load instructions of
// the per-element copies, which bound the other loops.
template <class M, int K1, int K2, int L>
struct WideRows {
  typedef typename M::W W;
  static constexpr int A = 16 / (int)sizeof(W);
  static constexpr int RS = (L + A - 1 + A - 1) / A * A;
  static constexpr int NC = RS / A;  // 16-byte chunks per row
  static constexpr int ROWS = p3(K1 + K2);
  static constexpr size_t kBuf = sizeof(W) * (size_t)ROWS * RS;
  // two buffers when they fit in a CTA's shared memory
  static constexpr int NB = 2 * kBuf <= 220 * 1024 ? 2 : 1;
  static constexpr size_t kSmem = NB * kBuf;
};

// Same arithmetic and per-element order as interp_tile_body; src may equal
// dst.  N: elements of every source array (copies stop at its end).  NB = 2:
// tile i + 1 is copied while tile i is interpolated.
template <class M, int K1, int K2, int L, bool FINAL, class TileFn, bool TR = false,
          class PtrFn = NoPtrs>
__device__ __forceinline__ void interp_tiles_wide(const typename M::W* src0, void* dst0,
                                                  long long lo, long long N, int n,
                                                  const TileFn& tile, unsigned char* smem,
                                                  const PtrFn& ptrs = PtrFn()) {
  typedef typename M::W W;
  typedef typename M::Out Out;
  typedef WideRows<M, K1, K2, L> S;
  constexpr int A = S::A, RS = S::RS, NC = S::NC, ROWS = S::ROWS, NB = S::NB;
  constexpr int NE = ROWS * RS;
  W* buf0 = reinterpret_cast<W*>(smem);
  W* buf1 = buf0 + (NB == 2 ? NE : 0);
  const int tid = threadIdx.x, nt = blockDim.x;
  auto arrays = [&](int i, const W*& s, void*& d) {
    if constexpr (std::is_same<PtrFn, NoPtrs>::value) {
      s = src0;
      d = dst0;
    } else {
      ptrs(i, s, d);
    }
  };
  auto fill = [&](int i, W* b) {
    long long base, l0;
    tile(i, base, l0);
    const W* src;
    void* dd;
    arrays(i, src, dd);
#pragma unroll 1
    for (int e = tid; e < ROWS * NC; e += nt) {
      const int row = e / NC, q = e - row * NC;
      const long long c = ((base + (long long)row * lo) & ~(long long)(A - 1)) + (long long)q * A;
      if (c < N) {
        const long long left = N - c;
        cp_async16(b + row * RS + q * A, src + c,
                   (int)(left < A ? left * (long long)sizeof(W) : 16));
      }
    }
    cp_async_commit();
  };
  if constexpr (NB == 2) {
    if (n > 0) fill(0, buf0);
  }
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    W* b = (NB == 2 && (i & 1)) ? buf1 : buf0;
    if constexpr (NB == 2) {
      if (i + 1 < n) {
        fill(i + 1, (i & 1) ? buf0 : buf1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
    } else {
      fill(i, b);
      cp_async_wait<0>();
    }
    __syncthreads();  // tile i's rows are in b
    long long base, l0;
    tile(i, base, l0);
    const W* src_i;
    void* dst_;
    arrays(i, src_i, dst_);
    const int bm = (int)(base & (A - 1)), lm = (int)(lo & (A - 1));
    auto at = [&](int row, int col) -> W& {
      return b[row * RS + ((bm + row * lm) & (A - 1)) + col];
    };
    if constexpr (TR) {
      // I^T: round 1 the outer K1 axes in place, round 2 the inner K2 axes
#pragma unroll 1
      for (int p = tid; p < p3(K2) * L; p += nt) {
        const int r = p / L, l = p - r * L;
        if (l0 + l >= lo) continue;
        W v[p3(K1)];
#pragma unroll
        for (int j = 0; j < p3(K1); ++j) v[j] = at(j * p3(K2) + r, l);
        interp_t_pencil<M, K1>(v);
#pragma unroll
        for (int j = 0; j < p3(K1); ++j) at(j * p3(K2) + r, l) = v[j];
      }
      __syncthreads();
#pragma unroll 1
      for (int p = tid; p < p3(K1) * L; p += nt) {
        const int o = p / L, l = p - o * L;
        if (l0 + l >= lo) continue;
        W v[p3(K2)];
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) v[j] = at(o * p3(K2) + j, l);
        interp_t_pencil<M, K2>(v);
        W* d = reinterpret_cast<W*>(dst_);
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) d[base + (long long)(o * p3(K2) + j) * lo + l] = v[j];
      }
    } else {
      // round 1: inner K2 axes, in place
#pragma unroll 1
      for (int p = tid; p < p3(K1) * L; p += nt) {
        const int o = p / L, l = p - o * L;
        if (l0 + l >= lo) continue;
        W v[p3(K2)];
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) v[j] = at(o * p3(K2) + j, l);
        interp_pencil<M, K2>(v);
#pragma unroll
        for (int j = 0; j < p3(K2); ++j) at(o * p3(K2) + j, l) = v[j];
      }
      __syncthreads();
      // round 2: outer K1 axes, shared -> global
#pragma unroll 1
      for (int p = tid; p < p3(K2) * L; p += nt) {
        const int r = p / L, l = p - r * L;
        if (l0 + l >= lo) continue;
        W v[p3(K1)];
#pragma unroll
        for (int j = 0; j < p3(K1); ++j) v[j] = at(j * p3(K2) + r, l);
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
    }
    __syncthreads();  // b is refilled by a later tile
  }
}

}  // namespace hc
