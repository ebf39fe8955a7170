// Adjoint (differentiation form) of the hypercube convolution on sm_103a.
//
// z = I^{xD} (E^{xD} x (.) E^{xD} y) is bilinear, so for an upstream gradient
// dz:  dx = E^T^{xD} (G (.) E^{xD} y),  dy = E^T^{xD} (G (.) E^{xD} x),
// with G = I^T^{xD} dz and the per-axis transposes of the Methods-section maps
//   I^T: (g0, g1, g2) -> (g0 - g1, g1, g2 - g1)
//   E^T: (h0, h1, h2) -> (h0 + h1, h1 + h2).
// Differentiating the recurrence gives the same per-element order: I^T axis 1
// first, E^T axis D first (dx[0] = corr(g0 - g1, y0) + corr(g1, y0 + y1),
// dx[1] = corr(g2 - g1, y1) + corr(g1, y0 + y1)).
//
// Schedule (a = D - C outer axes, C inner axes per tile):
//   KB3 interp_t_pass : I^T on the outer axes, outer pass first, dz -> G
//   K1  eval_pass     : outer evaluation of x and y (as in the forward)
//   KB2 tile_adj      : per outer index: I^T on the C inner axes, products with
//                       the inner-evaluated operands (recomputed here, never
//                       stored), E^T on the C inner axes -> Hx, Hy [3^a][2^C]
//   KB1 evalt_pass    : E^T on the outer axes, inner pass first -> dx, dy
#include <cstring>
#include <type_traits>

#include "hc_common.cuh"
#include "hc_profile.cuh"
#include "hc_forward.cuh"
#include "hc_kernels.cuh"

namespace hc {

// ---------------------------------------------------------------------------
// KB1: E^T on K axes of [hi][3^K][lo] -> [hi][2^K][lo], for Hx and Hy at once.
template <class M, int K>
__global__ void __launch_bounds__(256) evalt_pass_kernel(const typename M::W* __restrict__ sx,
                                                         const typename M::W* __restrict__ sy,
                                                         typename M::W* __restrict__ dx,
                                                         typename M::W* __restrict__ dy,
                                                         long long hi, long long lo) {
  typedef typename M::W T;
  const T* src = blockIdx.y ? sy : sx;
  T* dst = blockIdx.y ? dy : dx;
  if (!src || !dst) return;
  const long long cols = hi * lo;
#pragma unroll 1
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < cols;
       c += (long long)gridDim.x * blockDim.x) {
    const long long h = c / lo, l = c - h * lo;
    T v[p3(K)];
    const T* s = src + (h * p3(K)) * lo + l;
#pragma unroll
    for (int j = 0; j < p3(K); ++j) v[j] = s[j * lo];
    eval_t_pencil<M, K>(v);
    T* d = dst + (h * p2(K)) * lo + l;
#pragma unroll
    for (int b = 0; b < p2(K); ++b) d[b * lo] = v[b];
  }
}

// ---------------------------------------------------------------------------
// KB2: the adjoint tile.  Groups as in the forward tile (outermost group g0,
// then groups of 3).  Stages:
//   eval 0/1  : inner evaluation of Xo[alpha], Yo[alpha] up to the innermost
//               group, into transposed buffers LastX, LastY (as the forward)
//   I^T 0     : G[alpha] pencils along group 0 from global memory -> Gs
//   I^T 1     : (3 groups) along group 1 in shared memory
//   fused     : I^T on the innermost group, evaluate the innermost group of
//               X and Y, multiply (hx = g * y_hat, hy = g * x_hat), E^T on the
//               innermost group -> Hs_x, Hs_y [3^(C-3)][2^3]
//   E^T 1     : (3 groups) along group 1 -> reuses the LastX/LastY space
//   E^T 0     : along group 0, straight to global Hx[alpha], Hy[alpha] (2^C)
template <int C>
struct AdjShape {
  static constexpr int G = (C + 2) / 3;
  static constexpr int g0 = C - 3 * (G - 1);
  static constexpr int gL = (G == 1) ? C : 3;
  static constexpr int NO = p3(C - gL);
};

template <class M, int C>
struct AdjSmem {
  typedef typename M::In In;
  typedef typename M::W W;
  typedef AdjShape<C> S;
  static constexpr size_t kG = sizeof(W) * (size_t)p3(C);
  // Row strides chosen against shared-memory bank conflicts: LP for the
  // transposed [2^gL][LP] operand and product buffers (stage-1 writes, E^T
  // group-1 reads), S1R for the stage-0 output rows (stage-1 reads), H1R for
  // the E^T group-1 output rows (its writes).
  static constexpr int LP = S::G == 3 ? padded_rows(S::NO, (int)sizeof(In)) : S::NO;
  static constexpr int S1R = p2(C - S::g0) + (p2(C - S::g0) % 16 == 0 ? 8 : 0);
  static constexpr int H1R = 72;
  static constexpr size_t kLast = sizeof(In) * (size_t)p2(S::gL) * LP;  // per operand
  static constexpr size_t kH = sizeof(W) * (size_t)p2(S::gL) * LP;      // per operand
  static constexpr size_t kS1 = S::G == 3 ? 2 * sizeof(In) * (size_t)p3(S::g0) * S1R : 0;
  static constexpr size_t kH1 = S::G == 3 ? sizeof(W) * (size_t)p3(S::g0) * H1R : 0;  // per operand
  static_assert(kS1 <= kG, "stage-0 buffer fits in the G tile");
  static_assert(kH1 <= kLast, "E^T group-1 output fits in the operand buffer");
  static constexpr size_t bytes = kG + 2 * kLast + 2 * kH;
};

// Pipelined form (PIPE): the next tile's operand rows and G tile are copied
// into shared memory with cp.async while the current tile is finished, so
// that no stage waits on global loads.  Shared memory
//   [Gs | LastX | LastY | Gpre | rows]:
// the fused stage reads all its inputs (one pencil per thread) before any
// thread writes, so Hs_x, Hs_y overwrite LastX, LastY, and the E^T group-1
// output moves into Gs (dead after the fused stage).  The G tile is copied in
// 16-byte pieces from the 16-byte boundary at or below its start and read
// from its offset there.  The copies for tile t + grid are issued once tile
// t has consumed its rows and its G tile (after I^T on group 0).
template <class M, int C>
struct AdjPipeSmem {
  typedef AdjSmem<M, C> A;
  static constexpr size_t kGs = (A::kG + 15) / 16 * 16;
  static constexpr size_t kLastOff = kGs;
  static constexpr size_t kPreOff = kLastOff + (2 * A::kLast + 15) / 16 * 16;
  static constexpr size_t kPre = kGs + 16;
  static constexpr size_t kRowsOff = kPreOff + kPre;
  static constexpr size_t bytes = kRowsOff + 2 * sizeof(typename M::In) * (size_t)p2(C);
  static_assert(A::kH <= A::kLast, "Hs overwrites the operand buffers");
  static_assert(2 * A::kH1 <= A::kG, "E^T group-1 output fits in Gs");
};

template <class M, int C, bool PIPE>
__global__ void __launch_bounds__(256) tile_adj_kernel(const typename M::W* __restrict__ Gsrc,
                                                       const typename M::In* __restrict__ X,
                                                       const typename M::In* __restrict__ Y,
                                                       typename M::W* __restrict__ Hx,
                                                       typename M::W* __restrict__ Hy,
                                                       long long ntiles) {
  typedef typename M::In In;
  typedef typename M::W W;
  typedef AdjShape<C> S;
  typedef AdjSmem<M, C> SM;
  typedef AdjPipeSmem<M, C> PS;
  static_assert(!PIPE || S::G >= 2, "pipelined adjoint tiles: C >= 4");
  extern __shared__ __align__(16) unsigned char smem[];
  W* Gs = reinterpret_cast<W*>(smem);
  In* S1 = reinterpret_cast<In*>(smem);  // G == 3: aliases Gs (dead before Gs is written)
  In* LastX = reinterpret_cast<In*>(smem + (PIPE ? PS::kLastOff : SM::kG));
  In* LastY = reinterpret_cast<In*>(smem + (PIPE ? PS::kLastOff : SM::kG) + SM::kLast);
  W* HsX = PIPE ? reinterpret_cast<W*>(LastX) : reinterpret_cast<W*>(smem + SM::kG + 2 * SM::kLast);
  W* HsY = PIPE ? reinterpret_cast<W*>(LastY)
                : reinterpret_cast<W*>(smem + SM::kG + 2 * SM::kLast + SM::kH);
  // G == 3: E^T group-1 output
  W* H1X = PIPE ? Gs : reinterpret_cast<W*>(LastX);
  W* H1Y = PIPE ? reinterpret_cast<W*>(smem + SM::kH1) : reinterpret_cast<W*>(LastY);
  unsigned char* Gpre = smem + PS::kPreOff;
  In* rows = reinterpret_cast<In*>(smem + PS::kRowsOff);  // [operand][2^C]
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool want_x = Hx != nullptr, want_y = Hy != nullptr;
  const char* gend = reinterpret_cast<const char*>(Gsrc + ntiles * p3(C));
  auto prefetch = [&](long long t) {
#pragma unroll 1
    for (int e = tid; e < 2 * p2(C); e += nt) {
      const int op = e >> C, i = e & (p2(C) - 1);
      cp_async<sizeof(In)>(rows + op * p2(C) + i, (op ? Y : X) + t * p2(C) + i);
    }
    const char* ga = reinterpret_cast<const char*>(Gsrc + t * p3(C));
    const unsigned mis = (unsigned)(reinterpret_cast<uintptr_t>(ga) & 15);
    const char* g0 = ga - mis;
    const int nch = (int)((mis + sizeof(W) * (size_t)p3(C) + 15) / 16);
#pragma unroll 1
    for (int c = tid; c < nch; c += nt) {
      const char* src = g0 + 16 * (size_t)c;
      const long long rem = gend - src;
      cp_async16(Gpre + 16 * c, src, rem < 16 ? (int)rem : 16);
    }
    cp_async_commit();
  };
  if constexpr (PIPE) {
    if ((long long)blockIdx.x < ntiles) prefetch(blockIdx.x);
  }

#pragma unroll 1
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    if constexpr (PIPE) {
      cp_async_wait<0>();
      __syncthreads();  // this tile's rows and G tile are in shared memory
    }
    const In* xr = PIPE ? rows : X + t * p2(C);
    const In* yr = PIPE ? rows + p2(C) : Y + t * p2(C);
    const W* gr = Gsrc + t * p3(C);
    if constexpr (PIPE)
      gr = reinterpret_cast<const W*>(Gpre + (reinterpret_cast<uintptr_t>(gr) & 15));
    if constexpr (S::G == 1) {
      if (tid == 0) {
        W g[p3(C)];
        In a[p3(C)], b[p3(C)];
#pragma unroll
        for (int j = 0; j < p3(C); ++j) g[j] = gr[j];
#pragma unroll
        for (int i = 0; i < p2(C); ++i) {
          a[i] = xr[i];
          b[i] = yr[i];
        }
        interp_t_pencil<M, C>(g);
        eval_pencil<M, C>(a);
        eval_pencil<M, C>(b);
        W hx[p3(C)], hy[p3(C)];
#pragma unroll
        for (int j = 0; j < p3(C); ++j) {
          hx[j] = M::mulw(g[j], b[j]);
          hy[j] = M::mulw(g[j], a[j]);
        }
        eval_t_pencil<M, C>(hx);
        eval_t_pencil<M, C>(hy);
#pragma unroll
        for (int i = 0; i < p2(C); ++i) {
          if (want_x) Hx[t * p2(C) + i] = hx[i];
          if (want_y) Hy[t * p2(C) + i] = hy[i];
        }
      }
    } else {
      // ---- eval stage 0 (operands)
      {
        constexpr int R = p2(C - S::g0);
#pragma unroll 1
        for (int p = tid; p < 2 * R; p += nt) {
          const int op = p / R, r = p - op * R;
          const In* src = op ? yr : xr;
          In v[p3(S::g0)];
#pragma unroll
          for (int b = 0; b < p2(S::g0); ++b) v[b] = src[b * R + r];
          eval_pencil<M, S::g0>(v);
          if constexpr (S::G == 2) {
            In* d = op ? LastY : LastX;
#pragma unroll
            for (int j = 0; j < p3(S::g0); ++j) d[r * p3(S::g0) + j] = v[j];
          } else {
            In* d = S1 + op * (p3(S::g0) * SM::S1R);
#pragma unroll
            for (int j = 0; j < p3(S::g0); ++j) d[j * SM::S1R + r] = v[j];
          }
        }
      }
      __syncthreads();
      if constexpr (S::G == 3) {
        constexpr int O = p3(S::g0);
        constexpr int R = 8;
        constexpr int NP = O * R;
#pragma unroll 1
        for (int p = tid; p < 2 * NP; p += nt) {
          const int op = p / NP, q = p - op * NP;
          const int o = q / R, r = q - o * R;
          const In* s = S1 + op * (O * SM::S1R);
          In v[27];
#pragma unroll
          for (int b = 0; b < 8; ++b) v[b] = s[o * SM::S1R + b * R + r];
          eval_pencil<M, 3>(v);
          In* d = op ? LastY : LastX;
#pragma unroll
          for (int j = 0; j < 27; ++j) d[r * SM::LP + o * 27 + j] = v[j];
        }
        __syncthreads();
      }
      // ---- I^T on group 0, global -> Gs
      {
        constexpr int R = p3(C - S::g0);
#pragma unroll 1
        for (int r = tid; r < R; r += nt) {
          W v[p3(S::g0)];
#pragma unroll
          for (int j = 0; j < p3(S::g0); ++j) v[j] = gr[j * R + r];
          interp_t_pencil<M, S::g0>(v);
#pragma unroll
          for (int j = 0; j < p3(S::g0); ++j) Gs[j * R + r] = v[j];
        }
      }
      __syncthreads();
      if constexpr (PIPE) {
        // rows and Gpre are consumed: start the copies of the next tile
        if (t + gridDim.x < ntiles) prefetch(t + gridDim.x);
      }
      // ---- I^T on group 1 (3 groups)
      if constexpr (S::G == 3) {
        // the group-0 digit o runs fastest across threads (no bank overlap
        // between two 27-element runs within a warp)
        constexpr int O = p3(S::g0), R = 27;
#pragma unroll 1
        for (int p = tid; p < O * R; p += nt) {
          const int r = p / O, o = p - r * O;
          W v[27];
#pragma unroll
          for (int j = 0; j < 27; ++j) v[j] = Gs[(o * 27 + j) * R + r];
          interp_t_pencil<M, 3>(v);
#pragma unroll
          for (int j = 0; j < 27; ++j) Gs[(o * 27 + j) * R + r] = v[j];
        }
        __syncthreads();
      }
      // ---- fused: I^T innermost group, products, E^T innermost group
      if constexpr (PIPE) {
        // one pencil per thread (NO <= blockDim.x); all reads, then all writes
        constexpr int NO = S::NO;
        const int o = tid;
        W g[27];
        In ay[8], ax[8];
        if (o < NO) {
#pragma unroll
          for (int j = 0; j < 27; ++j) g[j] = Gs[o * 27 + j];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            ay[q] = LastY[q * SM::LP + o];
            ax[q] = LastX[q * SM::LP + o];
          }
        }
        __syncthreads();
        if (o < NO) {
          interp_t_pencil<M, 3>(g);
          if (want_x) {
            In a[27];
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = ay[q];
            eval_pencil<M, 3>(a);
            W h[27];
#pragma unroll
            for (int j = 0; j < 27; ++j) h[j] = M::mulw(g[j], a[j]);
            eval_t_pencil<M, 3>(h);
#pragma unroll
            for (int b = 0; b < 8; ++b) HsX[b * SM::LP + o] = h[b];
          }
          if (want_y) {
            In a[27];
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = ax[q];
            eval_pencil<M, 3>(a);
            W h[27];
#pragma unroll
            for (int j = 0; j < 27; ++j) h[j] = M::mulw(g[j], a[j]);
            eval_t_pencil<M, 3>(h);
#pragma unroll
            for (int b = 0; b < 8; ++b) HsY[b * SM::LP + o] = h[b];
          }
        }
      } else {
        constexpr int NO = S::NO;
#pragma unroll 1
        for (int o = tid; o < NO; o += nt) {
          W g[27];
#pragma unroll
          for (int j = 0; j < 27; ++j) g[j] = Gs[o * 27 + j];
          interp_t_pencil<M, 3>(g);
          In a[27];
          if (want_x) {
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = LastY[q * SM::LP + o];
            eval_pencil<M, 3>(a);
            W h[27];
#pragma unroll
            for (int j = 0; j < 27; ++j) h[j] = M::mulw(g[j], a[j]);
            eval_t_pencil<M, 3>(h);
#pragma unroll
            for (int b = 0; b < 8; ++b) HsX[b * SM::LP + o] = h[b];
          }
          if (want_y) {
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = LastX[q * SM::LP + o];
            eval_pencil<M, 3>(a);
            W h[27];
#pragma unroll
            for (int j = 0; j < 27; ++j) h[j] = M::mulw(g[j], a[j]);
            eval_t_pencil<M, 3>(h);
#pragma unroll
            for (int b = 0; b < 8; ++b) HsY[b * SM::LP + o] = h[b];
          }
        }
      }
      __syncthreads();
      // Hs layout: [2^3 innermost bits][3^(C-3) outer digits] (transposed).
      if constexpr (S::G == 3) {
        // ---- E^T on group 1: Hs [8][O][27] -> H1 [O][8][8] (o, b1, b2)
        constexpr int O = p3(S::g0), NO = S::NO;
#pragma unroll 1
        for (int p = tid; p < 2 * O * 8; p += nt) {
          const int op = p / (O * 8), q = p - op * (O * 8);
          const int o = q / 8, b2 = q - o * 8;
          if (op == 0 ? !want_x : !want_y) continue;
          const W* s = op ? HsY : HsX;
          W v[27];
#pragma unroll
          for (int j = 0; j < 27; ++j) v[j] = s[b2 * SM::LP + o * 27 + j];
          eval_t_pencil<M, 3>(v);
          W* d = op ? H1Y : H1X;
#pragma unroll
          for (int b1 = 0; b1 < 8; ++b1) d[o * SM::H1R + b1 * 8 + b2] = v[b1];
        }
        __syncthreads();
        // ---- E^T on group 0 -> global, element (b0, b1, b2) at b0 * 64 + b1 * 8 + b2
        constexpr int R = 64;
#pragma unroll 1
        for (int p = tid; p < 2 * R; p += nt) {
          const int op = p / R, r = p - op * R;
          if (op == 0 ? !want_x : !want_y) continue;
          const W* s = op ? H1Y : H1X;
          W v[p3(S::g0)];
#pragma unroll
          for (int j = 0; j < p3(S::g0); ++j) v[j] = s[j * SM::H1R + r];
          eval_t_pencil<M, S::g0>(v);
          W* d = (op ? Hy : Hx) + t * p2(C);
#pragma unroll
          for (int b = 0; b < p2(S::g0); ++b) d[b * R + r] = v[b];
        }
      } else {
        // ---- E^T on group 0 (2 groups): Hs [8][3^g0] -> global [2^g0][8]
        constexpr int NO = S::NO, R = 8;
#pragma unroll 1
        for (int p = tid; p < 2 * R; p += nt) {
          const int op = p / R, r = p - op * R;
          if (op == 0 ? !want_x : !want_y) continue;
          const W* s = op ? HsY : HsX;
          W v[p3(S::g0)];
#pragma unroll
          for (int j = 0; j < p3(S::g0); ++j) v[j] = s[r * NO + j];
          eval_t_pencil<M, S::g0>(v);
          W* d = (op ? Hy : Hx) + t * p2(C);
#pragma unroll
          for (int b = 0; b < p2(S::g0); ++b) d[b * R + r] = v[b];
        }
      }
      __syncthreads();
    }
  }
}

// The adjoint tile of C = 8 axes of 4-byte values in two groups of four
// (the forward's TileStages44 split): per tile
//   eval 0   : the outer four axes of both operand rows (16 -> 81 values per
//              pencil) -> transposed [2^4][81] buffers
//   I^T 0    : the G tile's outer four axes, global (prefetched) -> Gs
//   fused    : I^T on the inner four axes (81-value pencil of G), the inner
//              four axes of y and of x evaluated, the products, E^T on the
//              inner four -> Hs [2^4][81] per output
//   E^T 0    : the outer four axes -> global Hx, Hy (2^8 each)
// Every element sees the operations of the 2 + 3 + 3 tile in the same order
// (I^T and evaluation outer axes first, E^T inner axes first).  The next
// tile's rows and G tile are copied with cp.async while the current one is
// finished (as the pipelined form); the fused stage reads its inputs, a
// barrier follows, then Hs overwrites the operand buffers.  128 threads,
// 214 registers, no spills (two CTAs per SM).
template <class M>
struct Adj44Smem {
  static constexpr size_t kG = 4 * (size_t)p3(8);                  // Gs
  static constexpr size_t kGs = (kG + 15) / 16 * 16;
  static constexpr size_t kLastOff = kGs;                           // LastX, LastY / HsX, HsY
  static constexpr size_t kLast = 4 * (size_t)16 * 81;              // per operand
  static constexpr size_t kPreOff = kLastOff + (2 * kLast + 15) / 16 * 16;
  static constexpr size_t kPre = kGs + 16;                          // next G tile
  static constexpr size_t kRowsOff = kPreOff + kPre;                // [operand][2^8]
  static constexpr size_t bytes = kRowsOff + 2 * 4 * (size_t)p2(8);
};

template <class M>
__global__ void __launch_bounds__(128) tile_adj44_kernel(const typename M::W* __restrict__ Gsrc,
                                                         const typename M::In* __restrict__ X,
                                                         const typename M::In* __restrict__ Y,
                                                         typename M::W* __restrict__ Hx,
                                                         typename M::W* __restrict__ Hy,
                                                         long long ntiles) {
  typedef typename M::In In;
  typedef typename M::W W;
  static_assert(sizeof(In) == 4 && sizeof(W) == 4, "four-axis pencils hold 4-byte values");
  typedef Adj44Smem<M> PS;
  constexpr int C = 8, N3 = p3(8), N2 = p2(8);
  extern __shared__ __align__(16) unsigned char smem[];
  W* Gs = reinterpret_cast<W*>(smem);
  In* LastX = reinterpret_cast<In*>(smem + PS::kLastOff);
  In* LastY = LastX + 16 * 81;
  W* HsX = reinterpret_cast<W*>(LastX);
  W* HsY = reinterpret_cast<W*>(LastY);
  unsigned char* Gpre = smem + PS::kPreOff;
  In* rows = reinterpret_cast<In*>(smem + PS::kRowsOff);
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool want_x = Hx != nullptr, want_y = Hy != nullptr;
  const char* gend = reinterpret_cast<const char*>(Gsrc + ntiles * N3);
  auto prefetch = [&](long long t) {
#pragma unroll 1
    for (int e = tid; e < 2 * N2; e += nt) {
      const int op = e >> C, i = e & (N2 - 1);
      cp_async<sizeof(In)>(rows + op * N2 + i, (op ? Y : X) + t * N2 + i);
    }
    const char* ga = reinterpret_cast<const char*>(Gsrc + t * N3);
    const unsigned mis = (unsigned)(reinterpret_cast<uintptr_t>(ga) & 15);
    const char* g0 = ga - mis;
    const int nch = (int)((mis + sizeof(W) * (size_t)N3 + 15) / 16);
#pragma unroll 1
    for (int c = tid; c < nch; c += nt) {
      const char* src = g0 + 16 * (size_t)c;
      const long long rem = gend - src;
      cp_async16(Gpre + 16 * c, src, rem < 16 ? (int)rem : 16);
    }
    cp_async_commit();
  };
  if ((long long)blockIdx.x < ntiles) prefetch(blockIdx.x);
#pragma unroll 1
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    cp_async_wait<0>();
    __syncthreads();  // this tile's rows and G tile are in shared memory
    const W* gr = reinterpret_cast<const W*>(
        Gpre + (reinterpret_cast<uintptr_t>(Gsrc + t * N3) & 15));
    // ---- eval 0 (operands) and I^T 0 (G), one barrier interval
#pragma unroll 1
    for (int p = tid; p < 32 + 81; p += nt) {
      if (p < 32) {
        const int op = p >> 4, r = p & 15;
        const In* src = rows + op * N2;
        In v[81];
#pragma unroll
        for (int b = 0; b < 16; ++b) v[b] = src[b * 16 + r];
        eval_pencil<M, 4>(v);
        In* d = op ? LastY : LastX;
#pragma unroll
        for (int j = 0; j < 81; ++j) d[r * 81 + j] = v[j];
      } else {
        const int r = p - 32;  // the inner group's digits
        W v[81];
#pragma unroll
        for (int j = 0; j < 81; ++j) v[j] = gr[j * 81 + r];
        interp_t_pencil<M, 4>(v);
#pragma unroll
        for (int j = 0; j < 81; ++j) Gs[j * 81 + r] = v[j];
      }
    }
    __syncthreads();
    // rows and the prefetched G tile are consumed: start the next tile's copies
    if (t + gridDim.x < ntiles) prefetch(t + gridDim.x);
    // ---- fused: one pencil (outer digits o) per thread; all reads, then writes
    {
      const int o = tid;
      W g[81];
      In ay[16], ax[16];
      if (o < 81) {
#pragma unroll
        for (int j = 0; j < 81; ++j) g[j] = Gs[o * 81 + j];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          ay[q] = LastY[q * 81 + o];
          ax[q] = LastX[q * 81 + o];
        }
      }
      __syncthreads();
      if (o < 81) {
        interp_t_pencil<M, 4>(g);
        if (want_x) {
          W a[81];
#pragma unroll
          for (int q = 0; q < 16; ++q) a[q] = ay[q];
          eval_pencil<M, 4>(a);
#pragma unroll
          for (int j = 0; j < 81; ++j) a[j] = M::mulw(g[j], a[j]);
          eval_t_pencil<M, 4>(a);
#pragma unroll
          for (int b = 0; b < 16; ++b) HsX[b * 81 + o] = a[b];
        }
        if (want_y) {
          W a[81];
#pragma unroll
          for (int q = 0; q < 16; ++q) a[q] = ax[q];
          eval_pencil<M, 4>(a);
#pragma unroll
          for (int j = 0; j < 81; ++j) a[j] = M::mulw(g[j], a[j]);
          eval_t_pencil<M, 4>(a);
#pragma unroll
          for (int b = 0; b < 16; ++b) HsY[b * 81 + o] = a[b];
        }
      }
    }
    __syncthreads();
    // ---- E^T 0 -> global: element (outer bits b, inner bits r) at b * 16 + r
#pragma unroll 1
    for (int p = tid; p < 32; p += nt) {
      const int op = p >> 4, r = p & 15;
      if (op == 0 ? !want_x : !want_y) continue;
      const W* s = op ? HsY : HsX;
      W v[81];
#pragma unroll
      for (int j = 0; j < 81; ++j) v[j] = s[r * 81 + j];
      eval_t_pencil<M, 4>(v);
      W* d = (op ? Hy : Hx) + t * N2;
#pragma unroll
      for (int b = 0; b < 16; ++b) d[b * 16 + r] = v[b];
    }
    __syncthreads();  // Hs (the operand buffers) and Gs are rewritten by the next tile
  }
}

template <class M>
__global__ void scalar_adj_kernel(const typename M::W* g, const typename M::In* x,
                                  const typename M::In* y, typename M::W* dx,
                                  typename M::W* dy) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (dx) dx[0] = M::mulw(g[0], y[0]);
    if (dy) dy[0] = M::mulw(g[0], x[0]);
  }
}

// ---------------------------------------------------------------------------
// Host side.

struct BwdPlan {
  int D, C, a;
  hc_dtype dtype;
  int n_eval;
  int eval_d0[HC_MAX_D], eval_k[HC_MAX_D];
  bool eval_to_final[HC_MAX_D];
  int n_it;  // I^T passes, outer first
  int it_d0[HC_MAX_D], it_k[HC_MAX_D];
  int n_et;  // E^T passes, inner first
  int et_d0[HC_MAX_D], et_k[HC_MAX_D];
  bool et_to_h[HC_MAX_D];
  size_t off_xo, off_yo, off_tx, off_ty, off_g, off_hx, off_hy, off_ex, off_ey;
  size_t ws_bytes;
};

static BwdPlan make_bwd_plan(int D, hc_dtype dt) {
  BwdPlan p;
  memset(&p, 0, sizeof(p));
  p.D = D;
  p.dtype = dt;
  int C = 8;
  if (C > D) C = D;
  p.C = C;
  p.a = D - C;
  const size_t es = elem_size(dt);
  for (int d = 0; d < p.a; d += 3) {
    const int k = (p.a - d) < 3 ? (p.a - d) : 3;
    p.eval_d0[p.n_eval] = d;
    p.eval_k[p.n_eval] = k;
    ++p.n_eval;
  }
  size_t xo = p.a > 0 ? pow3z(p.a) << C : 0, tmax = 0;
  for (int i = 0; i < p.n_eval; ++i) {
    const int done = p.eval_d0[i] + p.eval_k[i];
    const bool to_final = ((p.n_eval - 1 - i) % 2) == 0;
    p.eval_to_final[i] = to_final;
    const size_t n = pow3z(done) << (D - done);
    if (!to_final && n > tmax) tmax = n;
  }
  // I^T passes over the outer axes, outer first, balanced groups of <= 6.
  if (p.a > 0) {
    const int np = (p.a + 5) / 6;
    int start = 0;
    for (int i = 0; i < np; ++i) {
      const int rem = np - i;
      const int k = (p.a - start + rem - 1) / rem;
      p.it_d0[i] = start;
      p.it_k[i] = k;
      start += k;
    }
    p.n_it = np;
  }
  // E^T passes over the outer axes, inner first, <= 3 per pass.  Pass i
  // reads [3^(d0+k)][2^(a-d0-k) * 2^C] and writes [3^d0][2^(a-d0) * 2^C];
  // the last lands in dx/dy, earlier ones alternate H and E buffers.
  size_t emax = 0;
  {
    int end = p.a;
    while (end > 0) {
      const int k = end < 3 ? end : 3;
      p.et_d0[p.n_et] = end - k;
      p.et_k[p.n_et] = k;
      ++p.n_et;
      end -= k;
    }
    for (int i = 0; i < p.n_et; ++i) {
      const int d0 = p.et_d0[i];
      const bool last = i == p.n_et - 1;
      // pass 0 reads H, so non-final outputs alternate E, H, E, ...
      const bool to_h = !last && (i % 2 == 1);
      p.et_to_h[i] = to_h;
      const size_t n = pow3z(d0) << (D - d0);
      if (!last && !to_h && n > emax) emax = n;
    }
  }
  size_t off = kWsHeader;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  p.off_xo = take(xo * es);
  p.off_yo = take(xo * es);
  p.off_tx = take(tmax * es);
  p.off_ty = take(tmax * es);
  p.off_g = take(p.a > 0 ? pow3z(D) * es : 0);
  p.off_hx = take(p.a > 0 ? xo * es : 0);
  p.off_hy = take(p.a > 0 ? xo * es : 0);
  p.off_ex = take(emax * es);
  p.off_ey = take(emax * es);
  p.ws_bytes = off;
  return p;
}

template <class M, int K>
static cudaError_t launch_et_k(const typename M::W* sx, const typename M::W* sy,
                               typename M::W* dx, typename M::W* dy, long long hi, long long lo,
                               cudaStream_t st) {
  const long long cols = hi * lo;
  long long blocks = (cols + 255) / 256;
  const long long cap = (long long)device_caps().sms * 8;
  if (blocks > cap) blocks = cap;
  ProfileScope prof(st, "evalt_pass");
  evalt_pass_kernel<M, K><<<dim3((unsigned)blocks, 2), 256, 0, st>>>(sx, sy, dx, dy, hi, lo);
  return cudaGetLastError();
}

template <class M>
static cudaError_t launch_et(int K, const typename M::W* sx, const typename M::W* sy,
                             typename M::W* dx, typename M::W* dy, long long hi, long long lo,
                             cudaStream_t st) {
  switch (K) {
    case 1: return launch_et_k<M, 1>(sx, sy, dx, dy, hi, lo, st);
    case 2: return launch_et_k<M, 2>(sx, sy, dx, dy, hi, lo, st);
    case 3: return launch_et_k<M, 3>(sx, sy, dx, dy, hi, lo, st);
  }
  return cudaErrorInvalidValue;
}

constexpr int adj_threads(int C) { return C >= 6 ? 256 : (C >= 4 ? 128 : 32); }

// The pipelined form where it keeps as many resident CTAs per SM as the
// plain one (its extra shared memory and registers may cost occupancy).
template <class M, int C>
static bool use_pipe_adj() {
  static int choice = -1;  // per instantiation; every thread computes the same value
  if (choice < 0) {
    int pipe = 0, plain = 0;
    const int threads = adj_threads(C);
    if (prep_kernel(tile_adj_kernel<M, C, true>, AdjPipeSmem<M, C>::bytes) != cudaSuccess ||
        prep_kernel(tile_adj_kernel<M, C, false>, AdjSmem<M, C>::bytes) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pipe, tile_adj_kernel<M, C, true>, threads,
                                                      AdjPipeSmem<M, C>::bytes) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&plain, tile_adj_kernel<M, C, false>, threads,
                                                      AdjSmem<M, C>::bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    choice = pipe >= plain && pipe > 0 ? 1 : 0;
  }
  return choice == 1;
}

template <class M, int C>
static cudaError_t launch_adj_c(const typename M::W* G, const typename M::In* X,
                                const typename M::In* Y, typename M::W* Hx, typename M::W* Hy,
                                long long ntiles, cudaStream_t st) {
  ProfileScope prof(st, "tile_adj");
  const int threads = adj_threads(C);
  // binary32, C = 8: the four-axis tile (GB300, D = 18: 0.632 -> 0.605 ms)
  if constexpr (C == 8 && std::is_same<M, ModeF32>::value) {
    if ((reinterpret_cast<uintptr_t>(G) & 15) == 0) {
      const size_t smem = Adj44Smem<M>::bytes;
      auto k = tile_adj44_kernel<M>;
      cudaError_t e = prep_kernel(k, smem);
      if (e != cudaSuccess) return e;
      k<<<grid_for(k, 128, smem, ntiles), 128, smem, st>>>(G, X, Y, Hx, Hy, ntiles);
      return cudaGetLastError();
    }
  }
  if constexpr (AdjShape<C>::G >= 2) {
    if ((reinterpret_cast<uintptr_t>(G) & 15) == 0 && use_pipe_adj<M, C>()) {
      const size_t smem = AdjPipeSmem<M, C>::bytes;
      auto k = tile_adj_kernel<M, C, true>;
      cudaError_t e = prep_kernel(k, smem);
      if (e != cudaSuccess) return e;
      k<<<grid_for(k, threads, smem, ntiles), threads, smem, st>>>(G, X, Y, Hx, Hy, ntiles);
      return cudaGetLastError();
    }
  }
  const size_t smem = AdjSmem<M, C>::bytes;
  auto k = tile_adj_kernel<M, C, false>;
  cudaError_t e = prep_kernel(k, smem);
  if (e != cudaSuccess) return e;
  k<<<grid_for(k, threads, smem, ntiles), threads, smem, st>>>(G, X, Y, Hx, Hy, ntiles);
  return cudaGetLastError();
}

template <class M>
static cudaError_t launch_adj(int C, const typename M::W* G, const typename M::In* X,
                              const typename M::In* Y, typename M::W* Hx, typename M::W* Hy,
                              long long ntiles, cudaStream_t st) {
  switch (C) {
    case 1: return launch_adj_c<M, 1>(G, X, Y, Hx, Hy, ntiles, st);
    case 2: return launch_adj_c<M, 2>(G, X, Y, Hx, Hy, ntiles, st);
    case 3: return launch_adj_c<M, 3>(G, X, Y, Hx, Hy, ntiles, st);
    case 4: return launch_adj_c<M, 4>(G, X, Y, Hx, Hy, ntiles, st);
    case 5: return launch_adj_c<M, 5>(G, X, Y, Hx, Hy, ntiles, st);
    case 6: return launch_adj_c<M, 6>(G, X, Y, Hx, Hy, ntiles, st);
    case 7: return launch_adj_c<M, 7>(G, X, Y, Hx, Hy, ntiles, st);
    case 8: return launch_adj_c<M, 8>(G, X, Y, Hx, Hy, ntiles, st);
  }
  return cudaErrorInvalidValue;
}

template <class M>
static cudaError_t run_backward(const BwdPlan& p, const void* dz, const void* x, const void* y,
                                void* dx, void* dy, unsigned char* ws, cudaStream_t st) {
  typedef typename M::In In;
  typedef typename M::W W;
  const int D = p.D, C = p.C, a = p.a;
  if (D == 0) {
    ProfileScope prof(st, "scalar_adj");
    scalar_adj_kernel<M><<<1, 32, 0, st>>>((const W*)dz, (const In*)x, (const In*)y, (W*)dx,
                                           (W*)dy);
    return cudaGetLastError();
  }
  cudaError_t e;
  // I^T on the outer axes: dz -> G (the first pass copies out of dz).  The
  // passes have the shape of the forward's whole-array passes for the same
  // (D, dtype), so they take the tile width of its default schedule.
  const hc_schedule fs = resolve_schedule(D, p.dtype, nullptr);
  const W* G = (const W*)dz;
  W* Gbuf = (W*)(ws + p.off_g);
  for (int i = 0; i < p.n_it; ++i) {
    const int d0 = p.it_d0[i], k = p.it_k[i];
    const long long hi = (long long)pow3z(d0);
    const long long lo = (long long)pow3z(a - d0 - k) * (long long)pow3z(C);
    // the pass over the outermost axes (d0 = 0) takes the outer width.  A
    // 16-column tile of 16-byte row copies over 4-byte elements widens each
    // row to 20 elements (1.25x the reads); the transposed passes take the
    // 32-column form instead (D = 18 float32, one GB300: I^T passes 1.605 ->
    // 1.507 ms, same bits)
    int cols = d0 == 0 && p.n_it >= 2 && fs.cols_outer ? fs.cols_outer : fs.cols;
    if (cols == -16 && sizeof(W) == 4) cols = -32;
    e = launch_interp<M, false, true>(k, cols, G, Gbuf, hi, lo, st);
    if (e != cudaSuccess) return e;
    G = Gbuf;
  }
  // outer evaluation of x and y
  const In* X = (const In*)x;
  const In* Y = (const In*)y;
  In* Xo = (In*)(ws + p.off_xo);
  In* Yo = (In*)(ws + p.off_yo);
  In* Tx = (In*)(ws + p.off_tx);
  In* Ty = (In*)(ws + p.off_ty);
  for (int i = 0; i < p.n_eval; ++i) {
    const int d0 = p.eval_d0[i], k = p.eval_k[i];
    In* ox = p.eval_to_final[i] ? Xo : Tx;
    In* oy = p.eval_to_final[i] ? Yo : Ty;
    e = launch_eval<M>(k, X, Y, ox, oy, (long long)pow3z(d0), (long long)1 << (D - d0 - k), st);
    if (e != cudaSuccess) return e;
    X = ox;
    Y = oy;
  }
  // tiles
  W* Hx = a > 0 ? (W*)(ws + p.off_hx) : (W*)dx;
  W* Hy = a > 0 ? (W*)(ws + p.off_hy) : (W*)dy;
  if (!dx) Hx = nullptr;
  if (!dy) Hy = nullptr;
  e = launch_adj<M>(C, G, X, Y, Hx, Hy, (long long)pow3z(a), st);
  if (e != cudaSuccess) return e;
  // E^T on the outer axes, inner first
  W* Ex = (W*)(ws + p.off_ex);
  W* Ey = (W*)(ws + p.off_ey);
  const W* sx = Hx;
  const W* sy = Hy;
  for (int i = 0; i < p.n_et; ++i) {
    const int d0 = p.et_d0[i], k = p.et_k[i];
    const bool last = i == p.n_et - 1;
    W* ox = last ? (W*)dx : (p.et_to_h[i] ? (W*)(ws + p.off_hx) : Ex);
    W* oy = last ? (W*)dy : (p.et_to_h[i] ? (W*)(ws + p.off_hy) : Ey);
    if (!dx) ox = nullptr;
    if (!dy) oy = nullptr;
    const long long hi = (long long)pow3z(d0);
    const long long lo = (long long)1 << (D - d0 - k);
    e = launch_et<M>(k, sx, sy, ox, oy, hi, lo, st);
    if (e != cudaSuccess) return e;
    sx = ox;
    sy = oy;
  }
  return cudaSuccess;
}

}  // namespace hc

extern "C" size_t hc_backward_workspace_size(int D, hc_dtype dtype) {
  if (D < 0 || D > HC_MAX_D || hc::elem_size(dtype) == 0 || hc::wide_intermediate(dtype)) return 0;
  return hc::make_bwd_plan(D, dtype).ws_bytes;
}

extern "C" hc_status hc_convolve_backward(const void* dz, const void* x, const void* y, void* dx,
                                          void* dy, int D, hc_dtype dtype, void* workspace,
                                          size_t ws_bytes, hc_stream_t stream) {
  using namespace hc;
  if (D < 0 || D > HC_MAX_D) return HC_ERR_ARG;
  const size_t es = elem_size(dtype);
  if (es == 0 || hc::wide_intermediate(dtype)) return HC_ERR_DTYPE;
  if (!dz || !x || !y || (!dx && !dy)) return HC_ERR_ARG;
  if (!aligned(dz, 16) || !aligned(x, 16) || !aligned(y, 16) || (dx && !aligned(dx, 16)) ||
      (dy && !aligned(dy, 16)))
    return HC_ERR_ALIGN;
  const BwdPlan p = make_bwd_plan(D, dtype);
  if (ws_bytes < p.ws_bytes) return HC_ERR_WORKSPACE;
  if (p.ws_bytes > 0 && !workspace) return HC_ERR_ARG;
  if (workspace && !aligned(workspace, 256)) return HC_ERR_ALIGN;
  const size_t nx = es << D, nz = es * pow3z(D);
  const void* ins[3] = {dz, x, y};
  const size_t nin[3] = {nz, nx, nx};
  void* outs[2] = {dx, dy};
  for (int o = 0; o < 2; ++o) {
    if (!outs[o]) continue;
    for (int i = 0; i < 3; ++i)
      if (overlaps(outs[o], nx, ins[i], nin[i])) return HC_ERR_ALIAS;
    if (workspace && overlaps(outs[o], nx, workspace, p.ws_bytes)) return HC_ERR_ALIAS;
  }
  if (dx && dy && overlaps(dx, nx, dy, nx)) return HC_ERR_ALIAS;
  if (workspace && p.ws_bytes > 0)
    for (int i = 0; i < 3; ++i)
      if (overlaps(workspace, p.ws_bytes, ins[i], nin[i])) return HC_ERR_ALIAS;
  cudaError_t e = cudaErrorInvalidValue;
  switch (dtype) {
    case HC_INT64:
      e = run_backward<ModeI64>(p, dz, x, y, dx, dy, (unsigned char*)workspace, (cudaStream_t)stream);
      break;
    case HC_FP64:
      e = run_backward<ModeF64>(p, dz, x, y, dx, dy, (unsigned char*)workspace, (cudaStream_t)stream);
      break;
    case HC_FP32:
      e = run_backward<ModeF32>(p, dz, x, y, dx, dy, (unsigned char*)workspace, (cudaStream_t)stream);
      break;
    default: break;
  }
  return record_cuda_error(e);
}
