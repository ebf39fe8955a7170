// Persistent ticket engine shared by the batched kernel (many independent
// convolutions) and the chunked forward kernel (one large convolution cut
// into chunks of C + m axes).
//
// A unit is one convolution of C + m axes.  Its inputs arrive with the first
// m_pre of the m outer ("middle") axes already evaluated: rows
// [3^m_pre][2^(m - m_pre)][2^C]; the remaining m - m_pre <= 6 middle axes are
// evaluated on the fly inside the tile loads.  A unit contributes 3^m tile tickets (tile_body: inner
// evaluation, products, inner interpolation of C axes, written to the unit's
// W region) followed by column tickets (the m middle axes interpolated over
// cpt column tiles of L columns each).
//
// Tickets are claimed in increasing order from one global counter.  A column
// ticket waits only for tile tickets of its own unit, which have smaller
// numbers; a CTA claims its next ticket early only
// while it cannot be waiting (during a tile, or after its wait ended), so a
// claimed ticket always belongs to a CTA that will reach it, the smallest
// unfinished claimed ticket only ever waits on finished work, and every wait
// ends.  The waits are
// bounded anyway: after ~1 s a wait gives up, marks its unit's counter and
// records HC_ERR_TIMEOUT in the workspace status word; later waiters on the
// same unit give up at once.
//
// A unit's column tickets follow its tiles within about one unit's worth of
// tickets, so its 3^(C+m) intermediate is still in L2 when they read it back
// (through L2 only: ld.global.cg).
#pragma once

#include <type_traits>

#include "hc_common.cuh"
#include "hc_tile.cuh"

namespace hc {

struct UnitDesc {
  const void* x;    // 2^(C+m) elements
  const void* y;
  void* w;          // tile outputs, 3^(C+m) W elements
  void* z;          // column outputs (Out elements when the columns finish the
                    // result in another type, else the same array as w)
  long long first;  // first ticket of the unit
  int C, m;
  int n_tiles;      // 3^m
  int n_cols;       // column tickets
  int cpt;          // column tiles per column ticket
  int need;         // finished tiles a column ticket waits for (n_tiles)
  int m_pre;        // leading middle axes already evaluated in x, y
  int pad;
};

// Units generated arithmetically: unit u reads x + u * in_stride and writes
// w + u * out_stride (and z + u * out_stride).
struct UniformUnits {
  const void* x;
  const void* y;
  void* w;
  void* z;
  long long in_stride, out_stride, per_unit;
  int C, m, n_tiles, n_cols, cpt, need, m_pre, units;
  int lag;  // tiles of unit u claimed before the column tickets of unit u - 1
};

constexpr unsigned long long kSpinLimit = 1ull << 22;  // x >= 256 ns sleeps: ~1 s
constexpr unsigned long long kPoison = 1ull << 63;

// Element i of operand op's row, evaluated on the digit-1 axes at the
// tile's middle digits: digit 0 / 2 selects bit 0 / 1 (folded into `base`);
// the m axes with digit 1 are summed as a pairwise tree whose first level
// pairs the outermost of them (the recursion evaluates axis 1 before axis 2,
// so its sums nest that way).  Leaves are loaded in blocks of 2^min(m,3)
// independent loads (one memory round trip per block; with m <= 3 the whole
// value is one loop-free block); a block is a subtree of the three outermost
// digit-1 axes, and blocks are combined in order.
template <class M>
struct OtfLoader {
  typedef typename M::In In;
  const In* x;
  const In* y;
  long long base;  // fixed bits, as a flat offset
  int m;           // digit-1 axes added so far
  int off[8];      // leaf offsets within a block: the three outermost digit-1 axes
  int hoff[8];     // block offsets: the digit-1 axes beyond the third

  __device__ __forceinline__ void init(const In* x_, const In* y_, long long base_) {
    x = x_;
    y = y_;
    base = base_;
    m = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) off[j] = hoff[j] = 0;
  }

  // Next digit-1 axis (axis order), `bit` its flat offset (< 2^31: a unit
  // row has at most 2^15 elements).  All indices are static after unrolling,
  // so the loader stays in registers.
  __device__ __forceinline__ void add_axis(int bit) {
    const int q = m++;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (q < 3) {
        if ((j >> q) & 1) off[j] += bit;
      } else {
        if ((j >> (q - 3)) & 1) hoff[j] += bit;
      }
    }
  }

  // The pairwise tree over one block of 2^mb leaves.
  __device__ __forceinline__ In block_sum(const In* s, int mb) const {
    In v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j < (1 << mb)) v[j] = s[off[j]];
    if (mb == 0) return v[0];
    if (mb == 1) return M::add(v[0], v[1]);
    if (mb == 2) return M::add(M::add(v[0], v[1]), M::add(v[2], v[3]));
    return M::add(M::add(M::add(v[0], v[1]), M::add(v[2], v[3])),
                  M::add(M::add(v[4], v[5]), M::add(v[6], v[7])));
  }

  __device__ __forceinline__ In operator()(int op, int i) const {
    const In* s = (op ? y : x) + base + i;
    if (m <= 3) return block_sum(s, m);  // one block: no loop, loads issue together
    const int nblocks = 1 << (m - 3);
    In stack[4];
    int sp = 0;
#pragma unroll 1
    for (int blk = 0; blk < nblocks; ++blk) {
      int h = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (j == blk) h = hoff[j];
      In r = block_sum(s + h, 3);
#pragma unroll 1
      for (int t = blk; t & 1; t >>= 1) r = M::add(stack[--sp], r);
      stack[sp++] = r;
    }
    return stack[0];
  }
};

template <class M>
struct PersistCols {
  static constexpr int L = kPersistCols;
};

template <class M>
__host__ __device__ constexpr int persist_cols() {
  return PersistCols<M>::L;
}

// Tile of runtime size C (batched units of any D).
template <class M, bool FINAL>
__device__ __forceinline__ void tile_any_c(int C, const OtfLoader<M>& ld, void* out,
                                           unsigned char* smem) {
  switch (C) {
    case 0:  // D = 0: z[0] = x[0] * y[0]
      if constexpr (FINAL) {
        if (threadIdx.x == 0) *(typename M::Out*)out = M::out(M::mul(ld(0, 0), ld(1, 0)));
      }
      break;
    case 1: tile_body<M, 1, FINAL>(ld, out, smem); break;
    case 2: tile_body<M, 2, FINAL>(ld, out, smem); break;
    case 3: tile_body<M, 3, FINAL>(ld, out, smem); break;
    case 4: tile_body<M, 4, FINAL>(ld, out, smem); break;
    case 5: tile_body<M, 5, FINAL>(ld, out, smem); break;
    case 6: tile_body<M, 6, FINAL>(ld, out, smem); break;
    case 7: tile_body<M, 7, FINAL>(ld, out, smem); break;
    case 8: tile_body<M, 8, FINAL>(ld, out, smem); break;
    case 9:
      if constexpr (sizeof(typename M::W) == 4) tile_body<M, 9, FINAL>(ld, out, smem);
      break;
  }
}

// m <= 3 middle axes: every thread takes whole columns of [c0, c1), no
// shared memory.
template <class M, int K, bool FIN, int SPOL = kPolNone, int LPOL = kPolNone>
__device__ __forceinline__ void cols_small_k(const typename M::W* src, void* dst, long long c0,
                                             long long c1, long long lo) {
  typedef typename M::W W;
  typedef typename M::Out Out;
#pragma unroll 1
  for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    W v[p3(K)];
#pragma unroll
    for (int j = 0; j < p3(K); ++j) v[j] = ld_cg_pol<LPOL>(src + j * lo + c);
    interp_pencil<M, K>(v);
    if constexpr (FIN) {
#pragma unroll
      for (int j = 0; j < p3(K); ++j)
        st_pol<SPOL>(reinterpret_cast<Out*>(dst) + j * lo + c, M::out(v[j]));
    } else {
#pragma unroll
      for (int j = 0; j < p3(K); ++j) st_pol<SPOL>(reinterpret_cast<W*>(dst) + j * lo + c, v[j]);
    }
  }
}

template <class M, bool FIN, int SPOL = kPolNone>
__device__ __forceinline__ void cols_small(int m, const typename M::W* src, void* dst,
                                           long long c0, long long c1, long long lo) {
  switch (m) {
    case 1: cols_small_k<M, 1, FIN, SPOL>(src, dst, c0, c1, lo); break;
    case 2: cols_small_k<M, 2, FIN, SPOL>(src, dst, c0, c1, lo); break;
    case 3: cols_small_k<M, 3, FIN, SPOL>(src, dst, c0, c1, lo); break;
  }
}

// Ticket order.  Unit u's tiles come before its column tickets; the column
// tickets of unit u - 1 are placed after the first `lag` tiles of unit u:
//   tiles(0), tiles(1)[0:lag], cols(0), tiles(1)[lag:], tiles(2)[0:lag],
//   cols(1), tiles(2)[lag:], ..., cols(units - 1).
// With lag about the number of resident CTAs, unit u - 1's last tiles are
// finished when its column tickets are claimed (they rarely wait), and only
// about 1 + lag / n_tiles units' intermediates are live in L2 at a time
// (two full units did not stay in L2: DRAM traffic doubled).
__device__ __forceinline__ void uniform_ticket(long long t, const UniformUnits& uu, int& u,
                                               long long& local) {
  // Ticket counts stay below 2^31 (at most 3^10 units of at most ~1600
  // tickets), so the decoding runs in 32-bit arithmetic.
  const unsigned nt = (unsigned)uu.n_tiles, nc = (unsigned)uu.n_cols;
  const unsigned per = nt + nc, lag = (unsigned)uu.lag;
  const unsigned tt = (unsigned)t;
  if (tt < nt) {
    u = 0;
    local = tt;
    return;
  }
  const unsigned tp = tt - nt;
  const unsigned body = (unsigned)(uu.units - 1) * per;
  if (tp < body) {
    const unsigned b = tp / per, r = tp - b * per;
    if (r < lag) {
      u = (int)b + 1;
      local = r;
    } else if (r < lag + nc) {
      u = (int)b;
      local = nt + (r - lag);
    } else {
      u = (int)b + 1;
      local = r - nc;
    }
  } else {
    u = uu.units - 1;
    local = nt + (tp - body);
  }
}

// counters[0]: ticket counter; counters[1 + u]: finished tiles of unit u.
// CT > 0: every unit has C = CT (compile-time tile); CT < 0: per-unit C.
// UNIFORM: units from `uu`; else (unit, local) = ticket_map[t], unit desc[unit].
// FIN: column tickets write Out elements to z (float-float -> binary32).
// L2HINT: tiles are stored with L2 priority evict_last (their unit's column
// tickets read them back from L2) and finished columns with evict_first
// (nothing in the launch reads them again), so that the units in flight keep
// their place in L2.
template <class M, int CT, bool UNIFORM, bool FIN, bool L2HINT = false>
__device__ __forceinline__ void persistent_loop(const UnitDesc* __restrict__ desc,
                                                const int2* __restrict__ ticket_map,
                                                const UniformUnits& uu, long long total,
                                                unsigned long long* counters, WsHeader* hdr,
                                                unsigned char* smem) {
  typedef typename M::In In;
  typedef typename M::W W;
  typedef typename M::Out Out;
  typedef typename std::conditional<FIN, Out, W>::type ZT;
  // Broadcast slots, double-buffered by iteration parity: thread 0 rewrites a
  // slot two iterations later, after every thread has passed the barrier at
  // the top of the iteration in between.
  __shared__ long long s_ticket[2], s_local[2];
  __shared__ int s_unit[2], s_ok[2];
  const int tid = threadIdx.x;
  // Thread 0 claims the next ticket early (its result is first read at the
  // top of the next iteration), but never while its CTA may still wait: a
  // CTA stalled in a wait must not hold a claimed ticket that others wait on.
  long long next = -1;
#pragma unroll 1
  for (int it = 0;; it ^= 1) {
    if (tid == 0) {
      const long long t = next >= 0 ? next : (long long)atomicAdd(&counters[0], 1ull);
      next = -1;
      int u = 0;
      long long local = 0;
      if (t < total) {
        if constexpr (UNIFORM) {
          uniform_ticket(t, uu, u, local);
        } else {
          const int2 e = ticket_map[t];
          u = e.x;
          local = e.y;
        }
      }
      s_ticket[it] = t;
      s_unit[it] = u;
      s_local[it] = local;
    }
    __syncthreads();
    const long long t = s_ticket[it];
    if (t >= total) break;
    const int u = s_unit[it];
    const long long local = s_local[it];
    UnitDesc d;
    if constexpr (UNIFORM) {
      d.x = (const In*)uu.x + u * uu.in_stride;
      d.y = (const In*)uu.y + u * uu.in_stride;
      d.w = (W*)uu.w + u * uu.out_stride;
      d.z = (ZT*)uu.z + u * uu.out_stride;
      d.C = uu.C;
      d.m = uu.m;
      d.n_tiles = uu.n_tiles;
      d.n_cols = uu.n_cols;
      d.cpt = uu.cpt;
      d.need = uu.need;
      d.m_pre = uu.m_pre;
    } else {
      d = desc[u];
    }
    const int C = CT > 0 ? CT : d.C;
    if (local < d.n_tiles) {
      if (tid == 0) next = (long long)atomicAdd(&counters[0], 1ull);  // tiles never wait
      // ---- tile at middle digits alpha = local (the unit's axis 1 most
      // significant): m_pre pre-evaluated digits (a row index), then the
      // m - m_pre on-the-fly ones.  32-bit arithmetic with constant divisors
      // only: this runs in every thread of every tile.
      const int m_otf = d.m - d.m_pre;
      const int p3otf = pow3i(m_otf);
      const int loc = (int)local;  // < 3^m <= 729
      const int pre_row = loc / p3otf;
      int rem = loc - pre_row * p3otf;
      int dg[6];
#pragma unroll
      for (int q = 5; q >= 0; --q) {
        dg[q] = rem % 3;
        rem /= 3;
      }
      OtfLoader<M> ld;
      ld.init((const In*)d.x, (const In*)d.y, (long long)pre_row << (C + m_otf));
#pragma unroll
      for (int q6 = 0; q6 < 6; ++q6) {
        if (q6 < 6 - m_otf) continue;
        const int bit = 1 << (C + 5 - q6);  // axis q6 - (6 - m_otf) of the m_otf
        if (dg[q6] == 2) ld.base += bit;
        if (dg[q6] == 1) ld.add_axis(bit);
      }
      if (d.m == 0) {
        if constexpr (CT > 0)
          tile_body<M, (CT > 0 ? CT : 1), true>(ld, (Out*)d.z, smem);
        else
          tile_any_c<M, true>(C, ld, (Out*)d.z, smem);
      } else {
        W* out = (W*)d.w + (long long)loc * (CT > 0 ? p3(CT > 0 ? CT : 1) : pow3i(C));
        if constexpr (CT > 0)
          tile_body<M, (CT > 0 ? CT : 1), false, OtfLoader<M>, false,
                    L2HINT ? kPolKeep : kPolNone>(ld, out, smem);
        else
          tile_any_c<M, false>(C, ld, out, smem);
        // release: a barrier (the tile body's last one for tiles of more than
        // three axes) orders every thread's stores before thread 0's fence,
        // which orders them before the counter increment
        if (C <= 3) __syncthreads();
        if (tid == 0) {
          __threadfence();
          atomicAdd(&counters[1 + u], 1ull);
        }
      }
    } else {
      // ---- column ticket: interpolate the m middle axes
      if (tid == 0) {
        const unsigned long long* done = &counters[1 + u];
        unsigned long long spins = 0;
        int ok = 1;
        for (;;) {
          unsigned long long v;  // acquire: the unit's tile outputs are visible after it
          asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(done) : "memory");
          if (v & kPoison) {
            ok = 0;
            break;
          }
          if (v >= (unsigned long long)d.need) break;
          __nanosleep(256);
          if (++spins > kSpinLimit) {
            ok = 0;
            atomicOr(&counters[1 + u], kPoison);
            atomicExch(&hdr->status, (unsigned int)HC_ERR_TIMEOUT);
            atomicExch(&hdr->where, (unsigned int)u);
            break;
          }
        }
        s_ok[it] = ok;
        next = (long long)atomicAdd(&counters[0], 1ull);  // the wait is over
      }
      __syncthreads();
      if (s_ok[it]) {
        constexpr int L = PersistCols<M>::L;
        const long long lo = CT > 0 ? p3(CT > 0 ? CT : 1) : pow3i(C);
        const long long c0 = (local - d.n_tiles) * d.cpt * L;
        const long long c1 = (c0 + (long long)d.cpt * L < lo) ? c0 + (long long)d.cpt * L : lo;
        constexpr int SP = L2HINT ? kPolStream : kPolNone;
        if (d.m <= 3) {
          cols_small<M, FIN, SP>(d.m, (const W*)d.w, d.z, c0, c1, lo);
        } else {
          const int n = (int)((c1 - c0 + L - 1) / L);
          auto tile = [&](int i, long long& base, long long& l0) {
            l0 = c0 + (long long)i * L;
            base = l0;
          };
          switch (d.m) {
            case 4:
              interp_tiles_pipelined<M, 1, 3, L, FIN, decltype(tile), false, NoPtrs, kPolNone, SP>(
                  (const W*)d.w, d.z, lo, n, tile, smem);
              break;
            case 5:
              interp_tiles_pipelined<M, 2, 3, L, FIN, decltype(tile), false, NoPtrs, kPolNone, SP>(
                  (const W*)d.w, d.z, lo, n, tile, smem);
              break;
            case 6:
              interp_tiles_pipelined<M, 3, 3, L, FIN, decltype(tile), false, NoPtrs, kPolNone, SP>(
                  (const W*)d.w, d.z, lo, n, tile, smem);
              break;
          }
        }
      }
    }
    // No barrier here: every smem-using body above ends with one, and the
    // broadcast slots are double-buffered.
  }
}

}  // namespace hc
