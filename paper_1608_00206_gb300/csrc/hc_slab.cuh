// The L2-resident chunk engine ("slab" kernel) of the chunked-bulk schedule.
//
// One persistent launch convolves the 3^a' units of C + m axes of a large
// convolution.  A unit is 3^m tiles of C axes (its middle digits) followed by
// column tickets that interpolate the m middle axes of the unit's 3^(C+m)
// intermediates.  Unlike the generic ticket engine (hc_persist.cuh), which
// evaluates up to three middle axes inside the tile loads, every middle axis
// here is evaluated beforehand by the whole-array evaluation passes, so a
// tile reads two plain rows of 2^C elements (prefetched with cp.async while
// the previous ticket runs) and the tile body keeps its registers.  Each
// finished tile leaves shared memory in one bulk copy (TMA engine) with L2
// priority evict_last, and drains while the CTA computes its next tile in the
// other W buffer; finished columns are stored with priority evict_first.  The
// unit in flight therefore stays in L2 between its tiles and its columns,
// and the finished ones leave it first.
//
// Ticket order, waits and their bounds are those of the generic engine
// (uniform_ticket, a ~1 s bounded spin that records HC_ERR_TIMEOUT).  A tile
// is counted as finished in its unit's counter once its bulk copy has
// completed: the CTA counts tile i after issuing the copy of tile i + 1, or
// before it takes a column ticket, or when it runs out of tickets -- always
// before any wait, so no CTA waits while holding an uncounted tile.
#pragma once

#include "hc_common.cuh"
#include "hc_persist.cuh"
#include "hc_tile.cuh"

namespace hc {

// Bulk (TMA engine) shared -> global store with an L2 priority; both
// addresses 16-byte aligned, bytes a multiple of 16; one thread issues it.
template <int POL>
__device__ __forceinline__ void bulk_store_pol(void* gmem, const void* smem, unsigned bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const unsigned long long pol = l2_policy<POL>();
  asm volatile(
      "cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;\n" ::"l"(
          gmem),
      "r"(s), "r"(bytes), "l"(pol)
      : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}

struct SlabArgs {
  const void* x;  // rows: tile g = unit * 3^m + middle digits at g * 2^C (all middle
  const void* y;  //       axes and the unit's outer axes evaluated)
  void* w;        // tiles: tile g's 3^C intermediates at g * 3^C
  void* z;        // column outputs (Out elements when FIN, else the same array as w)
  unsigned long long* ctr;  // [0] ticket counter; [1 + u] finished tiles of unit u
  WsHeader* hdr;
  UniformUnits uu;          // ticket order: n_tiles, n_cols, cpt, units, lag, per_unit
  long long total;
};

// Shared memory: two W tiles (TileBulk's layout), which the column tickets
// reuse for their column tile, then the two row buffers, placed above
// whichever of the two is larger.
// Columns per column tile of the slab kernel: 16 (128-byte row segments for
// 8-byte intermediates), twice the generic engine's 8, whose 64-byte segments
// halve what each load instruction moves.  A ticket's cpt * 8 columns are an
// even number, i.e. whole tiles except at the end of a unit's 3^C columns.
constexpr int kSlabCols = 16;

template <class M, int C, int MM>
struct SlabSmem {
  static constexpr size_t kCols =
      MM <= 3 ? 0 : sizeof(typename M::W) * (size_t)p3(MM) * kSlabCols;
  static constexpr size_t kRowsOff =
      TileBulk<M, C>::kOff > kCols ? TileBulk<M, C>::kOff : (kCols + 15) / 16 * 16;
  static constexpr size_t bytes = kRowsOff + 2 * 2 * sizeof(typename M::In) * (size_t)p2(C);
};

template <class M, int C, int MM, bool FIN>
__global__ void __launch_bounds__(256, (sizeof(typename M::W) == 4 ? 3 : 2))
    slab_kernel(SlabArgs a) {
  typedef typename M::In In;
  typedef typename M::W W;
  typedef typename M::Out Out;
  typedef TileBulk<M, C> B;
  typedef TileStages<M, C> St;
  typedef TileShape<C> S;
  static_assert(S::G >= 2, "slab tiles have C >= 4");
  constexpr int NT = p3(MM);  // tiles per unit
  constexpr int N = p3(C);    // elements per tile
  constexpr int L = kPersistCols;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_tk[2];
  __shared__ int s_ok;
  In* rows = reinterpret_cast<In*>(smem + SlabSmem<M, C, MM>::kRowsOff);  // [buf][operand][2^C]
  const int tid = threadIdx.x, nt = blockDim.x;
  const In* X = reinterpret_cast<const In*>(a.x);
  const In* Y = reinterpret_cast<const In*>(a.y);
  W* Wg = reinterpret_cast<W*>(a.w);

  auto prefetch = [&](long long g, int rb) {
#pragma unroll 1
    for (int e = tid; e < 2 * p2(C); e += nt) {
      const int op = e >> C, i = e & (p2(C) - 1);
      cp_async<sizeof(In)>(rows + (rb * 2 + op) * p2(C) + i, (op ? Y : X) + g * p2(C) + i);
    }
    cp_async_commit();
  };
  // tile g's W tile in buffer b, placed at its output's address modulo 16
  auto wtile = [&](long long g, int b) {
    return smem + b * B::kWB + (unsigned)(reinterpret_cast<uintptr_t>(Wg + g * N) & 15);
  };
  // thread 0: count a tile whose bulk copy has completed (and whose
  // per-thread head/tail stores precede this point by a barrier)
  auto release = [&](int u) {
    asm volatile("fence.proxy.async.global;\n" ::: "memory");
    __threadfence();
    atomicAdd(&a.ctr[1 + u], 1ull);
  };
  int pend_u = -1;  // thread 0: unit of the last tile whose copy is not counted yet

  if (tid == 0) s_tk[0] = (long long)atomicAdd(&a.ctr[0], 1ull);
  __syncthreads();
  long long t = s_tk[0];
  int it = 0, rb = 0, wb = 0;
  {
    int u;
    long long local;
    if (t < a.total) {
      uniform_ticket(t, a.uu, u, local);
      if (local < NT) prefetch((long long)u * NT + local, rb);
    }
  }
#pragma unroll 1
  while (t < a.total) {
    int u;
    long long local;
    uniform_ticket(t, a.uu, u, local);
    if (local < NT) {
      // ---- tile ticket: tile g of unit u (its rows are in buffer rb)
      const long long g = (long long)u * NT + local;
      if (tid == 0) s_tk[it ^ 1] = (long long)atomicAdd(&a.ctr[0], 1ull);  // tiles never wait
      cp_async_wait<0>();
      if (tid == 0) bulk_wait<1, true>();  // W buffer wb: tile i-2's copy has read it
      __syncthreads();
      const long long tn = s_tk[it ^ 1];
      if (tn < a.total) {
        int un;
        long long ln;
        uniform_ticket(tn, a.uu, un, ln);
        if (ln < NT) prefetch((long long)un * NT + ln, rb ^ 1);
      }
      unsigned char* w = wtile(g, wb);
      {
        RowLoader<In> ld{rows + (rb * 2) * p2(C), rows + (rb * 2 + 1) * p2(C)};
#pragma unroll 1
        for (int p = tid; p < St::kStage0; p += nt) St::stage0(ld, w, p);
      }
      __syncthreads();
      if constexpr (S::G == 3) {
        St::stage1(w);
        __syncthreads();
      }
      St::fused(w);
      __syncthreads();
      if constexpr (S::G == 3) {
        St::interp1(w);
        __syncthreads();
      }
#pragma unroll 1
      for (int r = tid; r < St::kInterp0; r += nt) St::template interp0<false, true>(nullptr, w, r);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
      // tile g is in w[0, N): head / body / tail split at 16-byte boundaries
      W* out = Wg + g * N;
      const unsigned mis = (unsigned)(reinterpret_cast<uintptr_t>(out) & 15);
      const int head = mis ? (int)((16 - mis) / sizeof(W)) : 0;
      const int body = (int)(((N - head) * sizeof(W)) / 16 * 16 / sizeof(W));
      const W* ws = reinterpret_cast<const W*>(w);
      if (tid == 0 && body > 0)
        bulk_store_pol<kPolKeep>(out + head, ws + head, (unsigned)(body * sizeof(W)));
      for (int e = tid; e < head; e += nt) st_pol<kPolKeep>(out + e, ws[e]);
      for (int e = head + body + tid; e < N; e += nt) st_pol<kPolKeep>(out + e, ws[e]);
      if (tid == 0) {
        if (pend_u >= 0) {
          bulk_wait<1, false>();  // the previous tile's copy has completed
          release(pend_u);
        }
        pend_u = u;
      }
      rb ^= 1;
      wb ^= 1;
      it ^= 1;
      t = tn;
    } else {
      // ---- column ticket: interpolate the m middle axes of unit u
      if (tid == 0) {
        if (pend_u >= 0) {
          bulk_wait<0, false>();
          release(pend_u);
          pend_u = -1;
        }
        const unsigned long long* done = &a.ctr[1 + u];
        unsigned long long spins = 0;
        int ok = 1;
        for (;;) {
          unsigned long long v;  // acquire: the unit's tiles are visible after it
          asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(done) : "memory");
          if (v & kPoison) {
            ok = 0;
            break;
          }
          if (v >= (unsigned long long)NT) break;
          __nanosleep(256);
          if (++spins > kSpinLimit) {
            ok = 0;
            atomicOr(&a.ctr[1 + u], kPoison);
            atomicExch(&a.hdr->status, (unsigned int)HC_ERR_TIMEOUT);
            atomicExch(&a.hdr->where, (unsigned int)u);
            break;
          }
        }
        s_ok = ok;
        s_tk[it ^ 1] = (long long)atomicAdd(&a.ctr[0], 1ull);  // the wait is over
      }
      __syncthreads();  // also: no bulk copy reads the W buffers any more
      if (s_ok) {
        const long long c0 = (local - NT) * a.uu.cpt * (long long)L;
        const long long c1 = c0 + (long long)a.uu.cpt * L < N ? c0 + (long long)a.uu.cpt * L : N;
        const W* src = Wg + (long long)u * NT * N;
        void* dst = FIN ? (void*)(reinterpret_cast<Out*>(a.z) + (long long)u * NT * N)
                        : (void*)(Wg + (long long)u * NT * N);
        // FIN: the columns write z, and the unit's intermediates are not
        // read again, so their reads drop them from L2 first
        constexpr int LP = FIN ? kPolStream : kPolNone;
        if constexpr (MM <= 3) {
          cols_small_k<M, MM, FIN, kPolStream, LP>(src, dst, c0, c1, N);
        } else {
          // one 3^m x 16 tile at a time: round 1 loads its pencils straight
          // from L2 into registers (27 independent loads per thread)
#pragma unroll 1
          for (long long l0 = c0; l0 < c1; l0 += kSlabCols)
            interp_tile_body<M, MM - 3, 3, kSlabCols, FIN, true, false, LP, kPolStream>(
                src, dst, l0, l0, N, smem);
        }
      }
      __syncthreads();  // s_tk, s_ok and shared memory reused by the next ticket
      const long long tn = s_tk[it ^ 1];
      if (tn < a.total) {
        int un;
        long long ln;
        uniform_ticket(tn, a.uu, un, ln);
        if (ln < NT) prefetch((long long)un * NT + ln, rb);
      }
      it ^= 1;
      t = tn;
    }
  }
  if (tid == 0 && pend_u >= 0) {
    bulk_wait<0, false>();
    release(pend_u);
  }
}

}  // namespace hc
