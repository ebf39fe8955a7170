// Batching form: many independent hypercube convolutions of uneven D in one
// persistent launch.
//
// Work list.  Instance i (C_i = min(D_i, tile axes), a_i = D_i - C_i <= 6)
// contributes 3^a_i tile tickets (the fused tile of the plain path, with the
// outer-axis evaluation done on the fly) followed, when a_i > 0, by
// ceil(3^C_i / L) column tickets that interpolate the a_i outer axes.
// Tickets are numbered instance by instance and claimed in increasing order
// from one global counter, so a column ticket only ever waits for tile
// tickets with smaller numbers, all already claimed by running CTAs: the
// wait always ends.  It is bounded anyway: past ~1 s it records
// HC_ERR_TIMEOUT in the workspace status word and skips the ticket.
//
// Consecutive tickets belong to the same instance, so an instance's 3^D
// intermediate (<= 19 MB for D = 14 float32) is still in L2 when its column
// tickets read it back.
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "hc_common.cuh"
#include "hc_profile.cuh"
#include "hc_kernels.cuh"
#include "hc_tile.cuh"

namespace hc {

struct BatchDesc {
  const void* x;
  const void* y;
  void* z;
  void* w;  // interpolation buffer: z, or a float-float buffer in the workspace
  long long first;  // first ticket
  int D, C, a;
  int n_tiles;  // 3^a
  int n_cols;   // column tickets (0 when a == 0)
  int need;     // finished tiles a column ticket waits for (n_tiles)
};
static_assert(sizeof(BatchDesc) == 64, "descriptor is 64 bytes");

constexpr unsigned long long kSpinLimit = 1ull << 22;  // x >= 256 ns sleeps: > 1 s

// Element i of the row of operand op evaluated on the outer axes at digits
// alpha.  Digit 0 / 2 picks bit 0 / 1; the m axes with digit 1 are summed as
// a pairwise tree whose first level pairs the outermost of them: the
// recurrence evaluates axis 1 before axis 2, so its sums nest that way.
template <class M>
struct OtfLoader {
  typedef typename M::In In;
  const In* x;
  const In* y;
  long long base;       // fixed bits, as a flat offset
  long long stride[6];  // flat offsets of the digit-1 axes, outermost first
  int m;
  __device__ __forceinline__ In operator()(int op, int i) const {
    const In* s = (op ? y : x) + base + i;
    if (m == 0) return s[0];
    In stack[7];
    int sp = 0;
#pragma unroll 1
    for (int c = 0; c < (1 << m); ++c) {
      long long off = 0;
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if (q < m && ((c >> q) & 1)) off += stride[q];
      In v = s[off];
#pragma unroll 1
      for (int t = c; t & 1; t >>= 1) v = M::add(stack[--sp], v);
      stack[sp++] = v;
    }
    return stack[0];
  }
};

template <class M>
struct BatchCols {
  static constexpr int L = sizeof(typename M::W) == 4 ? 32 : 16;
};

template <class M, bool FINAL>
__device__ __forceinline__ void batch_tile(int C, const OtfLoader<M>& ld, void* out,
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

template <class M>
__device__ __forceinline__ void batch_interp(int a, const typename M::W* src, void* dst,
                                             long long l0, long long lo, unsigned char* smem) {
  constexpr int L = BatchCols<M>::L;
  constexpr bool FIN = !std::is_same<typename M::W, typename M::Out>::value;
  switch (a) {
    case 1: interp_tile_body<M, 0, 1, L, FIN, true>(src, dst, l0, l0, lo, smem); break;
    case 2: interp_tile_body<M, 0, 2, L, FIN, true>(src, dst, l0, l0, lo, smem); break;
    case 3: interp_tile_body<M, 0, 3, L, FIN, true>(src, dst, l0, l0, lo, smem); break;
    case 4: interp_tile_body<M, 1, 3, L, FIN, true>(src, dst, l0, l0, lo, smem); break;
    case 5: interp_tile_body<M, 2, 3, L, FIN, true>(src, dst, l0, l0, lo, smem); break;
    case 6: interp_tile_body<M, 3, 3, L, FIN, true>(src, dst, l0, l0, lo, smem); break;
  }
}

// counters[0]: ticket counter; counters[1 + i]: finished tiles of instance i.
template <class M>
__global__ void __launch_bounds__(256) batched_kernel(const BatchDesc* __restrict__ desc, int n,
                                                      long long total,
                                                      unsigned long long* counters,
                                                      WsHeader* hdr) {
  typedef typename M::In In;
  typedef typename M::W W;
  typedef typename M::Out Out;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_ticket;
  __shared__ int s_inst;
  __shared__ int s_ok;
  const int tid = threadIdx.x;
#pragma unroll 1
  for (;;) {
    if (tid == 0) {
      const long long t = (long long)atomicAdd(&counters[0], 1ull);
      int lo = 0, hi = n - 1;
      if (t < total) {
        while (lo < hi) {  // last instance whose first ticket is <= t
          const int mid = (lo + hi + 1) >> 1;
          if (desc[mid].first <= t) lo = mid; else hi = mid - 1;
        }
      }
      s_ticket = t;
      s_inst = lo;
    }
    __syncthreads();
    const long long t = s_ticket;
    if (t >= total) break;
    const BatchDesc d = desc[s_inst];
    const long long local = t - d.first;
    if (local < d.n_tiles) {
      // ---- a fused tile at outer digits alpha = local (axis 1 most significant)
      OtfLoader<M> ld;
      ld.x = (const In*)d.x;
      ld.y = (const In*)d.y;
      ld.base = 0;
      ld.m = 0;
      const long long rem = local;
      long long w3 = 1;
      for (int q = 1; q < d.a; ++q) w3 *= 3;
      for (int q = 0; q < d.a; ++q) {  // q = 0 is axis 1
        const int digit = (int)((rem / w3) % 3);
        w3 /= 3;
        const long long bit = (long long)1 << (d.C + (d.a - 1 - q));
        if (digit == 2) ld.base += bit;
        if (digit == 1) ld.stride[ld.m++] = bit;
      }
      if (d.a == 0) {
        batch_tile<M, true>(d.C, ld, (Out*)d.z, smem);
      } else {
        batch_tile<M, false>(d.C, ld, (W*)d.w + local * (long long)pow3_dev(d.C), smem);
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd(&counters[1 + s_inst], 1ull);
      }
    } else {
      // ---- a column tile of the outer-axis interpolation
      if (tid == 0) {
        // Bit 63 of an instance's counter marks a wait on it that gave up:
        // later waiters on the same instance skip at once, other instances
        // are unaffected.
        volatile unsigned long long* done = &counters[1 + s_inst];
        constexpr unsigned long long kPoison = 1ull << 63;
        unsigned long long spins = 0;
        int ok = 1;
        for (;;) {
          const unsigned long long v = *done;
          if (v & kPoison) {
            ok = 0;
            break;
          }
          if (v >= (unsigned long long)d.need) break;
          __nanosleep(256);
          if (++spins > kSpinLimit) {
            ok = 0;
            atomicOr(&counters[1 + s_inst], kPoison);
            atomicExch(&hdr->status, (unsigned int)HC_ERR_TIMEOUT);
            atomicExch(&hdr->where, (unsigned int)s_inst);
            break;
          }
        }
        __threadfence();
        s_ok = ok;
      }
      __syncthreads();
      if (s_ok) {
        constexpr int L = BatchCols<M>::L;
        const long long l0 = (local - d.n_tiles) * L;
        const long long lo = pow3_dev(d.C);
        batch_interp<M>(d.a, (const W*)d.w, d.z, l0, lo, smem);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host side.

struct BatchPlan {
  hc_dtype dtype;
  int n;
  long long total;
  size_t smem;
  size_t off_ctr, off_desc, off_w, ws_bytes;
};

static std::mutex g_plans_mu;
static std::map<const void*, BatchPlan> g_plans;  // prepared workspaces

static int batch_cmax(hc_dtype dt) { return dt == HC_FP32 ? 9 : 8; }

static size_t tile_smem_bytes(hc_dtype dt, int C);
static size_t interp_smem_bytes(hc_dtype dt, int a);

template <class M>
static size_t tile_smem_m(int C) {
  switch (C) {
    case 1: return TileSmem<M, 1>::bytes;
    case 2: return TileSmem<M, 2>::bytes;
    case 3: return TileSmem<M, 3>::bytes;
    case 4: return TileSmem<M, 4>::bytes;
    case 5: return TileSmem<M, 5>::bytes;
    case 6: return TileSmem<M, 6>::bytes;
    case 7: return TileSmem<M, 7>::bytes;
    case 8: return TileSmem<M, 8>::bytes;
    case 9:
      if constexpr (sizeof(typename M::W) == 4) return TileSmem<M, 9>::bytes;
      return 0;
  }
  return 0;
}

static size_t tile_smem_bytes(hc_dtype dt, int C) {
  switch (dt) {
    case HC_INT64: return tile_smem_m<ModeI64>(C);
    case HC_FP64: return tile_smem_m<ModeF64>(C);
    case HC_FP32: return tile_smem_m<ModeF32>(C);
    case HC_FP32_MIXED: return tile_smem_m<ModeMixed>(C);
  }
  return 0;
}

static size_t interp_smem_bytes(hc_dtype dt, int a) {
  if (a <= 3) return 0;
  const size_t wsz = dt == HC_FP32 ? 4 : 8;
  const size_t L = wsz == 4 ? 32 : 16;
  return wsz * pow3z(a) * L;
}

static hc_status build_batch(const hc_instance* inst, int n, hc_dtype dt, BatchPlan* plan,
                             std::vector<BatchDesc>* descs, void* workspace) {
  if (n < 0 || (n > 0 && !inst)) return HC_ERR_ARG;
  const size_t es = elem_size(dt);
  if (es == 0) return HC_ERR_DTYPE;
  const int cmax = batch_cmax(dt);
  const int L = dt == HC_FP32 ? 32 : 16;
  BatchPlan p;
  memset(&p, 0, sizeof(p));
  p.dtype = dt;
  p.n = n;
  size_t off = kWsHeader;
  p.off_ctr = off;
  off = align_up(off + 8 * (size_t)(n + 1), 256);
  p.off_desc = off;
  off = align_up(off + sizeof(BatchDesc) * (size_t)n, 256);
  p.off_w = off;
  long long ticket = 0;
  size_t smem = 0;
  if (descs) descs->resize(n);
  for (int i = 0; i < n; ++i) {
    const hc_instance& q = inst[i];
    if (q.D < 0 || q.D > cmax + 6) return HC_ERR_ARG;
    if (!q.x || !q.y || !q.z) return HC_ERR_ARG;
    if (!aligned(q.x, 16) || !aligned(q.y, 16) || !aligned(q.z, 16)) return HC_ERR_ALIGN;
    const size_t nx = es << q.D, nz = es * pow3z(q.D);
    if (overlaps(q.z, nz, q.x, nx) || overlaps(q.z, nz, q.y, nx)) return HC_ERR_ALIAS;
    BatchDesc d;
    memset(&d, 0, sizeof(d));
    d.x = q.x;
    d.y = q.y;
    d.z = q.z;
    d.w = q.z;
    d.D = q.D;
    d.C = q.D < cmax ? q.D : cmax;
    d.a = q.D - d.C;
    d.n_tiles = (int)pow3z(d.a);
    d.n_cols = d.a > 0 ? (int)((pow3z(d.C) + L - 1) / L) : 0;
    d.first = ticket;
    d.need = d.n_tiles;
    ticket += d.n_tiles + d.n_cols;
    if (dt == HC_FP32_MIXED && d.a > 0) {
      d.w = (unsigned char*)workspace + off;  // may be NULL while sizing
      off = align_up(off + 8 * pow3z(q.D), 256);
    }
    size_t s = tile_smem_bytes(dt, d.C);
    if (interp_smem_bytes(dt, d.a) > s) s = interp_smem_bytes(dt, d.a);
    if (s > smem) smem = s;
    if (descs) (*descs)[i] = d;
  }
  p.total = ticket;
  p.smem = smem;
  p.ws_bytes = off;
  *plan = p;
  return HC_OK;
}

template <class M>
static cudaError_t launch_batched_m(const BatchPlan& p, unsigned char* ws, cudaStream_t st) {
  auto k = batched_kernel<M>;
  ProfileScope prof(st, "batched");
  cudaError_t e = prep_kernel(k, p.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, p.smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)device_caps().sms * per_sm;
  if (grid > p.total) grid = p.total;
  if (grid < 1) grid = 1;
  k<<<(unsigned)grid, 256, p.smem, st>>>((const BatchDesc*)(ws + p.off_desc), p.n, p.total,
                                           (unsigned long long*)(ws + p.off_ctr), (WsHeader*)ws);
  return cudaGetLastError();
}

static hc_status batched_launch_plan(const BatchPlan& p, void* workspace, cudaStream_t st) {
  if (p.n == 0 || p.total == 0) return HC_OK;
  unsigned char* ws = (unsigned char*)workspace;
  cudaError_t e = cudaMemsetAsync(ws, 0, kWsHeader, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + p.off_ctr, 0, 8 * (size_t)(p.n + 1), st);
  if (e != cudaSuccess) return record_cuda_error(e);
  switch (p.dtype) {
    case HC_INT64: e = launch_batched_m<ModeI64>(p, ws, st); break;
    case HC_FP64: e = launch_batched_m<ModeF64>(p, ws, st); break;
    case HC_FP32: e = launch_batched_m<ModeF32>(p, ws, st); break;
    case HC_FP32_MIXED: e = launch_batched_m<ModeMixed>(p, ws, st); break;
  }
  return record_cuda_error(e);
}

}  // namespace hc

extern "C" size_t hc_batched_workspace_size(const hc_instance* inst, int n, hc_dtype dtype) {
  hc::BatchPlan p;
  if (hc::build_batch(inst, n, dtype, &p, nullptr, nullptr) != HC_OK) return 0;
  return p.ws_bytes;
}

extern "C" hc_status hc_batched_prepare(const hc_instance* inst, int n, hc_dtype dtype,
                                        void* workspace, size_t ws_bytes, hc_stream_t stream) {
  using namespace hc;
  BatchPlan p;
  hc_status s = build_batch(inst, n, dtype, &p, nullptr, nullptr);
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
  std::vector<BatchDesc> descs;
  s = build_batch(inst, n, dtype, &p, &descs, workspace);
  if (s != HC_OK) return s;
  if (n > 0) {
    cudaError_t e = cudaMemcpyAsync((unsigned char*)workspace + p.off_desc, descs.data(),
                                    sizeof(BatchDesc) * (size_t)n, cudaMemcpyHostToDevice,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return record_cuda_error(e);
  }
  std::lock_guard<std::mutex> g(g_plans_mu);
  g_plans[workspace] = p;
  return HC_OK;
}

extern "C" hc_status hc_batched_launch(void* workspace, size_t ws_bytes, hc_stream_t stream) {
  using namespace hc;
  if (!workspace) return HC_ERR_ARG;
  BatchPlan p;
  {
    std::lock_guard<std::mutex> g(g_plans_mu);
    auto it = g_plans.find(workspace);
    if (it == g_plans.end()) return HC_ERR_ARG;
    p = it->second;
  }
  if (ws_bytes < p.ws_bytes) return HC_ERR_WORKSPACE;
  return batched_launch_plan(p, workspace, (cudaStream_t)stream);
}

extern "C" hc_status hc_batched_inject_stall(void* workspace, int instance) {
  using namespace hc;
  if (!workspace) return HC_ERR_ARG;
  BatchPlan p;
  {
    std::lock_guard<std::mutex> g(g_plans_mu);
    auto it = g_plans.find(workspace);
    if (it == g_plans.end()) return HC_ERR_ARG;
    p = it->second;
  }
  if (instance < 0 || instance >= p.n) return HC_ERR_ARG;
  unsigned char* d = (unsigned char*)workspace + p.off_desc + sizeof(BatchDesc) * (size_t)instance;
  BatchDesc desc;
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
