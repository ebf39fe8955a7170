// Batching form: many independent hypercube convolutions of uneven D in one
// persistent launch.
//
// Each instance is one unit of the persistent ticket engine (hc_persist.cuh):
// C = min(D, tile axes), m = D - C <= 6 middle axes evaluated on the fly;
// 3^m tile tickets, then column tickets interpolating the middle axes while
// the instance's 3^D intermediate (<= 19 MB for D = 14 float32) is in L2.
// The host builds one descriptor per instance and a ticket -> (instance,
// local ticket) table in the interleaved order of hc_persist.cuh, so a CTA
// finds its work with a single load.
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
// Host side.

struct BatchPlan {
  hc_dtype dtype;
  int n;
  long long total;
  size_t smem;
  size_t off_ctr, off_desc, off_tab, off_w, ws_bytes;
};

static std::mutex g_plans_mu;
static std::map<const void*, BatchPlan> g_plans;  // prepared workspaces

static int batch_cmax(hc_dtype dt) { return dt == HC_FP32 ? 9 : 8; }

static hc_status build_batch(const hc_instance* inst, int n, hc_dtype dt, BatchPlan* plan,
                             std::vector<UnitDesc>* descs, std::vector<int2>* table,
                             void* workspace) {
  if (n < 0 || (n > 0 && !inst)) return HC_ERR_ARG;
  const size_t es = elem_size(dt);
  if (es == 0) return HC_ERR_DTYPE;
  const int cmax = batch_cmax(dt);
  const size_t wsz = (dt == HC_FP32_MIXED) ? 8 : es;
  const int L = kPersistCols;
  BatchPlan p;
  memset(&p, 0, sizeof(p));
  p.dtype = dt;
  p.n = n;
  long long ticket = 0;
  size_t smem = 0, wbytes = 0;
  if (descs) descs->resize(n);
  for (int i = 0; i < n; ++i) {
    const hc_instance& q = inst[i];
    if (q.D < 0 || q.D > cmax + 6) return HC_ERR_ARG;
    if (!q.x || !q.y || !q.z) return HC_ERR_ARG;
    if (!aligned(q.x, 16) || !aligned(q.y, 16) || !aligned(q.z, 16)) return HC_ERR_ALIGN;
    const size_t nx = es << q.D, nz = es * pow3z(q.D);
    if (overlaps(q.z, nz, q.x, nx) || overlaps(q.z, nz, q.y, nx)) return HC_ERR_ALIAS;
    UnitDesc d;
    memset(&d, 0, sizeof(d));
    d.x = q.x;
    d.y = q.y;
    d.z = q.z;
    d.w = q.z;
    // 8-axis tiles keep the persistent kernel at several CTAs per SM (a
    // 9-axis float32 tile needs 126 KB of shared memory); 9 only when D = 15.
    const int ctile = q.D > 8 + 6 ? cmax : 8;
    d.C = q.D < ctile ? q.D : ctile;
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
    if (dt == HC_FP32_MIXED && d.m > 0) {
      d.w = (void*)(uintptr_t)wbytes;  // offset for now; rebased below
      wbytes = align_up(wbytes + 8 * pow3z(q.D), 256);
    }
    size_t s = d.C > 0 ? tile_smem_bytes(dt, d.C) : 0;
    const size_t ism = d.m >= 4 ? 2 * wsz * pow3z(d.m) * L : 0;
    if (ism > s) s = ism;
    if (s > smem) smem = s;
    if (descs) (*descs)[i] = d;
  }
  p.total = ticket;
  p.smem = smem;
  size_t off = kWsHeader;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  p.off_ctr = take(8 * (size_t)(n + 1));
  p.off_desc = take(sizeof(UnitDesc) * (size_t)n);
  p.off_tab = take(sizeof(int2) * (size_t)ticket);
  p.off_w = take(wbytes);
  p.ws_bytes = off;
  if (descs && workspace && dt == HC_FP32_MIXED) {
    for (auto& d : *descs)
      if (d.m > 0) d.w = (unsigned char*)workspace + p.off_w + (uintptr_t)d.w;
  }
  if (table) {
    // tiles(0), tiles(1), cols(0), tiles(2), cols(1), ..., cols(n - 1)
    table->clear();
    table->reserve((size_t)ticket);
    const std::vector<UnitDesc>& ds = *descs;
    if (n > 0)
      for (int t = 0; t < ds[0].n_tiles; ++t) table->push_back(make_int2(0, t));
    for (int i = 0; i < n; ++i) {
      if (i + 1 < n)
        for (int t = 0; t < ds[i + 1].n_tiles; ++t) table->push_back(make_int2(i + 1, t));
      for (int c = 0; c < ds[i].n_cols; ++c)
        table->push_back(make_int2(i, ds[i].n_tiles + c));
    }
  }
  *plan = p;
  return HC_OK;
}

template <class M>
static cudaError_t launch_batched_m(const BatchPlan& p, unsigned char* ws, cudaStream_t st) {
  auto k = batched_kernel<M>;
  ProfileScope prof(st, "batched");
  cudaError_t e = prep_kernel(k, p.smem);
  if (e != cudaSuccess) return e;
  k<<<grid_for(k, 256, p.smem, p.total), 256, p.smem, st>>>(
      (const UnitDesc*)(ws + p.off_desc), (const int2*)(ws + p.off_tab), p.total,
      (unsigned long long*)(ws + p.off_ctr), (WsHeader*)ws);
  return cudaGetLastError();
}

static hc_status batched_launch_plan(const BatchPlan& p, void* workspace, cudaStream_t st) {
  if (p.n == 0 || p.total == 0) return HC_OK;
  unsigned char* ws = (unsigned char*)workspace;
  // status word and counters are contiguous from the start of the workspace
  cudaError_t e = cudaMemsetAsync(ws, 0, p.off_ctr + 8 * (size_t)(p.n + 1), st);
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
  if (hc::build_batch(inst, n, dtype, &p, nullptr, nullptr, nullptr) != HC_OK) return 0;
  return p.ws_bytes;
}

extern "C" hc_status hc_batched_prepare(const hc_instance* inst, int n, hc_dtype dtype,
                                        void* workspace, size_t ws_bytes, hc_stream_t stream) {
  using namespace hc;
  BatchPlan p;
  hc_status s = build_batch(inst, n, dtype, &p, nullptr, nullptr, nullptr);
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
  s = build_batch(inst, n, dtype, &p, &descs, &table, workspace);
  if (s != HC_OK) return s;
  if (n > 0) {
    cudaError_t e = cudaMemcpyAsync((unsigned char*)workspace + p.off_desc, descs.data(),
                                    sizeof(UnitDesc) * (size_t)n, cudaMemcpyHostToDevice,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess && !table.empty())
      e = cudaMemcpyAsync((unsigned char*)workspace + p.off_tab, table.data(),
                          sizeof(int2) * table.size(), cudaMemcpyHostToDevice,
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
  unsigned char* d = (unsigned char*)workspace + p.off_desc + sizeof(UnitDesc) * (size_t)instance;
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
