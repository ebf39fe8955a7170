// Forward plan shared between the plain, no-allocation and batched paths.
#pragma once

#include "hc_common.cuh"

namespace hc {

struct FwdPlan {
  int D;
  hc_dtype dtype;
  int C;  // inner axes handled inside one tile
  int a;  // outer axes handled by whole-array passes
  int n_eval;
  int eval_d0[HC_MAX_D], eval_k[HC_MAX_D];
  bool eval_to_final[HC_MAX_D];
  int n_interp;
  int interp_d0[HC_MAX_D], interp_k[HC_MAX_D];
  size_t off_xo, off_yo, off_tx, off_ty, off_w;
  size_t ws_bytes;
  int cols;        // columns per whole-array interpolation tile (0 = default)
  int cols_outer;  // the same for the pass over the outermost axes (0 = cols)
  // HC_SCHED_PADDED: the intermediate in the workspace with a 128-byte tile
  // pitch (off_w, 3^a * pitch elements), so that every row of the passes is
  // aligned; the last pass writes z's own layout
  bool padded;
  long long pitch;
};

// The default schedule ("chunked"): the a' = D - C - m outermost axes are
// evaluated by whole-array passes, then one persistent launch convolves the
// 3^a' chunks of C + m axes (tiles of C axes, m <= 6 middle axes
// interpolated while the chunk is in L2), then whole-array passes
// interpolate the a' outer axes.  For D <= C + 6 it is a single launch.
struct ChunkPlan {
  int D;
  hc_dtype dtype;
  int C, m, ap;
  int m_pre;  // middle axes evaluated by the whole-array passes (with the a' outer axes)
  int n_eval;
  int eval_d0[HC_MAX_D], eval_k[HC_MAX_D];
  bool eval_to_final[HC_MAX_D];
  int n_interp;
  int interp_d0[HC_MAX_D], interp_k[HC_MAX_D];
  long long units, per_unit, total;
  int n_tiles, n_cols, cpt, L;
  size_t smem;
  size_t off_ctr, off_xo, off_yo, off_tx, off_ty, off_w;
  size_t ws_bytes;
  int cols;        // columns per whole-array interpolation tile (0 = default)
  int cols_outer;  // the same for the pass over the outermost axes (0 = cols)
  bool bulk;       // chunked-bulk: every middle axis pre-evaluated, slab kernel
};

// c_req: tile axes (0 = default); m_req: middle axes per chunk (0 = default);
// bulk: the chunked-bulk variant (all m middle axes evaluated by the
// whole-array passes, tiles stored by bulk copies).
ChunkPlan make_chunk_plan(int D, hc_dtype dt, int c_req, int m_req, bool bulk = false);

cudaError_t chunk_forward_i64(const ChunkPlan& p, const void* x, const void* y, void* z,
                              unsigned char* ws, cudaStream_t st, void* w = nullptr);
cudaError_t chunk_forward_f64(const ChunkPlan& p, const void* x, const void* y, void* z,
                              unsigned char* ws, cudaStream_t st, void* w = nullptr);
cudaError_t chunk_forward_f32(const ChunkPlan& p, const void* x, const void* y, void* z,
                              unsigned char* ws, cudaStream_t st, void* w = nullptr);
cudaError_t chunk_forward_mix(const ChunkPlan& p, const void* x, const void* y, void* z,
                              unsigned char* ws, cudaStream_t st, void* w = nullptr);
cudaError_t chunk_forward_ff(const ChunkPlan& p, const void* x, const void* y, void* z,
                             unsigned char* ws, cudaStream_t st, void* w = nullptr);

// The hybrid schedule (hc_hybrid.cu): direct form on the top mt axes.
struct HybPlan {
  int D, mt, C, a;
  hc_dtype dtype;
  int n_eval;
  int eval_d0[HC_MAX_D], eval_k[HC_MAX_D];
  bool eval_to_final[HC_MAX_D];
  int n_interp;
  int interp_d0[HC_MAX_D], interp_k[HC_MAX_D];
  size_t off_xo, off_yo, off_tx, off_ty;
  size_t ws_bytes;
  int cols, cols_outer;
  bool ok;  // false: mt outside 1..6 or fewer than 4 tile axes left
};
HybPlan make_hybrid_plan(int D, hc_dtype dt, int mt, int c_req, int kmax_req);
bool hybrid_dtype_ok(hc_dtype dt);
cudaError_t hybrid_dispatch(const HybPlan& p, const void* x, const void* y, void* z,
                            unsigned char* ws, cudaStream_t st, void* w);

// The low-workspace schedule (hc_lowmem.cu): the top r axes leaf by leaf.
struct LowPlan {
  int D, r;
  hc_dtype dtype;
  FwdPlan leaf;  // the plan every leaf of D - r axes runs
  int n_top;
  int top_d0[6], top_k[6];
  int cols_top;
  size_t off_xl, off_yl, off_leaf;
  size_t ws_bytes;
  bool ok;  // false: r outside 1..6, D - r < 1, or a float-float dtype
};
LowPlan make_lowmem_plan(int D, hc_dtype dt, int r, int c_req, int kmax_req, int cols,
                         int cols_outer);
cudaError_t lowmem_dispatch(const LowPlan& p, const void* x, const void* y, void* z,
                            unsigned char* ws, cudaStream_t st, void* w);

// c_req, kmax_req <= 0 select the defaults (largest tile, 6 axes per pass).
FwdPlan make_fwd_plan(int D, hc_dtype dt, int c_req, int kmax_req, bool padded = false);

cudaError_t forward_dispatch(const FwdPlan& p, const void* x, const void* y, void* z,
                             unsigned char* ws, cudaStream_t st, void* w = nullptr);

// Validated schedule with kind resolved (1 = passes, 2 = chunked).
bool schedule_valid(const hc_schedule& s, hc_dtype dtype);
hc_schedule resolve_schedule(int D, hc_dtype dtype, const hc_schedule* s);
size_t schedule_ws(int D, hc_dtype dtype, const hc_schedule& s);

// w: the caller's device array for the 3^D intermediate (nullptr: the
// intermediate lives in z, or in the workspace for HC_FP32_MIXED); with w,
// z is written only by the final stores.
hc_status convolve_checked(const void* x, const void* y, void* z, int D, hc_dtype dtype,
                           void* workspace, size_t ws_bytes, cudaStream_t stream,
                           const hc_schedule* sched, void* w = nullptr);

}  // namespace hc
