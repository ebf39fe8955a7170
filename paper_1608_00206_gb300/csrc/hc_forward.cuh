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
};

// c_req, kmax_req <= 0 select the defaults (largest tile, 6 axes per pass).
FwdPlan make_fwd_plan(int D, hc_dtype dt, int c_req, int kmax_req);

cudaError_t forward_dispatch(const FwdPlan& p, const void* x, const void* y, void* z,
                             unsigned char* ws, cudaStream_t st);

hc_status convolve_checked(const void* x, const void* y, void* z, int D, hc_dtype dtype,
                           void* workspace, size_t ws_bytes, cudaStream_t stream, int c_req,
                           int kmax_req);

}  // namespace hc
