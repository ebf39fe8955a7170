// Chunked forward schedule, ModeFF instantiation.
#include "hc_chunk_impl.cuh"

namespace hc {

cudaError_t chunk_forward_ff(const ChunkPlan& p, const void* x, const void* y, void* z,
                             unsigned char* ws, cudaStream_t st, void* w) {
  return chunk_forward_m<ModeFF>(p, x, y, z, ws, st, w);
}

}  // namespace hc
