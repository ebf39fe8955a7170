// Chunked forward schedule, ModeI64 instantiation.
#include "hc_chunk_impl.cuh"

namespace hc {

cudaError_t chunk_forward_i64(const ChunkPlan& p, const void* x, const void* y, void* z,
                            unsigned char* ws, cudaStream_t st, void* w) {
  return chunk_forward_m<ModeI64>(p, x, y, z, ws, st, w);
}

}  // namespace hc
