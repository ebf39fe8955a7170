// Chunked forward schedule, ModeF32 instantiation.
#include "hc_chunk_impl.cuh"

namespace hc {

cudaError_t chunk_forward_f32(const ChunkPlan& p, const void* x, const void* y, void* z,
                            unsigned char* ws, cudaStream_t st, void* w) {
  return chunk_forward_m<ModeF32>(p, x, y, z, ws, st, w);
}

}  // namespace hc
