// Chunked forward schedule, ModeF64 instantiation.
#include "hc_chunk_impl.cuh"

namespace hc {

cudaError_t chunk_forward_f64(const ChunkPlan& p, const void* x, const void* y, void* z,
                            unsigned char* ws, cudaStream_t st, void* w) {
  return chunk_forward_m<ModeF64>(p, x, y, z, ws, st, w);
}

}  // namespace hc
