// Launch tracing hooks (see hc_profile_enable in hc.h).
#pragma once

#include <cuda_runtime.h>

namespace hc {

bool profile_on();
void profile_begin(cudaStream_t st, const char* name);
void profile_end(cudaStream_t st);

// Brackets one kernel launch with profile events when tracing is on.
struct ProfileScope {
  cudaStream_t st;
  ProfileScope(cudaStream_t s, const char* name) : st(s) { profile_begin(s, name); }
  ~ProfileScope() { profile_end(st); }
};

}  // namespace hc
