// Kernel tracing: when enabled, every kernel launch of the library is
// bracketed by a pair of CUDA events recorded on the launching stream, and
// hc_profile_collect() reports per-kernel launch counts and total device time.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hc_common.cuh"
#include "hc_profile.cuh"

namespace hc {

namespace {
struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
thread_local Rec* g_open = nullptr;
thread_local size_t g_open_idx = 0;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

bool profile_on() { return g_on; }

void profile_begin(cudaStream_t st, const char* name) {
  if (!g_on) return;
  std::lock_guard<std::mutex> g(g_mu);
  Rec r{name, get_event(), get_event()};
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  g_open_idx = g_recs.size() - 1;
  g_open = &g_recs.back();
}

void profile_end(cudaStream_t st) {
  if (!g_on || !g_open) return;
  std::lock_guard<std::mutex> g(g_mu);
  cudaEventRecord(g_recs[g_open_idx].b, st);
  g_open = nullptr;
}

}  // namespace hc

extern "C" hc_status hc_profile_enable(int on) {
  std::lock_guard<std::mutex> g(hc::g_mu);
  hc::g_on = on != 0;
  return HC_OK;
}

extern "C" int hc_profile_collect(char* names, int name_len, double* total_ms, int* counts,
                                  int max_kernels) {
  using namespace hc;
  std::lock_guard<std::mutex> g(g_mu);
  std::vector<std::string> keys;
  std::vector<double> ms;
  std::vector<int> cnt;
  for (Rec& r : g_recs) {
    cudaEventSynchronize(r.b);
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) t = 0.0f;
    size_t k = 0;
    while (k < keys.size() && keys[k] != r.name) ++k;
    if (k == keys.size()) {
      keys.push_back(r.name);
      ms.push_back(0.0);
      cnt.push_back(0);
    }
    ms[k] += t;
    cnt[k] += 1;
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  cudaGetLastError();  // clear a not-ready or invalid-handle status left by the queries
  const int n = (int)keys.size() < max_kernels ? (int)keys.size() : max_kernels;
  for (int i = 0; i < n; ++i) {
    if (names && name_len > 0) {
      strncpy(names + (size_t)i * name_len, keys[i].c_str(), name_len - 1);
      names[(size_t)i * name_len + name_len - 1] = 0;
    }
    if (total_ms) total_ms[i] = ms[i];
    if (counts) counts[i] = cnt[i];
  }
  return n;
}
