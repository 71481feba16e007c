// Launch profiler of the library: when enabled, every kernel launch is bracketed by
// CUDA events recorded on its own stream and attributed to the kernel's name.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/luqr.h"
#include "internal.cuh"

namespace luqr {
namespace {
struct Rec {
  int id;
  cudaEvent_t e0, e1;
};
std::mutex g_mtx;
bool g_enabled = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
std::vector<std::string> g_names;
std::map<std::string, int> g_ids;
std::vector<int64_t> g_launches;
std::vector<double> g_ms;
thread_local int t_open = -1;   // index of the record opened by prof_begin on this thread

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void drain_locked() {
  for (Rec& r : g_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.e1) == cudaSuccess && cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess)
      g_ms[r.id] += ms;
    g_launches[r.id] += 1;
    g_pool.push_back(r.e0);
    g_pool.push_back(r.e1);
  }
  g_recs.clear();
}
}  // namespace

void prof_begin(const char* name, cudaStream_t s) {
  if (!g_enabled) return;
  std::lock_guard<std::mutex> lk(g_mtx);
  auto it = g_ids.find(name);
  int id;
  if (it == g_ids.end()) {
    id = (int)g_names.size();
    g_ids[name] = id;
    g_names.push_back(name);
    g_launches.push_back(0);
    g_ms.push_back(0.0);
  } else {
    id = it->second;
  }
  if (g_recs.size() >= 200000) drain_locked();   // bound the number of live events
  Rec r{id, take_event(), take_event()};
  cudaEventRecord(r.e0, s);
  g_recs.push_back(r);
  t_open = (int)g_recs.size() - 1;
}

void prof_end(cudaStream_t s) {
  if (!g_enabled || t_open < 0) return;
  std::lock_guard<std::mutex> lk(g_mtx);
  if (t_open < (int)g_recs.size()) cudaEventRecord(g_recs[t_open].e1, s);
  t_open = -1;
}

}  // namespace luqr

extern "C" int luqr_profile(int enable, int reset) {
  std::lock_guard<std::mutex> lk(luqr::g_mtx);
  if (reset) {
    luqr::drain_locked();
    std::fill(luqr::g_launches.begin(), luqr::g_launches.end(), 0);
    std::fill(luqr::g_ms.begin(), luqr::g_ms.end(), 0.0);
  }
  luqr::g_enabled = enable != 0;
  return LUQR_OK;
}

extern "C" int luqr_profile_read(const char** names, int64_t* launches, double* total_ms, int cap) {
  std::lock_guard<std::mutex> lk(luqr::g_mtx);
  luqr::drain_locked();
  int n = 0;
  for (size_t i = 0; i < luqr::g_names.size() && n < cap; ++i) {
    if (luqr::g_launches[i] == 0) continue;
    if (names) names[n] = luqr::g_names[i].c_str();
    if (launches) launches[n] = luqr::g_launches[i];
    if (total_ms) total_ms[n] = luqr::g_ms[i];
    ++n;
  }
  return n;
}
