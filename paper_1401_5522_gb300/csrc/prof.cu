// Launch profiler of the library: when enabled, every kernel launch is bracketed by
// CUDA events recorded on its own stream and attributed to the kernel's name.  In trace
// mode each launch's start and end are also kept, relative to an event recorded when
// tracing was switched on, with the stream it ran on.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "../../include/luqr.h"
#include "internal.cuh"

namespace luqr {
namespace {
struct Rec {
  int id;
  cudaEvent_t e0, e1;
  cudaStream_t s;
};
struct TraceRec {
  int id;
  float t0, t1;
  cudaStream_t s;
};
bool g_trace = false;
std::set<std::string> g_select;   // when non-empty, only these kernels get events
cudaEvent_t g_base = nullptr;
std::vector<TraceRec> g_trace_recs;
constexpr size_t kMaxTrace = 4u << 20;
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
    if (cudaEventSynchronize(r.e1) == cudaSuccess && cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
      g_ms[r.id] += ms;
      float t0 = 0.f;
      if (g_trace && g_base && g_trace_recs.size() < kMaxTrace &&
          cudaEventElapsedTime(&t0, g_base, r.e0) == cudaSuccess)
        g_trace_recs.push_back(TraceRec{r.id, t0, t0 + ms, r.s});
    }
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
  if (!g_select.empty() && g_select.count(g_names[id]) == 0) {
    g_launches[id] += 1;   // counted, not timed
    t_open = -1;
    return;
  }
  if (g_recs.size() >= 200000) drain_locked();   // bound the number of live events
  Rec r{id, take_event(), take_event(), s};
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
  if (enable < 0 || enable > 2) return LUQR_ERR_INVALID;
  if (reset) {
    luqr::drain_locked();
    std::fill(luqr::g_launches.begin(), luqr::g_launches.end(), 0);
    std::fill(luqr::g_ms.begin(), luqr::g_ms.end(), 0.0);
    luqr::g_trace_recs.clear();
  }
  if (enable == 2 && !luqr::g_trace) {
    luqr::drain_locked();
    if (!luqr::g_base && cudaEventCreate(&luqr::g_base) != cudaSuccess) return LUQR_ERR_CUDA;
    if (cudaEventRecord(luqr::g_base, 0) != cudaSuccess) return LUQR_ERR_CUDA;
    luqr::g_trace_recs.clear();
  }
  luqr::g_trace = enable == 2;
  luqr::g_enabled = enable != 0;
  return LUQR_OK;
}

extern "C" int luqr_profile_select(const char* const* names, int count) {
  std::lock_guard<std::mutex> lk(luqr::g_mtx);
  if (count < 0 || (count > 0 && names == nullptr)) return LUQR_ERR_INVALID;
  luqr::g_select.clear();
  for (int i = 0; i < count; ++i)
    if (names[i]) luqr::g_select.insert(names[i]);
  return LUQR_OK;
}

extern "C" int luqr_profile_trace(const char** names, float* t0_ms, float* t1_ms,
                                  uint64_t* stream, int64_t cap) {
  std::lock_guard<std::mutex> lk(luqr::g_mtx);
  luqr::drain_locked();
  const int64_t n = std::min<int64_t>(cap, (int64_t)luqr::g_trace_recs.size());
  for (int64_t i = 0; i < n; ++i) {
    const luqr::TraceRec& r = luqr::g_trace_recs[(size_t)i];
    if (names) names[i] = luqr::g_names[r.id].c_str();
    if (t0_ms) t0_ms[i] = r.t0;
    if (t1_ms) t1_ms[i] = r.t1;
    if (stream) stream[i] = (uint64_t)(uintptr_t)r.s;
  }
  return (int)std::min<int64_t>((int64_t)luqr::g_trace_recs.size(), INT32_MAX);
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
