// Host-side record of the dynamic shared-memory limit raised for one kernel, per device.
// cudaFuncSetAttribute acts on the current device only, so each device keeps its own value
// (devices 0 .. kDevices-1; others are not recorded and get the attribute set on every
// launch that needs more than the default).  Shared by the host threads under a lock.
// Header-only and free of CUDA types so that its bookkeeping can be checked on the host.
#pragma once

#include <cstddef>
#include <mutex>

namespace luqr {

struct SmemRecord {
  static constexpr int kDevices = 64;
  static constexpr size_t kDefault = 48 * 1024;   // the limit every kernel starts with
  std::mutex mu;
  size_t cur[kDevices] = {};                      // 0: the default

  // Calls set(bytes) (which returns true on success) when `bytes` exceeds the limit
  // recorded for device `dev`, and records it on success.  Returns false only when the
  // limit had to be raised and set() failed.
  template <class Set>
  bool ensure(int dev, size_t bytes, Set&& set) {
    if (dev < 0 || dev >= kDevices) return bytes <= kDefault || set(bytes);
    std::lock_guard<std::mutex> lk(mu);
    const size_t have = cur[dev] ? cur[dev] : kDefault;
    if (bytes <= have) return true;
    if (!set(bytes)) return false;
    cur[dev] = bytes;
    return true;
  }
};

}  // namespace luqr
