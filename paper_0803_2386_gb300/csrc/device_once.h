// device_once.h -- per-device one-time set-up of the library's kernels.
//
// A kernel's function attributes (its dynamic shared-memory limit, its
// carveout) are set for the device that is current when they are set, and
// the grid of a persistent kernel is sized from that device's SM count and
// occupancy.  A process that runs plans on two GPUs therefore needs the
// set-up once per device, not once per process, and host threads that
// launch at the same time must not race on it.  DeviceOnce keeps one value
// per device ordinal, computed once under a mutex; a failed set-up is not
// cached, so the next call tries again.
//
// Pure C++ (no CUDA types), so the logic is tested on the host.
#pragma once

#include <atomic>
#include <mutex>

namespace moafft {

constexpr int kMaxDevices = 64;

struct DeviceOnce {
    std::mutex mu;
    std::atomic<bool> done[kMaxDevices] = {};
    long long value[kMaxDevices] = {};
};

// The value init(dev, &value) computed for device ordinal `dev`, running init
// only the first time for that ordinal.  init returns 0 on success; any other
// code is returned as it is and nothing is recorded.  Returns -1 for an
// ordinal outside 0..kMaxDevices-1.
template <typename F>
int device_once(DeviceOnce &d, int dev, long long *value, F &&init)
{
    if (dev < 0 || dev >= kMaxDevices) return -1;
    if (!d.done[dev].load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lk(d.mu);
        if (!d.done[dev].load(std::memory_order_relaxed)) {
            long long v = 0;
            const int code = init(dev, &v);
            if (code != 0) return code;
            d.value[dev] = v;
            d.done[dev].store(true, std::memory_order_release);
        }
    }
    if (value) *value = d.value[dev];
    return 0;
}

}  // namespace moafft
