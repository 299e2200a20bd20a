// per_device.h -- one-time set-up that must be done once on every device.
//
// Kernel attributes (the dynamic shared-memory limit) and occupancy figures
// belong to a device, not to the process: a process that drives two GPUs must
// set a kernel's attribute with each device current before launching there.
// PerDevice<R> runs a set-up function the first time it is asked for a given
// device index and keeps its result (an error code, an occupancy, ...) per
// device; later calls for that device return the kept result without calling
// the function again.  Host-only and independent of CUDA, so its bookkeeping
// can be tested without a GPU.
#pragma once
#include <atomic>
#include <cstdint>
#include <mutex>

namespace nm {

constexpr int kMaxDevicesPerProcess = 64;

template <typename R> class PerDevice {
  public:
    // The result for device `dev` (0 <= dev < kMaxDevicesPerProcess), calling
    // make() once for that device; `fallback` is returned for an index out of
    // range.  Safe to call from several host threads at once: make() runs once
    // per device, under a lock; later reads take no lock.
    template <class F> R get(int dev, F&& make, R fallback) {
        if (dev < 0 || dev >= kMaxDevicesPerProcess) return fallback;
        const uint64_t bit = (uint64_t)1 << dev;
        if (ready_.load(std::memory_order_acquire) & bit) return res_[dev];
        std::lock_guard<std::mutex> lk(mu_);
        if (!(ready_.load(std::memory_order_relaxed) & bit)) {
            res_[dev] = make();
            ready_.fetch_or(bit, std::memory_order_release);
        }
        return res_[dev];
    }
    // Whether device `dev` has been set up.
    bool ready(int dev) const {
        return dev >= 0 && dev < kMaxDevicesPerProcess &&
               (ready_.load(std::memory_order_acquire) & ((uint64_t)1 << dev)) != 0;
    }

  private:
    std::atomic<uint64_t> ready_{0};
    std::mutex mu_;
    R res_[kMaxDevicesPerProcess]{};
};

}  // namespace nm
