// tel_once.cuh -- one-time, per-device host set-up of a kernel attribute.
//
// Kernel attributes such as the dynamic shared-memory limit are set per
// device context, so "done once" is recorded per device (devices 0-63; a
// device beyond that sets the attribute on every launch).  Setting an
// attribute twice is harmless, so two threads racing on the first launch
// need no lock.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

namespace tel {

class DeviceOnce {
public:
    template <typename Fn>
    cudaError_t run(Fn fn)
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
        if (bit && (done_.load(std::memory_order_acquire) & bit)) return cudaSuccess;
        e = fn();
        if (e == cudaSuccess && bit) done_.fetch_or(bit, std::memory_order_release);
        return e;
    }

private:
    std::atomic<unsigned long long> done_{0};
};

}  // namespace tel
