// device_once.h -- thread-safe one-time setup per CUDA device for the kernel launchers (internal).
#pragma once

#include <cuda_runtime.h>

#include <mutex>

namespace ck {

constexpr int MAX_DEVICES = 64;

// run(init) calls init(device) for the current device until one call succeeds; later calls on that device
// return cudaSuccess at once.  Values init stores per device may be read after run() returned success.
class DeviceOnce {
  public:
    template <typename F>
    cudaError_t run(F &&init) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lock(mu_);
        if (done_[dev]) return cudaSuccess;
        e = init(dev);
        done_[dev] = e == cudaSuccess;
        return e;
    }

  private:
    std::mutex mu_;
    bool done_[MAX_DEVICES] = {};
};

}  // namespace ck
