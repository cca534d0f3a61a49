// A value looked up once per device and then read without locking: kernel
// occupancy, the device address of a file-scope array, the SM count. The
// entry points on device tensors may run from several host threads at once,
// so the first lookup on a device is serialised by a mutex while every later
// read is one atomic load. Host code only; no CUDA types, so that the
// thread-safety test can build it without the CUDA toolkit.
#pragma once
#include <atomic>
#include <mutex>

namespace ss {

class DeviceCache {
 public:
  static constexpr int MAXDEV = 64;

  // *out = the value cached for device `dev` (0 means "none yet"). When there
  // is none, init(&v) runs once under the lock; it returns 0 and sets a
  // nonzero v, or returns its nonzero error code, which is passed back and
  // caches nothing (the next call tries again). Returns -1 for a device index
  // outside [0, MAXDEV).
  template <class Init>
  int get(int dev, long long* out, Init&& init) {
    if (dev < 0 || dev >= MAXDEV) return -1;
    long long v = val_[dev].load(std::memory_order_acquire);
    if (v == 0) {
      std::lock_guard<std::mutex> lock(mu_);
      v = val_[dev].load(std::memory_order_relaxed);
      if (v == 0) {
        const int rc = init(&v);
        if (rc != 0) return rc;
        if (v == 0) return -1;
        val_[dev].store(v, std::memory_order_release);
      }
    }
    *out = v;
    return 0;
  }

 private:
  std::atomic<long long> val_[MAXDEV] = {};
  std::mutex mu_;
};

}  // namespace ss
