// Runs under ThreadSanitizer: (1) the per-device lookup cache of the library
// (csrc/ss_devcache.h, used for the status word and the static array
// addresses and the resident-CTA counts of the persistent kernels) hammered
// from many threads, with first lookups racing each other and a lookup that
// fails once; (2) the host planner and the public entry points on device
// tensors (device launchers stubbed: "no device") from several threads at
// once, as the header allows. Prints "ok" on success.
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <thread>
#include <vector>

#include "../../include/spinsum.h"
#include "../../paper_1705_06661_gb300/csrc/ss_devcache.h"

extern "C" int ss_debug_plan(int d, int O, int V, const double* coef, int nfactors, int mode, double alpha,
                             double beta, double* expanded, int64_t* info, int* ci, int* mp);

int main() {
  int bad = 0;
  // (1) the cache: 16 threads x 8 devices x 200 reads, init once per device
  {
    ss::DeviceCache cache;
    std::atomic<int> inits[8];
    std::atomic<int> fails{0};
    for (auto& x : inits) x = 0;
    std::atomic<int> wrong{0};
    std::vector<std::thread> th;
    for (int t = 0; t < 16; t++)
      th.emplace_back([&, t] {
        for (int it = 0; it < 200; it++) {
          const int dev = (t + it) % 8;
          long long v = 0;
          const int rc = cache.get(dev, &v, [&](long long* val) {
            if (dev == 5 && fails.fetch_add(1) == 0) return 7;  // the first lookup on device 5 fails
            inits[dev].fetch_add(1);
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            *val = 1000 + dev;
            return 0;
          });
          if (rc == 7) continue;
          if (rc != 0 || v != 1000 + dev) wrong.fetch_add(1);
        }
      });
    for (auto& x : th) x.join();
    for (int dev = 0; dev < 8; dev++)
      if (inits[dev].load() != 1) {
        std::printf("FAIL device %d initialised %d times\n", dev, inits[dev].load());
        bad = 1;
      }
    if (wrong.load()) {
      std::printf("FAIL %d wrong reads\n", wrong.load());
      bad = 1;
    }
    long long v = 0;
    if (cache.get(64, &v, [](long long*) { return 0; }) != -1) bad = 1;
  }
  // (2) planner and entry points from 8 threads
  {
    std::atomic<int> wrong{0};
    std::vector<std::thread> th;
    for (int t = 0; t < 8; t++)
      th.emplace_back([&, t] {
        double ex[24];
        int64_t info[32];
        std::vector<int> ci(8 * 24), mp(501);
        std::vector<double> c24(24), c6 = {4, -2, -2, 1, 1, -2};
        for (int k = 0; k < 24; k++) c24[k] = (double)((k * 7 + t) % 5 - 2);
        double A[4096] = {0}, B[4096] = {0};
        int64_t ext[6] = {2, 2, 2, 3, 3, 3}, ld[6] = {1, 2, 4, 8, 24, 72};
        for (int it = 0; it < 40; it++) {
          const int d = 3 + (it + t) % 2;
          const int rc = ss_debug_plan(d, 3 + it % 7, 1 + it % 5, d == 3 ? c6.data() : c24.data(), 1, it % 2, 1.0,
                                       it % 3 ? 0.0 : 1.0, ex, info, ci.data(), mp.data());
          if (rc != SPINSUM_OK) wrong.fetch_add(1);
          // a valid call without a device fails cleanly with this thread's message
          const int r2 = spinsum_3d(SPINSUM_F64, ext, A, ld, B, ld, c6.data(), 1, 0, 1.0, 0.0, 0, nullptr);
          if (r2 == SPINSUM_OK || spinsum_last_error()[0] == 0) wrong.fetch_add(1);
          int64_t bad_ext[6] = {2, 2, 2, 3, 3, 4};
          if (spinsum_3d(SPINSUM_F64, bad_ext, A, ld, B, ld, c6.data(), 1, 0, 1.0, 0.0, 0, nullptr) != SPINSUM_ERR_ARG)
            wrong.fetch_add(1);
        }
      });
    for (auto& x : th) x.join();
    if (wrong.load()) {
      std::printf("FAIL %d unexpected results from concurrent planner calls\n", wrong.load());
      bad = 1;
    }
  }
  std::printf(bad ? "failed\n" : "ok\n");
  return bad;
}
