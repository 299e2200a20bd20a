// Host-only check of the per-device set-up bookkeeping (csrc/per_device.h):
// each device index is set up exactly once, results are kept per device,
// concurrent callers agree, and an index out of range gets the fallback.
// Prints "ok" and exits 0 on success.
#include <atomic>
#include <cstdio>
#include <thread>
#include <vector>

#include "../../paper_2301_06763_gb300/csrc/per_device.h"

int main() {
    nm::PerDevice<int> pd;
    std::atomic<int> calls[nm::kMaxDevicesPerProcess];
    for (auto& c : calls) c.store(0);
    const int devices[] = {0, 1, 5, 63};
    std::vector<std::thread> ts;
    std::atomic<int> bad{0};
    for (int t = 0; t < 8; ++t)
        ts.emplace_back([&, t]() {
            for (int rep = 0; rep < 1000; ++rep)
                for (int d : devices) {
                    const int r = pd.get(d, [&]() { calls[d].fetch_add(1); return 100 + d; }, -1);
                    if (r != 100 + d) bad.fetch_add(1);
                }
            (void)t;
        });
    for (auto& th : ts) th.join();
    if (bad.load()) { std::printf("wrong result %d times\n", bad.load()); return 1; }
    for (int d = 0; d < nm::kMaxDevicesPerProcess; ++d) {
        const bool used = d == 0 || d == 1 || d == 5 || d == 63;
        if (calls[d].load() != (used ? 1 : 0)) {
            std::printf("device %d set up %d times\n", d, calls[d].load());
            return 1;
        }
        if (pd.ready(d) != used) { std::printf("device %d ready flag wrong\n", d); return 1; }
    }
    // a device set up later is independent of the earlier ones
    if (pd.get(2, []() { return 7; }, -1) != 7 || pd.get(2, []() { return 8; }, -1) != 7) {
        std::printf("second device kept the wrong result\n");
        return 1;
    }
    if (pd.get(-1, []() { return 9; }, -3) != -3 || pd.get(64, []() { return 9; }, -3) != -3) {
        std::printf("out-of-range index not rejected\n");
        return 1;
    }
    std::printf("ok\n");
    return 0;
}
