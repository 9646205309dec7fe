// Host test of the per-device set-up cache (device_once.h): compiled with
// g++ and run by tests/test_device_once_host.py; no CUDA involved.
#include <atomic>
#include <cstdio>
#include <thread>
#include <vector>

#include "device_once.h"

using moafft::DeviceOnce;
using moafft::device_once;

static int fails = 0;
#define CHECK(c)                                                     \
    do {                                                             \
        if (!(c)) {                                                  \
            std::fprintf(stderr, "line %d: %s\n", __LINE__, #c);     \
            fails++;                                                 \
        }                                                            \
    } while (0)

int main()
{
    // one set-up per ordinal, each with its own value
    {
        DeviceOnce d;
        int calls[4] = {0, 0, 0, 0};
        for (int rep = 0; rep < 3; rep++)
            for (int dev = 0; dev < 4; dev++) {
                long long v = -1;
                const int rc = device_once(d, dev, &v, [&](int devno, long long *out) -> int {
                    calls[devno]++;
                    *out = 100 + devno;
                    return 0;
                });
                CHECK(rc == 0);
                CHECK(v == 100 + dev);
            }
        for (int dev = 0; dev < 4; dev++) CHECK(calls[dev] == 1);
    }
    // a failed set-up is returned and not cached; the next call tries again
    {
        DeviceOnce d;
        int calls = 0;
        long long v = 0;
        int rc = device_once(d, 2, &v, [&](int, long long *out) -> int {
            calls++;
            *out = 7;
            return 9;
        });
        CHECK(rc == 9);
        rc = device_once(d, 2, &v, [&](int, long long *out) -> int {
            calls++;
            *out = 8;
            return 0;
        });
        CHECK(rc == 0 && v == 8 && calls == 2);
    }
    // ordinals outside the table are refused without calling init
    {
        DeviceOnce d;
        int calls = 0;
        auto init = [&](int, long long *) -> int {
            calls++;
            return 0;
        };
        CHECK(device_once(d, -1, nullptr, init) == -1);
        CHECK(device_once(d, moafft::kMaxDevices, nullptr, init) == -1);
        CHECK(device_once(d, moafft::kMaxDevices - 1, nullptr, init) == 0);
        CHECK(calls == 1);
    }
    // many host threads on a few devices at once: init runs once per device
    // and every thread sees that device's value
    {
        DeviceOnce d;
        std::atomic<int> calls[8];
        for (auto &c : calls) c = 0;
        std::atomic<int> wrong{0};
        std::vector<std::thread> th;
        for (int t = 0; t < 16; t++)
            th.emplace_back([&, t] {
                for (int i = 0; i < 2000; i++) {
                    const int dev = (t + i) % 8;
                    long long v = 0;
                    device_once(d, dev, &v, [&](int devno, long long *out) -> int {
                        calls[devno]++;
                        std::this_thread::yield();
                        *out = 1000 * (devno + 1);
                        return 0;
                    });
                    if (v != 1000 * (dev + 1)) wrong++;
                }
            });
        for (auto &x : th) x.join();
        for (int dev = 0; dev < 8; dev++) CHECK(calls[dev] == 1);
        CHECK(wrong == 0);
    }
    if (fails) return 1;
    std::printf("device_once ok\n");
    return 0;
}
