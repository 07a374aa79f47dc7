// Load replay for the serving benchmark: Poisson arrivals at a given rate,
// through the continuous-batching engine or through one plain launch per
// request, with each latency counted from the request's scheduled arrival.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>
#include <chrono>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/utf16wf.h"
#include "internal.h"
#include "runtime.h"

namespace u16wf {

namespace {

// xoshiro256** (Blackman and Vigna) seeded by SplitMix64, for the arrival
// process only.
struct Rng {
    uint64_t s[4];
    explicit Rng(uint64_t seed) {
        uint64_t x = seed;
        for (int i = 0; i < 4; ++i) {
            uint64_t z = (x += 0x9E3779B97F4A7C15ull);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            s[i] = z ^ (z >> 31);
        }
    }
    static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
    uint64_t next() {
        const uint64_t r = rotl(s[1] * 5, 7) * 9, t = s[1] << 17;
        s[2] ^= s[0];
        s[3] ^= s[1];
        s[1] ^= s[2];
        s[0] ^= s[3];
        s[2] ^= t;
        s[3] = rotl(s[3], 45);
        return r;
    }
    double unit() { return (double)(next() >> 11) * 0x1.0p-53; }
};

std::vector<int64_t> arrival_times(int64_t count, double rate, uint64_t seed, int64_t start) {
    std::vector<int64_t> t((size_t)count);
    Rng rng(seed);
    double at = (double)start;
    for (int64_t i = 0; i < count; ++i) {
        if (rate > 0) at += -log(1.0 - rng.unit()) / rate * 1e9;
        t[(size_t)i] = (int64_t)at;
    }
    return t;
}

void wait_until(int64_t t_ns) {
    while (true) {
        const int64_t now = utf16_server_clock_ns();
        if (now >= t_ns) return;
        if (t_ns - now > 200000) std::this_thread::sleep_for(std::chrono::microseconds((t_ns - now) / 2000));
    }
}

}  // namespace

}  // namespace u16wf

using namespace u16wf;

extern "C" int utf16_server_replay(utf16_server *S, const uint16_t *const *inputs, uint16_t *const *outputs,
                                   const int64_t *lengths, int64_t count, double rate_per_s, uint64_t seed,
                                   double *latency_s, int64_t *first_bad) {
    if (!S || count < 0 || (count > 0 && (!inputs || !outputs || !lengths || !latency_s || !first_bad)))
        return UTF16_EINVAL;
    const int64_t start = utf16_server_clock_ns() + 1000000;
    const std::vector<int64_t> at = arrival_times(count, rate_per_s, seed, start);
    std::vector<uint64_t> ticket((size_t)count, 0);
    std::vector<utf16_completion> done;
    done.reserve((size_t)count);
    int64_t expected = 0;
    std::atomic<int64_t> submitted_ok{0};
    std::atomic<bool> submitting{true};
    int rc = UTF16_OK;
    std::thread collector([&] {
        while (true) {
            if (!submitting.load() && (int64_t)done.size() >= submitted_ok.load()) break;
            utf16_completion c;
            const int r = utf16_server_next(S, &c, 2000);
            if (r == UTF16_OK) done.push_back(c);
            else if (r != UTF16_ETIMEOUT && r != UTF16_EAGAIN) break;
        }
    });
    for (int64_t i = 0; i < count; ++i) {
        wait_until(at[(size_t)i]);
        const int r = utf16_server_submit(S, inputs[i], outputs[i], lengths[i], at[(size_t)i], &ticket[(size_t)i]);
        if (r != UTF16_OK) {
            ticket[(size_t)i] = 0;
            latency_s[i] = 0;
            first_bad[i] = r;
        } else {
            ++expected;
            submitted_ok.store(expected);
        }
    }
    submitting.store(false);
    collector.join();
    std::unordered_map<uint64_t, const utf16_completion *> by_ticket;
    for (const utf16_completion &c : done) by_ticket[c.ticket] = &c;
    for (int64_t i = 0; i < count; ++i) {
        if (!ticket[(size_t)i]) continue;
        auto it = by_ticket.find(ticket[(size_t)i]);
        if (it == by_ticket.end()) {
            first_bad[i] = UTF16_ETIMEOUT;
            latency_s[i] = 0;
            rc = UTF16_ETIMEOUT;
            continue;
        }
        const utf16_completion &c = *it->second;
        latency_s[i] = (double)(c.done_ns - c.arrival_ns) * 1e-9;
        first_bad[i] = c.status == UTF16_OK ? c.first_bad : c.status;
    }
    return rc;
}

extern "C" int utf16_plain_replay(const uint16_t *const *inputs, uint16_t *const *outputs, const int64_t *lengths,
                                  int64_t count, double rate_per_s, uint64_t seed, double *latency_s,
                                  int64_t *first_bad) {
    if (count < 0 || (count > 0 && (!inputs || !outputs || !lengths || !latency_s || !first_bad))) return UTF16_EINVAL;
    int64_t max_n = 1;
    for (int64_t i = 0; i < count; ++i) max_n = lengths[i] > max_n ? lengths[i] : max_n;
    uint16_t *d = nullptr;
    int64_t *d_first = nullptr, *h_first = nullptr;
    cudaStream_t s = nullptr;
    if (cudaMalloc((void **)&d, (size_t)max_n * 2u) != cudaSuccess ||
        cudaMalloc((void **)&d_first, sizeof(int64_t)) != cudaSuccess ||
        cudaHostAlloc((void **)&h_first, sizeof(int64_t), cudaHostAllocDefault) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        if (d) cudaFree(d);
        if (d_first) cudaFree(d_first);
        if (h_first) cudaFreeHost(h_first);
        return UTF16_ENOMEM;
    }
    int rc = UTF16_OK;
    const int64_t start = utf16_server_clock_ns() + 1000000;
    const std::vector<int64_t> at = arrival_times(count, rate_per_s, seed, start);
    for (int64_t i = 0; i < count && rc == UTF16_OK; ++i) {
        wait_until(at[(size_t)i]);
        const int64_t n = lengths[i];
        if (n > 0) {
            if (cudaMemcpyAsync(d, inputs[i], (size_t)n * 2u, cudaMemcpyHostToDevice, s) != cudaSuccess) rc = UTF16_ECUDA;
            if (rc == UTF16_OK) rc = run_single(d, d, n, kModeInPlace, d_first, s, 0, 0);
            if (rc == UTF16_OK &&
                (cudaMemcpyAsync(outputs[i], d, (size_t)n * 2u, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                 cudaMemcpyAsync(h_first, d_first, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                 cudaStreamSynchronize(s) != cudaSuccess))
                rc = UTF16_ECUDA;
            first_bad[i] = *h_first;
        } else {
            first_bad[i] = 0;
        }
        latency_s[i] = (double)(utf16_server_clock_ns() - at[(size_t)i]) * 1e-9;
    }
    cudaStreamSynchronize(s);
    cudaGetLastError();
    cudaStreamDestroy(s);
    cudaFree(d);
    cudaFree(d_first);
    cudaFreeHost(h_first);
    return rc;
}

// One plain launch per request, pipelined: `streams` host threads each own a
// stream, a device buffer and a pinned first-error cell.  Each takes the next
// request in arrival order, waits for its arrival time, and runs H2D, the
// fused in-place repair + first-error kernel and D2H on its stream, then waits
// for them; up to `streams` requests are in flight at once.
extern "C" int utf16_plain_replay_streams(const uint16_t *const *inputs, uint16_t *const *outputs,
                                          const int64_t *lengths, int64_t count, double rate_per_s, uint64_t seed,
                                          int streams, double *latency_s, int64_t *first_bad) {
    if (count < 0 || streams < 1 || streams > 64 ||
        (count > 0 && (!inputs || !outputs || !lengths || !latency_s || !first_bad)))
        return UTF16_EINVAL;
    int64_t max_n = 1;
    for (int64_t i = 0; i < count; ++i) {
        if (lengths[i] < 0) return UTF16_EINVAL;
        max_n = lengths[i] > max_n ? lengths[i] : max_n;
    }
    struct Lane {
        uint16_t *d = nullptr;
        int64_t *d_first = nullptr, *h_first = nullptr;
        cudaStream_t s = nullptr;
    };
    std::vector<Lane> lanes((size_t)streams);
    int rc = UTF16_OK;
    for (Lane &l : lanes) {
        if (cudaMalloc((void **)&l.d, (size_t)max_n * 2u) != cudaSuccess ||
            cudaMalloc((void **)&l.d_first, sizeof(int64_t)) != cudaSuccess ||
            cudaHostAlloc((void **)&l.h_first, sizeof(int64_t), cudaHostAllocDefault) != cudaSuccess ||
            cudaStreamCreateWithFlags(&l.s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            rc = UTF16_ENOMEM;
            break;
        }
    }
    if (rc == UTF16_OK) {
        int dev = 0;
        cudaGetDevice(&dev);
        const int64_t start = utf16_server_clock_ns() + 1000000;
        const std::vector<int64_t> at = arrival_times(count, rate_per_s, seed, start);
        std::atomic<int64_t> next{0};
        std::atomic<int> err{UTF16_OK};
        std::vector<std::thread> workers;
        for (int w = 0; w < streams; ++w) {
            workers.emplace_back([&, w] {
                cudaSetDevice(dev);
                Lane &l = lanes[(size_t)w];
                for (;;) {
                    const int64_t i = next.fetch_add(1);
                    if (i >= count || err.load() != UTF16_OK) return;
                    wait_until(at[(size_t)i]);
                    const int64_t n = lengths[i];
                    int r = UTF16_OK;
                    if (n > 0) {
                        if (cudaMemcpyAsync(l.d, inputs[i], (size_t)n * 2u, cudaMemcpyHostToDevice, l.s) !=
                            cudaSuccess)
                            r = UTF16_ECUDA;
                        if (r == UTF16_OK) r = run_single(l.d, l.d, n, kModeInPlace, l.d_first, l.s, 0, 0);
                        if (r == UTF16_OK &&
                            (cudaMemcpyAsync(outputs[i], l.d, (size_t)n * 2u, cudaMemcpyDeviceToHost, l.s) !=
                                 cudaSuccess ||
                             cudaMemcpyAsync(l.h_first, l.d_first, sizeof(int64_t), cudaMemcpyDeviceToHost, l.s) !=
                                 cudaSuccess ||
                             cudaStreamSynchronize(l.s) != cudaSuccess))
                            r = UTF16_ECUDA;
                        first_bad[i] = r == UTF16_OK ? *l.h_first : r;
                    } else {
                        first_bad[i] = 0;
                    }
                    latency_s[i] = (double)(utf16_server_clock_ns() - at[(size_t)i]) * 1e-9;
                    if (r != UTF16_OK) {
                        int expect = UTF16_OK;
                        err.compare_exchange_strong(expect, r);
                    }
                }
            });
        }
        for (std::thread &t : workers) t.join();
        rc = err.load();
    }
    for (Lane &l : lanes) {
        if (l.s) {
            cudaStreamSynchronize(l.s);
            cudaStreamDestroy(l.s);
        }
        if (l.d) cudaFree(l.d);
        if (l.d_first) cudaFree(l.d_first);
        if (l.h_first) cudaFreeHost(l.h_first);
    }
    cudaGetLastError();
    return rc;
}
