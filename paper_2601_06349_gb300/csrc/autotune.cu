// Autotuner: times every candidate launch configuration on the caller's own
// buffers and keeps the fastest for the size bucket, so that later calls of
// that size use it.  Results are identical in every configuration (the
// kernels differ only in how data is brought in and how many blocks run).
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/utf16wf.h"
#include "internal.h"
#include "runtime.h"

namespace u16wf {

namespace {

struct Timer {
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    bool ok = false;
    Timer() {
        ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
    }
    ~Timer() {
        if (s) cudaStreamSynchronize(s);
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (s) cudaStreamDestroy(s);
    }
};

// Fastest of three trials of `reps` back-to-back launches (ms per trial):
// the minimum keeps a candidate that met a slow moment from losing.
template <typename F>
bool time_trials(Timer &t, int reps, F launch, float *best) {
    *best = 1e30f;
    for (int trial = 0; trial < 3; ++trial) {
        if (cudaEventRecord(t.a, t.s) != cudaSuccess) return false;
        for (int r = 0; r < reps; ++r)
            if (!launch()) return false;
        if (cudaEventRecord(t.b, t.s) != cudaSuccess || cudaEventSynchronize(t.b) != cudaSuccess) return false;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess) return false;
        if (ms < *best) *best = ms;
    }
    return true;
}

// Blocks-per-SM candidates below the occupancy limit `fit` (0 = all that fit).
std::vector<int> block_candidates(int fit) {
    std::vector<int> v = {0};
    for (int b : {1, 2, 3, 4, 6}) {
        if (b < fit) v.push_back(b);
    }
    return v;
}

}  // namespace

}  // namespace u16wf

using namespace u16wf;

extern "C" int utf16_autotune_single(const uint16_t *in, uint16_t *out, int64_t n, int reps, utf16_config *best) {
    if (n <= 0 || !in || !out || in == out || reps < 1 || ((uintptr_t)in & 1u) || ((uintptr_t)out & 1u))
        return UTF16_EINVAL;
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;
    Timer t;
    if (!t.ok) return UTF16_ECUDA;
    Slot *slot;
    rc = ctx->slot_for(t.s, &slot);
    if (rc) return rc;

    utf16_config base = ctx->def, winner = base;
    float best_ms = 1e30f;
    for (int variant = 0; variant <= 2; ++variant) {
        for (int u : {2, 4}) {
            if (variant == kVariantTma && u != 4) continue;
            utf16_config c = base;
            c.single_variant = variant;
            c.single_units_per_thread = u;
            const bool tma = variant == kVariantTma;
            const int fit = ctx->per_sm(single_kernel_for_occupancy(kModeOut, true, u, variant),
                                        tma ? single_tma_smem_bytes() : 0);
            for (int bps : block_candidates(fit)) {
                c.single_blocks_per_sm = bps;
                SingleLaunch L;
                L.in = in;
                L.out = out;
                L.n = n;
                L.mode = kModeOut;
                L.first_bad = true;
                configure_single(ctx, c, L);
                L.slot = slot;
                L.result = &slot->result;
                if (launch_single(L, t.s) != cudaSuccess) {
                    cudaGetLastError();
                    return UTF16_ECUDA;
                }
                float ms = 0.f;
                if (!time_trials(t, reps, [&] { return launch_single(L, t.s) == cudaSuccess; }, &ms)) {
                    cudaGetLastError();
                    return UTF16_ECUDA;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    winner = c;
                }
            }
        }
    }
    // The read-only check separately: each data path and grid on `out`, which
    // now holds the repaired (well-formed) string, so that every candidate
    // reads the whole string as for valid input (full_pass also turns off the
    // early exit).
    float best_check = 1e30f;
    utf16_config check_winner = winner;
    for (int variant = 0; variant <= 2; ++variant)
    for (int bps : block_candidates(ctx->per_sm(single_kernel_for_occupancy(kModeCheck, true, winner.single_units_per_thread,
                                                                            variant),
                                                variant == kVariantTma ? single_tma_smem_bytes() : 0))) {
        utf16_config c = winner;
        c.check_variant = variant;
        c.check_blocks_per_sm = bps;
        SingleLaunch L;
        L.in = out;
        L.n = n;
        L.mode = kModeCheck;
        L.first_bad = true;
        configure_single(ctx, c, L);
        L.slot = slot;
        L.result = &slot->result;
        L.full_pass = true;
        if (launch_single(L, t.s) != cudaSuccess) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
        float ms = 0.f;
        if (!time_trials(t, reps, [&] { return launch_single(L, t.s) == cudaSuccess; }, &ms)) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
        if (ms < best_check) {
            best_check = ms;
            check_winner = c;
        }
    }
    winner.check_variant = check_winner.check_variant;
    winner.check_blocks_per_sm = check_winner.check_blocks_per_sm;
    // In-place repair: each data path on a fresh copy of `in` in `out` per
    // launch; the copies alone are timed too and subtracted.
    {
        const size_t bytes = (size_t)n * 2u;
        auto timed = [&](const SingleLaunch *L, float *ms) -> bool {
            return time_trials(t, reps, [&] {
                return cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, t.s) == cudaSuccess &&
                       (!L || launch_single(*L, t.s) == cudaSuccess);
            }, ms);
        };
        float copies = 0.f;
        if (!timed(nullptr, &copies)) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
        float best_inplace = 1e30f;
        utf16_config inplace_winner = winner;
        for (int variant = 0; variant <= 2; ++variant)
        for (int bps : block_candidates(
                 ctx->per_sm(single_kernel_for_occupancy(kModeInPlace, false, winner.single_units_per_thread, variant),
                             variant == kVariantTma ? single_tma_smem_bytes() : 0))) {
            utf16_config c = winner;
            c.inplace_variant = variant;
            c.inplace_blocks_per_sm = bps;
            SingleLaunch L;
            L.in = out;
            L.out = out;
            L.n = n;
            L.mode = kModeInPlace;
            configure_single(ctx, c, L);
            float ms = 0.f;
            if (!timed(&L, &ms)) {
                cudaGetLastError();
                return UTF16_ECUDA;
            }
            if (ms - copies < best_inplace) {
                best_inplace = ms - copies;
                inplace_winner = c;
            }
        }
        winner.inplace_variant = inplace_winner.inplace_variant;
        winner.inplace_blocks_per_sm = inplace_winner.inplace_blocks_per_sm;
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        const int b = bucket_of(n);
        ctx->single_tuned[b] = winner;
        ctx->single_has[b] = true;
    }
    if (best) *best = winner;
    return UTF16_OK;
}

extern "C" int utf16_autotune_batch(const uint16_t *in, uint16_t *out, const int64_t *offsets, int64_t num_strings,
                                    int reps, utf16_config *best) {
    if (num_strings <= 0 || !in || !out || !offsets || in == out || reps < 1 || ((uintptr_t)in & 1u) ||
        ((uintptr_t)out & 1u) || ((uintptr_t)offsets & 7u))
        return UTF16_EINVAL;
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;
    Timer t;
    if (!t.ok) return UTF16_ECUDA;

    utf16_config base = ctx->def, winner = base;
    float best_ms = 1e30f;
    for (int u : {2, 4}) {
        for (int pf = 0; pf <= 1; ++pf) {
            utf16_config c = base;
            c.batch_units_per_thread = u;
            c.batch_prefetch = pf;
            const int fit = ctx->per_sm(batch_kernel_for_occupancy(kModeOut, u, pf != 0), 0);
            for (int bps : block_candidates(fit)) {
                c.batch_blocks_per_sm = bps;
                BatchLaunch L;
                L.in = in;
                L.out = out;
                L.offsets = (const long long *)offsets;
                L.count = num_strings;
                L.mode = kModeOut;
                configure_batch(ctx, c, L);
                if (launch_batch(L, t.s) != cudaSuccess) {
                    cudaGetLastError();
                    return UTF16_ECUDA;
                }
                float ms = 0.f;
                if (!time_trials(t, reps, [&] { return launch_batch(L, t.s) == cudaSuccess; }, &ms)) {
                    cudaGetLastError();
                    return UTF16_ECUDA;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    winner = c;
                }
            }
        }
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        const int b = bucket_of(num_strings);
        ctx->batch_tuned[b] = winner;
        ctx->batch_has[b] = true;
    }
    if (best) *best = winner;
    return UTF16_OK;
}
