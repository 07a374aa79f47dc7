// Autotuner: times every candidate launch configuration on the caller's own
// buffers and keeps the fastest for the size bucket, so that later calls of
// that size use it.  Results are identical in every configuration (the
// kernels differ only in how data is brought in and how many blocks run).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
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

// Writes over twice the L2 before a trial, so that every candidate starts
// with the same (cold) cache when the input does not fit in L2; otherwise the
// first candidate after a pass that wrote the input's tail would start warm.
struct L2Scrub {
    void *buf = nullptr;
    size_t bytes = 0;
    L2Scrub(int64_t input_bytes) {
        int dev = 0, l2 = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        if (input_bytes <= (int64_t)l2) return;
        bytes = (size_t)l2 * 2;
        if (cudaMalloc(&buf, bytes) != cudaSuccess) {
            cudaGetLastError();
            buf = nullptr;
        }
    }
    ~L2Scrub() {
        if (buf) cudaFree(buf);
    }
    bool run(cudaStream_t s) const { return !buf || cudaMemsetAsync(buf, 0, bytes, s) == cudaSuccess; }
};

// UTF16WF_TUNE_LOG=1 prints every candidate's time to stderr.
bool tune_log() {
    static const bool on = [] {
        const char *e = getenv("UTF16WF_TUNE_LOG");
        return e && *e && *e != '0';
    }();
    return on;
}

void log_candidate(const char *what, const utf16_config &c, float ms) {
    if (!tune_log()) return;
    fprintf(stderr,
            "utf16wf tune %s: single v%d U%d bps%d | repair v%d U%d bps%d t%d | check v%d bps%d t%d | inplace v%d "
            "bps%d t%d | batch U%d pf%d bps%d check-pf%d | threads %d vector %d: %.4f ms\n",
            what, c.single_variant, c.single_units_per_thread, c.single_blocks_per_sm, c.repair_variant,
            c.repair_units_per_thread, c.repair_blocks_per_sm, c.repair_block_threads, c.check_variant,
            c.check_blocks_per_sm, c.check_block_threads, c.inplace_variant, c.inplace_blocks_per_sm,
            c.inplace_block_threads, c.batch_units_per_thread, c.batch_prefetch, c.batch_blocks_per_sm,
            c.batch_check_prefetch, c.block_threads, c.vector_bytes, ms);
}

// Fastest of three trials of `reps` back-to-back launches (ms per trial):
// the minimum keeps a candidate that met a slow moment from losing.
template <typename F>
bool time_trials(Timer &t, int reps, F launch, float *best, const L2Scrub *scrub = nullptr) {
    *best = 1e30f;
    for (int trial = 0; trial < 3; ++trial) {
        if (scrub && !scrub->run(t.s)) return false;
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

    const L2Scrub scrub(n * 2);
    const PdlOffScope pdl_off;
    utf16_config base = ctx->def, winner = base;
    float best_ms = 1e30f;
    for (int variant = 0; variant <= 2; ++variant) {
        for (int u : {2, 4})
        for (int bt : {128, 256, 512}) {
            if (variant == kVariantTma && (u != 4 || bt != kBlockThreads)) continue;
            utf16_config c = base;
            c.single_variant = variant;
            c.single_units_per_thread = u;
            c.block_threads = bt;
            const bool tma = variant == kVariantTma;
            const int fit = ctx->per_sm(single_kernel_for_occupancy(kModeOut, true, u, variant),
                                        tma ? single_tma_smem_bytes() : 0, bt);
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
                if (!time_trials(t, reps, [&] { return launch_single(L, t.s) == cudaSuccess; }, &ms, &scrub)) {
                    cudaGetLastError();
                    return UTF16_ECUDA;
                }
                log_candidate("repair+first-error", c, ms);
                if (ms < best_ms) {
                    best_ms = ms;
                    winner = c;
                }
            }
        }
    }
    // The repair without the first-error index on its own: its kernel keeps
    // no first-error state, so a data path that costs the fused kernel
    // occupancy can be its fastest (1 GiB at 1e-2: next chunk in flight,
    // 332 against 343 us).  Kept only where it beats following the fused
    // form's settings (-1 / 0 / -1).
    {
        auto time_plain = [&](const utf16_config &c, float *ms) -> bool {
            SingleLaunch L;
            L.in = in;
            L.out = out;
            L.n = n;
            L.mode = kModeOut;
            L.first_bad = false;
            configure_single(ctx, c, L);
            if (launch_single(L, t.s) != cudaSuccess) return false;
            return time_trials(t, reps, [&] { return launch_single(L, t.s) == cudaSuccess; }, ms, &scrub);
        };
        utf16_config plain_winner = winner;
        plain_winner.repair_variant = -1;
        plain_winner.repair_units_per_thread = 0;
        plain_winner.repair_blocks_per_sm = -1;
        plain_winner.repair_block_threads = 0;
        float best_plain = 0.f;
        if (!time_plain(plain_winner, &best_plain)) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
        log_candidate("repair (as the fused form)", plain_winner, best_plain);
        for (int variant = 0; variant <= 2; ++variant)
            for (int u : {2, 4})
            for (int bt : {128, 256, 512}) {
                const bool tma = variant == kVariantTma;
                if (tma && (u != 4 || bt != kBlockThreads)) continue;
                const int fit = ctx->per_sm(single_kernel_for_occupancy(kModeOut, false, u, variant),
                                            tma ? single_tma_smem_bytes() : 0, bt);
                for (int bps : block_candidates(fit)) {
                    utf16_config c = winner;
                    c.repair_variant = variant;
                    c.repair_units_per_thread = u;
                    c.repair_blocks_per_sm = bps;
                    c.repair_block_threads = bt;
                    float ms = 0.f;
                    if (!time_plain(c, &ms)) {
                        cudaGetLastError();
                        return UTF16_ECUDA;
                    }
                    log_candidate("repair", c, ms);
                    if (ms < best_plain) {
                        best_plain = ms;
                        plain_winner = c;
                    }
                }
            }
        winner.repair_variant = plain_winner.repair_variant;
        winner.repair_units_per_thread = plain_winner.repair_units_per_thread;
        winner.repair_blocks_per_sm = plain_winner.repair_blocks_per_sm;
        winner.repair_block_threads = plain_winner.repair_block_threads;
    }
    // The read-only check separately: each data path and grid on `out`, which
    // now holds the repaired (well-formed) string, so that every candidate
    // reads the whole string as for valid input (full_pass also turns off the
    // early exit).
    float best_check = 1e30f;
    utf16_config check_winner = winner;
    for (int variant = 0; variant <= 2; ++variant)
    for (int bt : {128, 256, 512})
    for (int bps : block_candidates(ctx->per_sm(single_kernel_for_occupancy(kModeCheck, true, winner.single_units_per_thread,
                                                                            variant),
                                                variant == kVariantTma ? single_tma_smem_bytes() : 0,
                                                variant == kVariantTma ? kBlockThreads : bt))) {
        if (variant == kVariantTma && bt != kBlockThreads) continue;
        utf16_config c = winner;
        c.check_variant = variant;
        c.check_blocks_per_sm = bps;
        c.check_block_threads = bt;
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
        if (!time_trials(t, reps, [&] { return launch_single(L, t.s) == cudaSuccess; }, &ms, &scrub)) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
        log_candidate("check", c, ms);
        if (ms < best_check) {
            best_check = ms;
            check_winner = c;
        }
    }
    winner.check_variant = check_winner.check_variant;
    winner.check_blocks_per_sm = check_winner.check_blocks_per_sm;
    winner.check_block_threads = check_winner.check_block_threads;
    // In-place repair: each data path on a fresh copy of `in` in `out` per
    // launch; the copies alone are timed too and subtracted.
    {
        const size_t bytes = (size_t)n * 2u;
        auto timed = [&](const SingleLaunch *L, float *ms) -> bool {
            return time_trials(t, reps, [&] {
                return cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, t.s) == cudaSuccess &&
                       (!L || launch_single(*L, t.s) == cudaSuccess);
            }, ms, &scrub);
        };
        float copies = 0.f;
        if (!timed(nullptr, &copies)) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
        float best_inplace = 1e30f;
        utf16_config inplace_winner = winner;
        for (int variant = 0; variant <= 2; ++variant)
        for (int bt : {128, 256, 512})
        for (int bps : block_candidates(
                 ctx->per_sm(single_kernel_for_occupancy(kModeInPlace, false, winner.single_units_per_thread, variant),
                             variant == kVariantTma ? single_tma_smem_bytes() : 0,
                             variant == kVariantTma ? kBlockThreads : bt))) {
            if (variant == kVariantTma && bt != kBlockThreads) continue;
            utf16_config c = winner;
            c.inplace_variant = variant;
            c.inplace_blocks_per_sm = bps;
            c.inplace_block_threads = bt;
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
            log_candidate("in-place", c, ms - copies);
            if (ms - copies < best_inplace) {
                best_inplace = ms - copies;
                inplace_winner = c;
            }
        }
        winner.inplace_variant = inplace_winner.inplace_variant;
        winner.inplace_blocks_per_sm = inplace_winner.inplace_blocks_per_sm;
        winner.inplace_block_threads = inplace_winner.inplace_block_threads;
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
    int64_t range[2] = {0, 0};  // offsets[0] and offsets[num_strings]: the batch's extent
    if (cudaMemcpy(&range[0], offsets, 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&range[1], offsets + num_strings, 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    const L2Scrub scrub((range[1] - range[0]) * 2);
    const PdlOffScope pdl_off;

    utf16_config base = ctx->def, winner = base;
    float best_ms = 1e30f;
    for (int u : {2, 4})
    for (int bt : {128, 256, 512})
    for (int vb : {8, 16, 32}) {
        for (int pf = 0; pf <= 1; ++pf) {
            if (pf && (u != 2 || vb != 16)) continue;  // the next chunk in flight is built for 1024 units, 16 bytes
            utf16_config c = base;
            c.batch_units_per_thread = u;
            c.batch_prefetch = pf;
            c.block_threads = bt;
            c.vector_bytes = vb;
            const int fit = ctx->per_sm(batch_kernel_for_occupancy(kModeOut, u, pf != 0, vb), 0, bt);
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
                if (!time_trials(t, reps, [&] { return launch_batch(L, t.s) == cudaSuccess; }, &ms, &scrub)) {
                    cudaGetLastError();
                    return UTF16_ECUDA;
                }
                log_candidate("batch repair", c, ms);
                if (ms < best_ms) {
                    best_ms = ms;
                    winner = c;
                }
            }
        }
    }
    // A 1024-unit chunk is what the out-of-place repair takes by default:
    // store "by mode", so that the other batch forms keep their own width
    // (2048 units for the check and in place).
    if (winner.batch_units_per_thread == 2) winner.batch_units_per_thread = 0;
    // The same for the block size and the load width the out-of-place form
    // takes by default (512 threads, 16-byte loads; in place defaults to 32).
    if (winner.block_threads == kMaxBlockThreads) winner.block_threads = 0;
    if (winner.vector_bytes == 16) winner.vector_bytes = 0;
    // The per-string check: next chunk in flight or not, with the winner's
    // other settings (its results go to a scratch array).
    {
        long long *scratch_fb = nullptr;
        if (cudaMalloc((void **)&scratch_fb, (size_t)num_strings * 8u) != cudaSuccess) {
            cudaGetLastError();
            return UTF16_ENOMEM;
        }
        float best_check = 1e30f;
        int best_pf = winner.batch_check_prefetch;
        for (int pf = 0; pf <= 1; ++pf) {
            utf16_config c = winner;
            c.batch_check_prefetch = pf;
            BatchLaunch L;
            L.in = in;
            L.offsets = (const long long *)offsets;
            L.count = num_strings;
            L.first_bad = scratch_fb;
            L.mode = kModeCheck;
            configure_batch(ctx, c, L);
            float ms = 0.f;
            if (launch_batch(L, t.s) != cudaSuccess ||
                !time_trials(t, reps, [&] { return launch_batch(L, t.s) == cudaSuccess; }, &ms, &scrub)) {
                cudaGetLastError();
                cudaStreamSynchronize(t.s);
                cudaFree(scratch_fb);
                return UTF16_ECUDA;
            }
            log_candidate("batch check", c, ms);
            if (ms < best_check) {
                best_check = ms;
                best_pf = pf;
            }
        }
        cudaStreamSynchronize(t.s);
        cudaFree(scratch_fb);
        winner.batch_check_prefetch = best_pf;
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

// ---------------------------------------------------------------------------
// Tuning from a length histogram, on synthetic strings the library makes
// itself: 16-bit hashes of the unit index give mostly ASCII and other BMP
// text with about 8 % of its cells surrogate pairs and about 1 % lone
// surrogates, so that the slow path runs as on mixed text.

namespace u16wf {
namespace {

__device__ __forceinline__ uint32_t mix32(uint64_t x) {
    x ^= x >> 33;
    x *= 0xFF51AFD7ED558CCDull;
    x ^= x >> 33;
    x *= 0xC4CEB9FE1A85EC53ull;
    x ^= x >> 33;
    return (uint32_t)x;
}

// Cell k covers units 2k and 2k+1.
__global__ void synth_text_kernel(uint16_t *u, long long n, uint64_t seed) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; 2 * k < n; k += stride) {
        const uint32_t h = mix32(seed + (uint64_t)k);
        const uint32_t kind = h % 100u;
        uint16_t a, b;
        if (kind < 8) {  // a pair
            a = (uint16_t)(0xD800u + (h >> 8) % 1024u);
            b = (uint16_t)(0xDC00u + (h >> 18) % 1024u);
        } else if (kind < 9) {  // a lone surrogate, then ASCII
            a = (uint16_t)(0xD800u + (h >> 8) % 2048u);
            b = (uint16_t)(0x20u + (h >> 20) % 95u);
        } else if (kind < 30) {  // BMP text outside the surrogates
            a = (uint16_t)(0x0100u + (h >> 8) % 0xD700u);
            b = (uint16_t)(0x0100u + (h >> 20) % 0xD700u);
        } else {
            a = (uint16_t)(0x20u + (h >> 8) % 95u);
            b = (uint16_t)(0x20u + (h >> 16) % 95u);
        }
        u[2 * k] = a;
        if (2 * k + 1 < n) u[2 * k + 1] = b;
    }
}

constexpr long long kTuneMaxUnits = 1LL << 29;  // 1 GiB of synthetic input at most per tuning run

}  // namespace
}  // namespace u16wf

extern "C" int utf16_autotune(int op, const int64_t *length_histogram, int buckets) {
    if ((op != 0 && op != 1) || !length_histogram || buckets < 1 || buckets > 64) return UTF16_EINVAL;
    for (int b = 0; b < buckets; ++b)
        if (length_histogram[b] < 0) return UTF16_EINVAL;
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;
    const int reps = 3;
    if (op == 0) {
        // every non-empty bucket b: one string of 2^b units (capped)
        for (int b = 0; b < buckets; ++b) {
            if (!length_histogram[b]) continue;
            const long long n = std::min(1LL << b, kTuneMaxUnits);
            uint16_t *in = nullptr, *out = nullptr;
            if (cudaMalloc((void **)&in, (size_t)n * 2u) != cudaSuccess ||
                cudaMalloc((void **)&out, (size_t)n * 2u) != cudaSuccess) {
                cudaGetLastError();
                cudaFree(in);
                return UTF16_ENOMEM;
            }
            synth_text_kernel<<<ctx->sms * 4, 256>>>(in, n, 0x2601063490ull + (uint64_t)b);
            utf16_config cfg;
            rc = cudaDeviceSynchronize() == cudaSuccess ? utf16_autotune_single(in, out, n, reps, &cfg) : UTF16_ECUDA;
            cudaFree(in);
            cudaFree(out);
            cudaGetLastError();
            if (rc) return rc;
            if (bucket_of(n) != b) utf16_set_tuned(0, b, &cfg);  // sizes above the cap take the cap's result
        }
        return UTF16_OK;
    }
    // op 1: one batch whose string lengths follow the histogram (bucket b:
    // lengths in [2^b, 2^(b+1)), bucket 0 also holds empty strings), scaled
    // down to at most kTuneMaxUnits units in all
    long long total_strings = 0;
    double total_units = 0;
    for (int b = 0; b < buckets; ++b) {
        total_strings += length_histogram[b];
        total_units += (double)length_histogram[b] * 1.5 * (double)(1LL << b);
    }
    if (total_strings == 0) return UTF16_OK;
    const double scale = total_units > (double)kTuneMaxUnits ? (double)kTuneMaxUnits / total_units : 1.0;
    std::vector<long long> lens;
    uint64_t z = 0x9E3779B97F4A7C15ull;
    for (int b = 0; b < buckets; ++b) {
        const long long cnt = (long long)((double)length_histogram[b] * scale + 0.5);
        for (long long i = 0; i < cnt; ++i) {
            z ^= z << 13;
            z ^= z >> 7;
            z ^= z << 17;
            lens.push_back(b == 0 ? (long long)(z % 2u) : (1LL << b) + (long long)(z % (uint64_t)(1LL << b)));
        }
    }
    // interleave the buckets so that chunks see the mix
    for (size_t i = lens.size(); i > 1; --i) {
        z ^= z << 13;
        z ^= z >> 7;
        z ^= z << 17;
        std::swap(lens[i - 1], lens[(size_t)(z % i)]);
    }
    const long long count = (long long)lens.size();
    if (count == 0) return UTF16_OK;
    long long units = 0;
    for (long long v : lens) units += v;
    if (units == 0) return UTF16_OK;
    std::vector<int64_t> offs((size_t)count + 1, 0);
    for (long long i = 0; i < count; ++i) offs[(size_t)i + 1] = offs[(size_t)i] + lens[(size_t)i];
    uint16_t *in = nullptr, *out = nullptr;
    int64_t *d_off = nullptr;
    if (cudaMalloc((void **)&in, (size_t)units * 2u) != cudaSuccess ||
        cudaMalloc((void **)&out, (size_t)units * 2u) != cudaSuccess ||
        cudaMalloc((void **)&d_off, (size_t)(count + 1) * 8u) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(in);
        cudaFree(out);
        return UTF16_ENOMEM;
    }
    rc = UTF16_OK;
    if (cudaMemcpy(d_off, offs.data(), (size_t)(count + 1) * 8u, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = UTF16_ECUDA;
    if (!rc) {
        synth_text_kernel<<<ctx->sms * 4, 256>>>(in, units, 0x2601063491ull);
        if (cudaDeviceSynchronize() != cudaSuccess) rc = UTF16_ECUDA;
    }
    utf16_config cfg;
    if (!rc) rc = utf16_autotune_batch(in, out, d_off, count, reps, &cfg);
    cudaFree(in);
    cudaFree(out);
    cudaFree(d_off);
    cudaGetLastError();
    // a scaled-down batch also answers for the histogram's own string count
    if (!rc && bucket_of(total_strings) != bucket_of(count)) utf16_set_tuned(1, bucket_of(total_strings), &cfg);
    return rc;
}
