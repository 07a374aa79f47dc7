// Host runtime of libutf16wf: per-device context (SM count, occupancy-derived
// persistent grid sizes, scratch slots, launch configuration, staging for
// host buffers), argument validation and the C-ABI entry points declared in
// include/utf16wf.h.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "../../include/utf16wf.h"
#include "device.cuh"
#include "internal.h"
#include "runtime.h"

namespace u16wf {

static std::mutex g_mu;
static std::unordered_map<int, std::unique_ptr<DeviceCtx>> g_ctx;

static int env_int(const char *name, int dflt) {
    const char *s = getenv(name);
    if (!s || !*s) return dflt;
    return atoi(s);
}

int bucket_of(int64_t v) {
    int b = 0;
    while (v > 1 && b < kBuckets - 1) {
        v >>= 1;
        ++b;
    }
    return b;
}

int DeviceCtx::per_sm(const void *fn, size_t smem, int threads) {
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(fn, threads);
    auto it = occupancy.find(key);
    if (it != occupancy.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    occupancy[key] = n;
    return n;
}

int DeviceCtx::slot_for(cudaStream_t s, Slot **out) {
    std::lock_guard<std::mutex> lk(mu);
    auto it = slot_of.find(s);
    if (it != slot_of.end()) {
        *out = slots + it->second;
        return UTF16_OK;
    }
    if (slots_used >= kSlotCount) return UTF16_ENOMEM;
    const int idx = slots_used++;
    slot_of[s] = idx;
    *out = slots + idx;
    return UTF16_OK;
}

utf16_config DeviceCtx::single_config(int64_t n) {
    std::lock_guard<std::mutex> lk(mu);
    const int b = bucket_of(n);
    return single_has[b] ? single_tuned[b] : def;
}

utf16_config DeviceCtx::batch_config(int64_t units, int64_t count) {
    (void)units;
    std::lock_guard<std::mutex> lk(mu);
    const int b = bucket_of(count);
    return batch_has[b] ? batch_tuned[b] : def;
}

static bool threads_valid(int t) { return t == 0 || t == 128 || t == 256 || t == 512; }

static bool config_valid(const utf16_config &c) {
    return c.single_variant >= 0 && c.single_variant <= 2 && c.check_variant >= 0 && c.check_variant <= 2 &&
           c.inplace_variant >= 0 && c.inplace_variant <= 2 && c.check_blocks_per_sm >= 0 &&
           c.check_blocks_per_sm <= 64 && c.inplace_blocks_per_sm >= 0 && c.inplace_blocks_per_sm <= 64 &&
           (c.batch_check_prefetch == 0 || c.batch_check_prefetch == 1) &&
           (c.inplace_unit_stores == 0 || c.inplace_unit_stores == 1) &&
           (c.single_units_per_thread == 0 || c.single_units_per_thread == 2 || c.single_units_per_thread == 4) &&
           c.single_blocks_per_sm >= 0 &&
           c.single_blocks_per_sm <= 64 && (c.batch_units_per_thread == 0 || c.batch_units_per_thread == 2 || c.batch_units_per_thread == 4) &&
           (c.batch_prefetch == 0 || c.batch_prefetch == 1) && c.batch_blocks_per_sm >= 0 &&
           c.batch_blocks_per_sm <= 64 &&
           (c.block_threads == 0 || c.block_threads == 128 || c.block_threads == 256 || c.block_threads == 512) &&
           (c.vector_bytes == 0 || c.vector_bytes == 8 || c.vector_bytes == 16 || c.vector_bytes == 32) &&
           c.repair_variant >= -1 && c.repair_variant <= 2 &&
           (c.repair_units_per_thread == 0 || c.repair_units_per_thread == 2 || c.repair_units_per_thread == 4) &&
           c.repair_blocks_per_sm >= -1 && c.repair_blocks_per_sm <= 64 && threads_valid(c.repair_block_threads) &&
           threads_valid(c.check_block_threads) && threads_valid(c.inplace_block_threads);
}

int get_ctx(DeviceCtx **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_ctx.find(dev);
    if (it != g_ctx.end()) {
        *out = it->second.get();
        return UTF16_OK;
    }
    std::unique_ptr<DeviceCtx> c(new DeviceCtx());
    c->device = dev;
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    int pageable = 0;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) {
        cudaGetLastError();
        pageable = 0;
    }
    c->pageable_access = pageable != 0;
    if (prepare_single_tma() != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    if (cudaMalloc((void **)&c->slots, sizeof(Slot) * kSlotCount) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ENOMEM;
    }
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return UTF16_ECUDA;
    if (init_slots(c->slots, kSlotCount, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaStreamDestroy(s);
        return UTF16_ECUDA;
    }
    cudaStreamDestroy(s);
    utf16_config d;
    d.single_variant = env_int("UTF16WF_SINGLE_VARIANT", kVariantLdg);
    d.single_units_per_thread = env_int("UTF16WF_SINGLE_U", 0);
    d.single_blocks_per_sm = env_int("UTF16WF_SINGLE_BLOCKS_PER_SM", 0);
    // Batches: the chunk width of each mode (0; 1024 units out of place,
    // 2048 otherwise) and no next chunk in flight, which only cost registers
    // (1M strings out of place: 69.5 against 77 us).
    d.batch_units_per_thread = env_int("UTF16WF_BATCH_U", 0);
    d.batch_prefetch = env_int("UTF16WF_BATCH_PREFETCH", 0);
    d.batch_blocks_per_sm = env_int("UTF16WF_BATCH_BLOCKS_PER_SM", 0);
    d.check_variant = env_int("UTF16WF_CHECK_VARIANT", kVariantLdg);
    d.inplace_unit_stores = env_int("UTF16WF_INPLACE_UNIT_STORES", 0);
    // In place, the next chunk's loads in flight while this one is processed
    // measured faster on a 1 GiB string with 1e-2 lone surrogates (0.72 vs
    // 0.68 of the copy peak); out of place with the first-error index the
    // plain loads are (0.93 vs 0.89).
    d.inplace_variant = env_int("UTF16WF_INPLACE_VARIANT", kVariantLdgPrefetch);
    d.check_blocks_per_sm = env_int("UTF16WF_CHECK_BLOCKS_PER_SM", 0);
    d.inplace_blocks_per_sm = env_int("UTF16WF_INPLACE_BLOCKS_PER_SM", 0);
    // The batch check runs faster without the next chunk in flight (1M
    // strings: 43 against 64 us).
    d.batch_check_prefetch = env_int("UTF16WF_BATCH_CHECK_PREFETCH", 0);
    // Programmatic dependent launch: back-to-back small calls measured 7-11 %
    // faster (1024 units 3.12 -> 2.89 us, 1,000,000 units 5.21 -> 4.68 us),
    // long ones unchanged.
    g_pdl = env_int("UTF16WF_PDL", 1) != 0;
    // Block size (0: 256 threads) and bytes per lane load of the bit-word
    // kernels (0: 16 bytes).
    d.block_threads = env_int("UTF16WF_BLOCK_THREADS", 0);
    d.vector_bytes = env_int("UTF16WF_VECTOR_BYTES", 0);
    // The repair without the first-error index follows the fused form's
    // data path, chunk width and grid unless set (or tuned) on its own.
    d.repair_variant = env_int("UTF16WF_REPAIR_VARIANT", -1);
    d.repair_units_per_thread = env_int("UTF16WF_REPAIR_U", 0);
    d.repair_blocks_per_sm = env_int("UTF16WF_REPAIR_BLOCKS_PER_SM", -1);
    d.repair_block_threads = env_int("UTF16WF_REPAIR_BLOCK_THREADS", 0);
    d.check_block_threads = env_int("UTF16WF_CHECK_BLOCK_THREADS", 0);
    d.inplace_block_threads = env_int("UTF16WF_INPLACE_BLOCK_THREADS", 0);
    if (!config_valid(d))
        d = utf16_config{kVariantLdg, 0, 0, 0, 0, 0, kVariantLdg, 0, kVariantLdgPrefetch, 0, 0, 0, 0, 0, -1, 0, -1, 0, 0, 0};
    c->def = d;
    *out = c.get();
    g_ctx[dev] = std::move(c);
    return UTF16_OK;
}

void configure_single(DeviceCtx *ctx, const utf16_config &cfg, SingleLaunch &L) {
    // The out-of-place repair without the first-error index has settings of
    // its own where they are set: its kernel keeps no first-error state, so
    // its best shape can differ (1 GiB at 1e-2: 0.95 of the copy peak on its
    // own tuned settings, 0.92 on the fused form's).
    const bool plain = L.mode == kModeOut && !L.first_bad;
    L.variant = L.mode == kModeCheck     ? cfg.check_variant
                : L.mode == kModeInPlace ? cfg.inplace_variant
                : plain && cfg.repair_variant >= 0 ? cfg.repair_variant
                                                   : cfg.single_variant;
    L.unit_stores = L.mode == kModeInPlace && cfg.inplace_unit_stores != 0;
    // Unit stores exist in the 128-bit-load kernels only.
    if (L.unit_stores && L.variant == kVariantTma) L.variant = kVariantLdg;
    // U = 0: by size.  Below about 40 Ki units per SM, 2-vector chunks spread
    // the string over more warps and SMs (1M units: 3.2-3.5 against 4.4 us
    // per call back to back; from 8M units on, 4-vector chunks are as fast or
    // faster, and 23 against 31 us in place at 64M).
    const int cfg_u = plain && cfg.repair_units_per_thread != 0 ? cfg.repair_units_per_thread
                                                                 : cfg.single_units_per_thread;
    L.units_per_thread = cfg_u != 0 ? cfg_u : L.n < (long long)ctx->sms * kAutoWideChunkUnitsPerSm ? 2 : 4;
    const bool fb = L.first_bad || L.mode == kModeCheck;
    const bool tma = L.variant == kVariantTma;
    // Block size: the form's own, else the common one, else kBlockThreads.
    // The TMA kernel's tile is one chunk per warp of a kBlockThreads block.
    const int form_bt = L.mode == kModeCheck     ? cfg.check_block_threads
                        : L.mode == kModeInPlace ? cfg.inplace_block_threads
                        : plain                  ? cfg.repair_block_threads
                                                 : 0;
    const int bt = form_bt > 0 ? form_bt : cfg.block_threads;
    L.block_threads = tma ? kBlockThreads : bt > 0 ? bt : kBlockThreads;
    const void *fn = single_kernel_for_occupancy(L.mode, fb, L.units_per_thread, L.variant);
    const int fit = ctx->per_sm(fn, tma ? single_tma_smem_bytes() : 0, L.block_threads);
    const int want = L.mode == kModeCheck                    ? cfg.check_blocks_per_sm
                     : L.mode == kModeInPlace                ? cfg.inplace_blocks_per_sm
                     : plain && cfg.repair_blocks_per_sm >= 0 ? cfg.repair_blocks_per_sm
                                                              : cfg.single_blocks_per_sm;
    const int per = want > 0 ? std::min(want, fit) : fit;
    L.max_blocks = per * ctx->sms;
    L.full_occupancy = per == fit;
}

void configure_batch(DeviceCtx *ctx, const utf16_config &cfg, BatchLaunch &L) {
    L.units_per_thread = cfg.batch_units_per_thread;
    L.prefetch = (L.mode == kModeCheck ? cfg.batch_check_prefetch : cfg.batch_prefetch) != 0;
    // Unset (0): 512-thread blocks, and 32-byte loads in place, 16 otherwise
    // (1M strings: out of place 69.1 against 69.8 us at 256 threads; in place
    // 64.9 against 68.4 us with 16-byte loads; the check 43.2 against 49-50
    // with 32-byte ones).
    L.block_threads = cfg.block_threads > 0 ? cfg.block_threads : kMaxBlockThreads;
    L.vector_bytes = cfg.vector_bytes > 0 ? cfg.vector_bytes : L.mode == kModeInPlace ? 32 : 16;
    const int fit = ctx->per_sm(batch_kernel_for_occupancy(L.mode, L.units_per_thread, L.prefetch, L.vector_bytes), 0,
                                L.block_threads);
    const int per = cfg.batch_blocks_per_sm > 0 ? std::min(cfg.batch_blocks_per_sm, fit) : fit;
    L.blocks = per * ctx->sms;
    L.full_occupancy = per == fit;
}

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static bool overlaps(const void *a, const void *b, int64_t n) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    const uintptr_t bytes = (uintptr_t)n * 2u;
    return x != y && x < y + bytes && y < x + bytes;
}

static bool misaligned(const void *p) { return ((uintptr_t)p & 1u) != 0; }

int run_single(const uint16_t *in, uint16_t *out, int64_t n, int mode, int64_t *first_bad, cudaStream_t stream,
               uint32_t lead, uint32_t trail) {
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;
    const bool fb = first_bad != nullptr || mode == kModeCheck;
    const bool fb_on_device = fb && first_bad && is_device_ptr(first_bad);
    Slot *slot = nullptr;
    if (fb) {
        rc = ctx->slot_for(stream, &slot);
        if (rc) return rc;
    }
    SingleLaunch L;
    L.in = in;
    L.out = out;
    L.n = n;
    L.mode = mode;
    L.first_bad = fb;
    configure_single(ctx, ctx->single_config(n), L);
    L.slot = slot;
    L.result = fb ? (fb_on_device ? (long long *)first_bad : &slot->result) : nullptr;
    L.lead = lead;
    L.trail = trail;
    if (launch_single(L, stream) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    if (fb && first_bad && !fb_on_device) {
        if (cudaMemcpyAsync(first_bad, &slot->result, sizeof(int64_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
    }
    return UTF16_OK;
}

static int empty_first_bad(int64_t *first_bad, cudaStream_t stream) {
    if (!first_bad) return UTF16_OK;
    if (is_device_ptr(first_bad)) {
        if (cudaMemsetAsync(first_bad, 0, sizeof(int64_t), stream) != cudaSuccess) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
    } else {
        *first_bad = 0;
    }
    return UTF16_OK;
}

// Checked mode: -1 until first read (then UTF16WF_CHECKED, default off).
static std::atomic<int> g_checked{-1};

static bool checked_mode() {
    int c = g_checked.load(std::memory_order_relaxed);
    if (c < 0) {
        int expected = -1;
        g_checked.compare_exchange_strong(expected, env_int("UTF16WF_CHECKED", 0) != 0 ? 1 : 0);
        c = g_checked.load(std::memory_order_relaxed);
    }
    return c != 0;
}

// The offsets check of utf16_check_offsets into the stream's slot, read back
// on the host: *violation = smallest violating index or -1.
static int validate_offsets(DeviceCtx *ctx, const int64_t *offsets, int64_t count, cudaStream_t s,
                            int64_t *violation) {
    Slot *slot = nullptr;
    int rc = ctx->slot_for(s, &slot);
    if (rc) return rc;
    if (launch_check_offsets((const long long *)offsets, count, slot, &slot->result, ctx->sms * 8, s) != cudaSuccess ||
        cudaMemcpyAsync(violation, &slot->result, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    return UTF16_OK;
}

int run_batch(const uint16_t *in, uint16_t *out, const int64_t *offsets, int64_t count, int mode, int64_t *first_bad,
              cudaStream_t stream) {
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;
    if (checked_mode()) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
        if (cap != cudaStreamCaptureStatusNone) return UTF16_EINVAL;  // the check must read back
        int64_t violation = -1;
        rc = validate_offsets(ctx, offsets, count, stream, &violation);
        if (rc) return rc;
        if (violation >= 0) return UTF16_EINVAL;
    }
    BatchLaunch L;
    L.in = in;
    L.out = out;
    L.offsets = (const long long *)offsets;
    L.count = count;
    L.first_bad = (long long *)first_bad;
    L.mode = mode;
    configure_batch(ctx, ctx->batch_config(0, count), L);
    if (launch_batch(L, stream) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    return UTF16_OK;
}

}  // namespace u16wf

using namespace u16wf;

extern "C" {

const char *utf16_strerror(int code) {
    switch (code) {
        case UTF16_OK: return "success";
        case UTF16_EINVAL: return "invalid argument (null pointer, negative size, misaligned buffer or bad offsets)";
        case UTF16_EOVERLAP: return "input and output overlap without being the same buffer";
        case UTF16_ECUDA: return "a CUDA call failed";
        case UTF16_ETIMEOUT: return "a bounded wait gave up";
        case UTF16_ENOMEM: return "out of scratch slots, staging memory or serving budget";
        case UTF16_ECLOSED: return "the serving engine is shut down";
        case UTF16_EAGAIN: return "nothing ready yet";
        case UTF16_ETOOBIG: return "input longer than the no-allocation entry point accepts (2^40 units)";
        case UTF16_ECANCELED: return "the request was cancelled before admission";
        default: return "unknown status code";
    }
}

int utf16_init_device(void) {
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;
    for (int mode = 0; mode < 3; ++mode)
        for (int fb = 0; fb < 2; ++fb) {
            for (int u : {2, 4}) {  // both chunk widths, whatever the default picks by size
                utf16_config c = ctx->def;
                c.single_units_per_thread = u;
                SingleLaunch L;
                L.mode = mode;
                L.first_bad = fb != 0;
                configure_single(ctx, c, L);
            }
            BatchLaunch B;
            B.mode = mode;
            configure_batch(ctx, ctx->def, B);
        }
    return UTF16_OK;
}

int utf16_release_device(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    std::unique_ptr<DeviceCtx> c;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_ctx.find(dev);
        if (it == g_ctx.end()) return UTF16_OK;
        c = std::move(it->second);
        g_ctx.erase(it);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    c->release_staging();
    if (c->slots) cudaFree(c->slots);
    c->slots = nullptr;
    return UTF16_OK;
}

int utf16_get_config(utf16_config *cfg) {
    if (!cfg) return UTF16_EINVAL;
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    *cfg = ctx->def;
    return UTF16_OK;
}

int utf16_set_config(const utf16_config *cfg) {
    if (!cfg || !config_valid(*cfg)) return UTF16_EINVAL;
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->def = *cfg;
    for (int b = 0; b < kBuckets; ++b) ctx->single_has[b] = ctx->batch_has[b] = false;
    return UTF16_OK;
}

int utf16_get_tuned(int op, int bucket, utf16_config *cfg) {
    if ((op != 0 && op != 1) || bucket < 0 || bucket >= kBuckets || !cfg) return UTF16_EINVAL;
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    const bool has = op == 0 ? ctx->single_has[bucket] : ctx->batch_has[bucket];
    if (!has) return UTF16_EAGAIN;
    *cfg = op == 0 ? ctx->single_tuned[bucket] : ctx->batch_tuned[bucket];
    return UTF16_OK;
}

int utf16_set_tuned(int op, int bucket, const utf16_config *cfg) {
    if ((op != 0 && op != 1) || bucket < 0 || bucket >= kBuckets || !cfg || !config_valid(*cfg)) return UTF16_EINVAL;
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (op == 0) {
        ctx->single_tuned[bucket] = *cfg;
        ctx->single_has[bucket] = true;
    } else {
        ctx->batch_tuned[bucket] = *cfg;
        ctx->batch_has[bucket] = true;
    }
    return UTF16_OK;
}

int utf16_selftest_bounded_wait(int64_t limit_ns) {
    if (limit_ns <= 0 || limit_ns > 2000000000LL) return UTF16_EINVAL;
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;
    const int r = run_bounded_wait_probe(limit_ns);
    if (r < 0) return UTF16_ECUDA;
    return r ? UTF16_ETIMEOUT : UTF16_OK;
}

int utf16_check_device_errors(void) {
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    return read_and_clear_tma_timeout() ? UTF16_ETIMEOUT : UTF16_OK;
}

int utf16_to_well_formed(const uint16_t *in, uint16_t *out, int64_t n, utf16_stream_t stream) {
    if (n < 0) return UTF16_EINVAL;
    if (n == 0) return UTF16_OK;
    if (!in || !out || misaligned(in) || misaligned(out)) return UTF16_EINVAL;
    if (overlaps(in, out, n)) return UTF16_EOVERLAP;
    return run_single(in, out, n, in == out ? kModeInPlace : kModeOut, nullptr, (cudaStream_t)stream, 0, 0);
}

int utf16_to_well_formed_inplace(uint16_t *buf, int64_t n, utf16_stream_t stream) {
    if (n < 0) return UTF16_EINVAL;
    if (n == 0) return UTF16_OK;
    if (!buf || misaligned(buf)) return UTF16_EINVAL;
    return run_single(buf, buf, n, kModeInPlace, nullptr, (cudaStream_t)stream, 0, 0);
}

int utf16_to_well_formed_first_bad(const uint16_t *in, uint16_t *out, int64_t n, int64_t *first_bad,
                                   utf16_stream_t stream) {
    if (n < 0 || !first_bad) return UTF16_EINVAL;
    if (n == 0) return empty_first_bad(first_bad, (cudaStream_t)stream);
    if (!in || !out || misaligned(in) || misaligned(out)) return UTF16_EINVAL;
    if (overlaps(in, out, n)) return UTF16_EOVERLAP;
    return run_single(in, out, n, in == out ? kModeInPlace : kModeOut, first_bad, (cudaStream_t)stream, 0, 0);
}

int utf16_is_well_formed(const uint16_t *in, int64_t n, int64_t *first_bad, utf16_stream_t stream) {
    if (n < 0 || !first_bad) return UTF16_EINVAL;
    if (n == 0) return empty_first_bad(first_bad, (cudaStream_t)stream);
    if (!in || misaligned(in)) return UTF16_EINVAL;
    return run_single(in, nullptr, n, kModeCheck, first_bad, (cudaStream_t)stream, 0, 0);
}

int utf16_error_positions(const uint16_t *in, int64_t n, int64_t *positions, int64_t capacity, int64_t *count,
                          utf16_stream_t stream) {
    if (n < 0 || capacity < 0 || !count || (capacity > 0 && !positions)) return UTF16_EINVAL;
    if (n == 0) return empty_first_bad(count, (cudaStream_t)stream);
    if (!in || misaligned(in) || ((uintptr_t)positions & 7u)) return UTF16_EINVAL;
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const bool on_device = is_device_ptr(count);
    Slot *slot = nullptr;
    rc = ctx->slot_for(s, &slot);
    if (rc) return rc;
    SingleLaunch L;
    L.in = in;
    L.n = n;
    L.mode = kModeList;
    utf16_config cfg = ctx->single_config(n);
    cfg.single_variant = cfg.single_variant == kVariantTma ? kVariantLdg : cfg.single_variant;
    configure_single(ctx, cfg, L);
    L.slot = slot;
    L.result = on_device ? (long long *)count : &slot->result;
    L.positions = (long long *)positions;
    L.capacity = capacity;
    if (launch_single(L, s) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    if (!on_device) {
        if (cudaMemcpyAsync(count, &slot->result, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
    }
    return UTF16_OK;
}

int utf16_to_well_formed_batch(const uint16_t *in, uint16_t *out, const int64_t *offsets, int64_t num_strings,
                               utf16_stream_t stream) {
    if (num_strings < 0) return UTF16_EINVAL;
    if (num_strings == 0) return UTF16_OK;
    if (!in || !out || !offsets || misaligned(in) || misaligned(out) || ((uintptr_t)offsets & 7u)) return UTF16_EINVAL;
    return run_batch(in, out, offsets, num_strings, in == out ? kModeInPlace : kModeOut, nullptr,
                     (cudaStream_t)stream);
}

int utf16_to_well_formed_batch_inplace(uint16_t *buf, const int64_t *offsets, int64_t num_strings,
                                       utf16_stream_t stream) {
    if (num_strings < 0) return UTF16_EINVAL;
    if (num_strings == 0) return UTF16_OK;
    if (!buf || !offsets || misaligned(buf) || ((uintptr_t)offsets & 7u)) return UTF16_EINVAL;
    return run_batch(buf, buf, offsets, num_strings, kModeInPlace, nullptr, (cudaStream_t)stream);
}

int utf16_is_well_formed_batch(const uint16_t *in, const int64_t *offsets, int64_t num_strings, int64_t *first_bad,
                               utf16_stream_t stream) {
    if (num_strings < 0) return UTF16_EINVAL;
    if (num_strings == 0) return UTF16_OK;
    if (!in || !offsets || !first_bad || misaligned(in) || ((uintptr_t)offsets & 7u) || ((uintptr_t)first_bad & 7u))
        return UTF16_EINVAL;
    return run_batch(in, nullptr, offsets, num_strings, kModeCheck, first_bad, (cudaStream_t)stream);
}

int utf16_set_checked(int on) {
    g_checked.store(on != 0 ? 1 : 0, std::memory_order_relaxed);
    return UTF16_OK;
}

int utf16_get_checked(void) { return checked_mode() ? 1 : 0; }

int utf16_check_offsets(const int64_t *offsets, int64_t num_strings, int64_t *first_violation,
                        utf16_stream_t stream) {
    if (num_strings < 0 || !offsets || !first_violation || ((uintptr_t)offsets & 7u)) return UTF16_EINVAL;
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const bool on_device = is_device_ptr(first_violation);
    Slot *slot = nullptr;
    rc = ctx->slot_for(s, &slot);
    if (rc) return rc;
    long long *res = on_device ? (long long *)first_violation : &slot->result;
    if (launch_check_offsets((const long long *)offsets, num_strings, slot, res, ctx->sms * 8, s) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    if (!on_device) {
        if (cudaMemcpyAsync(first_violation, &slot->result, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
    }
    return UTF16_OK;
}

}  // extern "C"
