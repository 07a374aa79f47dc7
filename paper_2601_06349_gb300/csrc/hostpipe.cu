// toWellFormed plus first-error index on host buffers.
//
// Both buffers page-locked (pinned): one pass of the fused kernel reads the
// input and writes the output over the host link itself, no staging.
//
// Otherwise: chunks of the string go host -> device, are repaired in place in
// a device staging buffer and go back, on three library-owned streams so
// that both copy directions and the kernels of different chunks overlap.
// Each chunk gets its outside neighbours (the units just before and after it
// in the whole string) from the host buffer, so the chunked result equals the
// whole-string result (the rule reads only a unit's immediate neighbours,
// Section 1).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <vector>

#include "../../include/utf16wf.h"
#include "runtime.h"

namespace u16wf {

static int64_t host_chunk_units() {
    const char *s = getenv("UTF16WF_HOST_CHUNK_UNITS");
    long long v = (s && *s) ? atoll(s) : (4LL << 20);
    if (v < 4096) v = 4096;
    return (int64_t)v;
}

static int ensure_lanes(DeviceCtx *ctx) {
    if (!ctx->lanes[0]) {
        for (int i = 0; i < kHostLanes; ++i)
            if (cudaStreamCreateWithFlags(&ctx->lanes[i], cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                return UTF16_ECUDA;
            }
    }
    return UTF16_OK;
}

int DeviceCtx::ensure_staging(int64_t units, int64_t chunks) {
    const int rc = ensure_lanes(this);
    if (rc) return rc;
    if (stage_units < units) {
        for (int i = 0; i < kHostLanes; ++i) {
            if (stage[i]) cudaFree(stage[i]);
            stage[i] = nullptr;
        }
        stage_units = 0;
        for (int i = 0; i < kHostLanes; ++i)
            if (cudaMalloc((void **)&stage[i], (size_t)units * 2u) != cudaSuccess) {
                cudaGetLastError();
                return UTF16_ENOMEM;
            }
        stage_units = units;
    }
    if (chunk_first_cap < chunks) {
        if (chunk_first) cudaFreeHost(chunk_first);
        chunk_first = nullptr;
        chunk_first_cap = 0;
        if (cudaHostAlloc((void **)&chunk_first, (size_t)chunks * sizeof(int64_t), cudaHostAllocDefault) !=
            cudaSuccess) {
            cudaGetLastError();
            return UTF16_ENOMEM;
        }
        chunk_first_cap = chunks;
    }
    return UTF16_OK;
}

void DeviceCtx::release_staging() {
    for (int i = 0; i < kHostLanes; ++i) {
        if (stage[i]) cudaFree(stage[i]);
        stage[i] = nullptr;
        if (lanes[i]) cudaStreamDestroy(lanes[i]);
        lanes[i] = nullptr;
    }
    stage_units = 0;
    if (chunk_first) cudaFreeHost(chunk_first);
    chunk_first = nullptr;
    chunk_first_cap = 0;
}

static bool is_device_memory(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice;
}

// Device address of `bytes` bytes of page-locked host memory at p, or
// nullptr when any of them is not page-locked (one mapping end to end).
const void *pinned_view(const void *p, int64_t bytes) {
    cudaPointerAttributes a, b;
    const char *last = (const char *)p + bytes - 1;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    if ((const char *)b.devicePointer - (const char *)a.devicePointer != bytes - 1) return nullptr;
    return a.devicePointer;
}

const void *host_view(DeviceCtx *ctx, const void *p, int64_t bytes) {
    if (const void *v = pinned_view(p, bytes)) return v;
    if (!ctx->pageable_access) return nullptr;
    const char *e = getenv("UTF16WF_HOST_PAGEABLE_DIRECT");
    if (e && *e && atoi(e) == 0) return nullptr;
    return p;
}

// Both buffers visible to kernels (pinned, or pageable memory on a device
// that accesses it coherently): one fused pass on a library stream.
static int host_direct(DeviceCtx *ctx, const uint16_t *din, uint16_t *dout, int64_t n, int64_t *first_bad_host) {
    int rc = ensure_lanes(ctx);
    if (rc) return rc;
    cudaStream_t s = ctx->lanes[0];
    Slot *slot;
    rc = ctx->slot_for(s, &slot);
    if (rc) return rc;
    SingleLaunch L;
    L.in = din;
    L.out = dout;
    L.n = n;
    L.mode = din == dout ? kModeInPlace : kModeOut;
    L.first_bad = true;
    utf16_config cfg = ctx->single_config(n);
    // Host memory is far: keep the next chunk's loads in flight (and no bulk copies).
    cfg.single_variant = cfg.inplace_variant = kVariantLdgPrefetch;
    configure_single(ctx, cfg, L);
    L.slot = slot;
    L.result = &slot->result;
    int64_t fb = n;
    if (launch_single(L, s) != cudaSuccess ||
        cudaMemcpyAsync(&fb, &slot->result, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    if (first_bad_host) *first_bad_host = fb;
    return UTF16_OK;
}

}  // namespace u16wf

using namespace u16wf;

extern "C" int utf16_to_well_formed_host(const uint16_t *host_in, uint16_t *host_out, int64_t n,
                                         int64_t *first_bad_host) {
    if (n < 0) return UTF16_EINVAL;
    if (n == 0) {
        if (first_bad_host) *first_bad_host = 0;
        return UTF16_OK;
    }
    if (!host_in || !host_out || ((uintptr_t)host_in & 1u) || ((uintptr_t)host_out & 1u)) return UTF16_EINVAL;
    if (is_device_memory(host_in) || is_device_memory(host_out)) return UTF16_EINVAL;
    {
        const uintptr_t x = (uintptr_t)host_in, y = (uintptr_t)host_out, b = (uintptr_t)n * 2u;
        if (x != y && x < y + b && y < x + b) return UTF16_EOVERLAP;
    }
    DeviceCtx *ctx;
    int rc = get_ctx(&ctx);
    if (rc) return rc;

    std::lock_guard<std::mutex> lk(ctx->stage_mu);
    {
        const void *din = host_view(ctx, host_in, n * 2);
        const void *dout = din ? (host_out == host_in ? din : host_view(ctx, host_out, n * 2)) : nullptr;
        if (din && dout) return host_direct(ctx, (const uint16_t *)din, (uint16_t *)dout, n, first_bad_host);
    }
    const int64_t chunk = host_chunk_units();
    const int64_t chunks = (n + chunk - 1) / chunk;
    rc = ctx->ensure_staging(n < chunk ? n : chunk, chunks);
    if (rc) return rc;

    // Outside neighbours of every chunk, read before any result is copied
    // back (host_out may be host_in).
    std::vector<uint32_t> lead((size_t)chunks), trail((size_t)chunks);
    for (int64_t k = 0; k < chunks; ++k) {
        const int64_t c0 = k * chunk, c1 = (c0 + chunk < n) ? c0 + chunk : n;
        lead[(size_t)k] = c0 > 0 ? host_in[c0 - 1] : 0u;
        trail[(size_t)k] = c1 < n ? host_in[c1] : 0u;
    }

    Slot *slots[kHostLanes];
    for (int i = 0; i < kHostLanes; ++i) {
        rc = ctx->slot_for(ctx->lanes[i], &slots[i]);
        if (rc) return rc;
    }
    for (int64_t k = 0; k < chunks; ++k) {
        const int lane = (int)(k % kHostLanes);
        cudaStream_t s = ctx->lanes[lane];
        uint16_t *buf = ctx->stage[lane];
        const int64_t c0 = k * chunk, len = (c0 + chunk < n) ? chunk : n - c0;
        if (cudaMemcpyAsync(buf, host_in + c0, (size_t)len * 2u, cudaMemcpyHostToDevice, s) != cudaSuccess)
            goto cuda_fail;
        {
            SingleLaunch L;
            L.in = buf;
            L.out = buf;
            L.n = len;
            L.mode = kModeInPlace;
            L.first_bad = true;
            configure_single(ctx, ctx->single_config(len), L);
            L.slot = slots[lane];
            L.result = &slots[lane]->result;
            L.lead = lead[(size_t)k];
            L.trail = trail[(size_t)k];
            if (launch_single(L, s) != cudaSuccess) goto cuda_fail;
        }
        if (cudaMemcpyAsync(&ctx->chunk_first[k], &slots[lane]->result, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
            goto cuda_fail;
        if (cudaMemcpyAsync(host_out + c0, buf, (size_t)len * 2u, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            goto cuda_fail;
    }
    for (int i = 0; i < kHostLanes; ++i)
        if (cudaStreamSynchronize(ctx->lanes[i]) != cudaSuccess) goto cuda_fail;
    if (first_bad_host) {
        int64_t fb = n;
        for (int64_t k = 0; k < chunks; ++k) {
            const int64_t c0 = k * chunk, len = (c0 + chunk < n) ? chunk : n - c0;
            if (ctx->chunk_first[k] < len) {
                fb = c0 + ctx->chunk_first[k];
                break;
            }
        }
        *first_bad_host = fb;
    }
    return UTF16_OK;

cuda_fail:
    cudaGetLastError();
    for (int i = 0; i < kHostLanes; ++i) cudaStreamSynchronize(ctx->lanes[i]);
    cudaGetLastError();
    return UTF16_ECUDA;
}
