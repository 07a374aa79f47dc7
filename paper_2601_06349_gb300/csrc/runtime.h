// Host-side runtime state shared by the entry points (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <unordered_map>
#include <utility>

#include "../../include/utf16wf.h"
#include "device.cuh"
#include "internal.h"

namespace u16wf {

constexpr int kSlotCount = 4096;
constexpr int kHostLanes = 3;
constexpr int kBuckets = 64;  // log2 size buckets for tuned launch configurations

// Default chunk width by size: strings shorter than this many units per SM
// take 2-vector chunks, longer ones 4-vector chunks.
constexpr long long kAutoWideChunkUnitsPerSm = 40960;

struct DeviceCtx {
    int device = 0;
    int sms = 1;
    bool pageable_access = false;  // kernels may read and write pageable host memory (coherently)
    std::mutex mu;
    Slot *slots = nullptr;  // device pool of kSlotCount slots
    int slots_used = 0;
    std::unordered_map<cudaStream_t, int> slot_of;
    std::map<std::pair<const void *, int>, int> occupancy;  // (kernel, block size) -> resident blocks per SM

    // Launch configuration: the default, and per log2 bucket what the
    // autotuner measured best (single strings: bucket of n; batches: bucket
    // of the mean string length).
    utf16_config def;
    utf16_config single_tuned[kBuckets];
    bool single_has[kBuckets] = {};
    utf16_config batch_tuned[kBuckets];
    bool batch_has[kBuckets] = {};

    // Host-buffer pipeline: kHostLanes streams, each with a device staging
    // buffer of `stage_units` units; pinned per-chunk first-error results.
    std::mutex stage_mu;
    cudaStream_t lanes[kHostLanes] = {nullptr, nullptr, nullptr};
    uint16_t *stage[kHostLanes] = {nullptr, nullptr, nullptr};
    int64_t stage_units = 0;
    int64_t *chunk_first = nullptr;  // pinned host
    int64_t chunk_first_cap = 0;

    int per_sm(const void *fn, size_t smem, int threads = kBlockThreads);
    int slot_for(cudaStream_t s, Slot **out);
    int ensure_staging(int64_t units, int64_t chunks);
    void release_staging();
    utf16_config single_config(int64_t n);
    utf16_config batch_config(int64_t units, int64_t count);
};

int get_ctx(DeviceCtx **out);
int bucket_of(int64_t v);

// Fill a single-string launch from a configuration (grid size included).
void configure_single(DeviceCtx *ctx, const utf16_config &cfg, SingleLaunch &L);
void configure_batch(DeviceCtx *ctx, const utf16_config &cfg, BatchLaunch &L);

// Single-string launch with optional first-error output (host or device
// pointer) and outside neighbours `lead` / `trail` (0 = none).
int run_single(const uint16_t *in, uint16_t *out, int64_t n, int mode, int64_t *first_bad, cudaStream_t stream,
               uint32_t lead, uint32_t trail);

int run_batch(const uint16_t *in, uint16_t *out, const int64_t *offsets, int64_t count, int mode, int64_t *first_bad,
              cudaStream_t stream);

// Device address of `bytes` bytes of page-locked, mapped host memory at p, or
// nullptr when any of them is not (checks both ends of the range).
const void *pinned_view(const void *p, int64_t bytes);

// Device address of a host range for a kernel: its pinned view, else on a
// device that accesses pageable memory coherently the address itself
// (unless UTF16WF_HOST_PAGEABLE_DIRECT=0), else nullptr.
const void *host_view(DeviceCtx *ctx, const void *p, int64_t bytes);

}  // namespace u16wf
