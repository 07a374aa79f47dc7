// toWellFormed + first-error index for callers that cannot allocate device
// memory.
//
// The regular entry point keeps its first-error scratch (one 32-byte slot per
// stream) in a pool that the library allocates with cudaMalloc on first use.
// Some callers cannot let a library do that: code whose device memory is all
// pre-reserved by a host framework or a fixed memory budget, code that runs
// with allocation forbidden after start-up (real-time or certified
// pipelines), or code that must not change the device's memory footprint.
// This entry point instead keeps its scratch in a fixed array compiled into
// the library (g_noalloc_scratch below): every GPU that loads the library
// holds those 256 bytes until the process exits, and the call itself
// allocates nothing -- no cudaMalloc, no cudaFree, no allocating library
// routine.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call clears the fields that must start at their initial
// value, in stream order, before its kernel runs.  Calls whose work overlaps
// on the GPU (different streams, or different host threads) race on it and
// give wrong first-error indices: serialise them.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/utf16wf.h"
#include "device.cuh"
#include "internal.h"
#include "runtime.h"

namespace u16wf {

// One first-error slot (32 bytes) in a 256-byte aligned array.
constexpr int kNoAllocSlots = 1;
static __device__ __align__(256) Slot g_noalloc_scratch[kNoAllocSlots];
static_assert(sizeof(Slot) * kNoAllocSlots <= 256, "the scratch array stays at 256 bytes");

// The longest string this entry point accepts.  The scratch it needs does not
// grow with n (always one slot), so this bound only keeps the kernel's 64-bit
// chunk arithmetic far from overflow: 2^40 units = 2 TiB of code units.
constexpr int64_t kNoAllocMaxUnits = 1LL << 40;

constexpr int kMaxDevices = 64;

struct NoAllocDevice {
    bool ready = false;
    Slot *scratch = nullptr;  // device address of g_noalloc_scratch on this device
    int sms = 0;
    // Persistent grid per kernel the call can launch: [in place][4-vector chunks].
    int max_blocks[2][2] = {{0, 0}, {0, 0}};
};

static std::mutex g_noalloc_mu;
static NoAllocDevice g_noalloc_dev[kMaxDevices];

// The data path of each form, as the regular entry points use by default:
// out of place one chunk at a time, in place with the next chunk's loads in
// flight.
static int noalloc_variant(bool in_place) { return in_place ? kVariantLdgPrefetch : kVariantLdg; }

// Set-up, once per device, with that device current: the device address of
// the array (host code cannot use the symbol itself) and the persistent grid
// size of every kernel the call can launch.  None of these calls allocates.
static int noalloc_setup(NoAllocDevice **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return UTF16_EINVAL;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDevice &d = g_noalloc_dev[dev];
    if (!d.ready) {
        Slot *ptr = nullptr;
        if (cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
        for (int ip = 0; ip < 2; ++ip) {
            for (int wide = 0; wide < 2; ++wide) {
                const void *fn = single_kernel_for_occupancy(ip ? kModeInPlace : kModeOut, true, wide ? 4 : 2,
                                                             noalloc_variant(ip != 0));
                int per_sm = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlockThreads, 0) != cudaSuccess ||
                    per_sm < 1) {
                    cudaGetLastError();
                    per_sm = 1;
                }
                d.max_blocks[ip][wide] = sms * per_sm;
            }
        }
        d.scratch = ptr;
        d.sms = sms;
        d.ready = true;
    }
    *out = &d;
    return UTF16_OK;
}

static bool noalloc_is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace u16wf

using namespace u16wf;

extern "C" int utf16_to_well_formed_first_bad_noalloc(const uint16_t *in, uint16_t *out, int64_t n,
                                                      int64_t *first_bad, utf16_stream_t stream) {
    if (n < 0 || !first_bad) return UTF16_EINVAL;
    if (n > kNoAllocMaxUnits) return UTF16_ETOOBIG;
    if (n > 0) {
        if (!in || !out || ((uintptr_t)in & 1u) || ((uintptr_t)out & 1u)) return UTF16_EINVAL;
        const uintptr_t x = (uintptr_t)in, y = (uintptr_t)out, b = (uintptr_t)n * 2u;
        if (x != y && x < y + b && y < x + b) return UTF16_EOVERLAP;
    }
    NoAllocDevice *d = nullptr;
    int rc = noalloc_setup(&d);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const bool on_device = noalloc_is_device_ptr(first_bad);
    if (n == 0) {
        if (on_device) {
            if (cudaMemsetAsync(first_bad, 0, sizeof(int64_t), s) != cudaSuccess) {
                cudaGetLastError();
                return UTF16_ECUDA;
            }
        } else {
            *first_bad = 0;
        }
        return UTF16_OK;
    }
    // The shared slot keeps whatever the previous call left: clear the
    // running minimum (all ones = none) and the finished-block counter.
    Slot *slot = d->scratch;
    if (cudaMemsetAsync(&slot->min, 0xFF, sizeof(slot->min), s) != cudaSuccess ||
        cudaMemsetAsync(&slot->done, 0, sizeof(slot->done), s) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    SingleLaunch L;
    L.in = in;
    L.out = out;
    L.n = n;
    const bool in_place = in == out;
    L.mode = in_place ? kModeInPlace : kModeOut;
    L.first_bad = true;
    L.variant = noalloc_variant(in_place);
    // Chunk width by size, as the regular entry points choose it: 2-vector
    // chunks below kAutoWideChunkUnitsPerSm units per SM spread a short string
    // over more SMs.
    const bool wide = n >= (int64_t)d->sms * kAutoWideChunkUnitsPerSm;
    L.units_per_thread = wide ? 4 : 2;
    L.max_blocks = d->max_blocks[in_place ? 1 : 0][wide ? 1 : 0];
    L.full_occupancy = true;
    L.slot = slot;
    L.result = on_device ? (long long *)first_bad : &slot->result;
    L.lead = 0;
    L.trail = 0;
    if (launch_single(L, s) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ECUDA;
    }
    if (!on_device) {
        if (cudaMemcpyAsync(first_bad, &slot->result, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return UTF16_ECUDA;
        }
    }
    return UTF16_OK;
}
