// Internal interface between the kernels' translation units and the host
// runtime.  Not installed; the public ABI is include/utf16wf.h.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace u16wf {

struct Slot;

// Block size by default; launches may choose 128 to kMaxBlockThreads threads
// (the single-string and batch kernels are built for that maximum).
constexpr int kBlockThreads = 256;
constexpr int kMaxBlockThreads = 512;

enum Mode : int {
    kModeOut = 0,      // out-of-place repair
    kModeInPlace = 1,  // in-place repair, stores only changed 16-byte blocks
    kModeCheck = 2,    // read-only first-error index
    kModeInPlaceFirst = 3,  // batches only: in-place repair plus per-string first-error index
    kModeList = 4,          // single strings: positions of all mismatched units (unordered) and their count
};

// How the single-string kernels bring data in.
enum Variant : int {
    kVariantLdg = 0,          // 128-bit loads, one chunk at a time
    kVariantLdgPrefetch = 1,  // 128-bit loads, next chunk requested before this one is processed
    kVariantTma = 2,          // bulk copies (TMA) into a 4-stage shared-memory ring
};

struct SingleLaunch {
    const uint16_t *in = nullptr;
    uint16_t *out = nullptr;
    long long n = 0;
    int mode = kModeOut;
    bool first_bad = false;
    int units_per_thread = 4;  // U: 16-byte vectors per thread per chunk (2 or 4; TMA uses 4)
    int variant = kVariantLdg;
    int max_blocks = 1;        // persistent grid cap (SMs x resident blocks)
    Slot *slot = nullptr;
    long long *result = nullptr;
    uint32_t lead = 0, trail = 0;  // outside neighbours (0 = none)
    bool unit_stores = false;      // in place: 2-byte stores of the replaced units instead of 16-byte blocks
    long long *positions = nullptr;  // kModeList: output array
    long long capacity = 0;          // kModeList: its length
    bool full_pass = false;          // kModeCheck: read the whole string (no early exit), for timing
    bool full_occupancy = false;     // max_blocks is every block slot of the GPU
    int block_threads = kBlockThreads;  // 128-bit-load kernels; the TMA kernel always uses kBlockThreads
};

cudaError_t launch_single(const SingleLaunch &L, cudaStream_t stream);
const void *single_kernel_for_occupancy(int mode, bool fb, int u, int variant = kVariantLdg);
// In-place repair on bit words (single_words.cu), chunks of u = 4 or 8 slices.
const void *inplace_words_kernel_for(bool fb, int u, bool pf);
size_t single_tma_smem_bytes();
cudaError_t prepare_single_tma();
unsigned int read_and_clear_tma_timeout();
int run_bounded_wait_probe(long long limit_ns);  // 1: the wait gave up, 0: it completed, -1: CUDA error

struct BatchLaunch {
    const uint16_t *in = nullptr;
    uint16_t *out = nullptr;
    const long long *offsets = nullptr;
    long long count = 0;
    long long *first_bad = nullptr;  // kModeCheck and kModeInPlaceFirst
    int mode = kModeOut;
    int units_per_thread = 4;
    bool prefetch = false;
    int blocks = 1;                  // persistent grid size
    bool full_occupancy = false;     // blocks is every block slot of the GPU
    long long units_hint = 0;        // units in the batch when the caller knows them (0: unknown)
    int block_threads = kBlockThreads;
    int vector_bytes = 16;           // bytes per lane load: 8, 16 or 32
};

cudaError_t launch_batch(const BatchLaunch &L, cudaStream_t stream);
const void *batch_kernel_for_occupancy(int mode, int u, bool prefetch = false, int vector_bytes = 16);

// Smallest index violating "offsets[0] >= 0, non-decreasing" (or -1) into
// *result, through the stream's slot.
cudaError_t launch_check_offsets(const long long *offsets, long long count, Slot *slot, long long *result,
                                 int max_blocks, cudaStream_t stream);

// Launch with programmatic dependent launch when enabled and `pdl` allows it,
// else a plain launch.  pdl_fits(): short launches (at most
// kPdlMaxWorkPerWarp warp chunks per warp) are latency-bound and gain from
// overlapping the next launch with this one's end; a grid with every block
// slot of the GPU taken leaves the next launch no room to start early.  A
// long launch on a reduced grid measured slower with it (the 1 GiB check at
// 3 blocks per SM: 0.86 -> 0.79 of the copy peak back to back).
extern bool g_pdl;
// Off for this thread while it lives (the autotuner compares kernels, not
// overlaps between back-to-back launches).
struct PdlOffScope {
    PdlOffScope();
    ~PdlOffScope();
    bool saved;
};
constexpr long long kPdlMaxWorkPerWarp = 16;
inline bool pdl_fits(long long work_per_warp, bool full_occupancy) {
    return full_occupancy || work_per_warp <= kPdlMaxWorkPerWarp;
}
cudaError_t launch_kernel(const void *fn, dim3 grid, dim3 block, void **args, size_t smem, cudaStream_t stream,
                          bool pdl = true);

// Initialise a pool of scratch slots (min = all ones, done = 0).
cudaError_t init_slots(Slot *slots, int count, cudaStream_t stream);

}  // namespace u16wf
