// Internal interface between the kernels' translation units and the host
// runtime.  Not installed; the public ABI is include/utf16wf.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace u16wf {

struct Slot;

constexpr int kBlockThreads = 256;

enum Mode : int {
    kModeOut = 0,      // out-of-place repair
    kModeInPlace = 1,  // in-place repair, stores only changed 16-byte blocks
    kModeCheck = 2,    // read-only first-error index
};

struct SingleLaunch {
    const uint16_t *in;
    uint16_t *out;
    long long n;
    int mode;
    bool first_bad;
    int units_per_thread;  // U: 16-byte vectors per thread per chunk (1, 2 or 4)
    int max_blocks;        // persistent grid cap (SMs x resident blocks)
    Slot *slot;
    long long *result;
    uint32_t lead, trail;  // outside neighbours (0 = none)
};

cudaError_t launch_single(const SingleLaunch &L, cudaStream_t stream);
const void *single_kernel_for_occupancy(int mode, bool fb, int u);

struct BatchLaunch {
    const uint16_t *in;
    uint16_t *out;
    const long long *offsets;
    long long count;
    long long *first_bad;  // kModeCheck only
    int mode;
    int units_per_thread;
    int blocks;            // persistent grid size
};

cudaError_t launch_batch(const BatchLaunch &L, cudaStream_t stream);
const void *batch_kernel_for_occupancy(int mode, int u);

// Initialise a pool of scratch slots (min = all ones, done = 0).
cudaError_t init_slots(Slot *slots, int count, cudaStream_t stream);

}  // namespace u16wf
