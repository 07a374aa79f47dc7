// Validation of a ragged batch's offsets: the batch kernels require
// offsets[0] >= 0 and a non-decreasing array (string s is
// in[offsets[s] .. offsets[s+1]), Section 3.1's string ends taken per
// string).  One read of the array; the smallest violating index wins.
#include <cuda_runtime.h>
#include <limits.h>

#include "device.cuh"
#include "internal.h"

namespace u16wf {

// Index i in [0, count] violates when i == 0 and offsets[0] < 0, or i > 0 and
// offsets[i] < offsets[i - 1].  The last block publishes the smallest such
// index (or -1) and resets the slot.
__global__ void __launch_bounds__(kBlockThreads) check_offsets_kernel(const long long *offsets, long long count,
                                                                      Slot *slot, long long *result) {
    __shared__ unsigned long long s_min;
    wait_prior_grids();
    if (threadIdx.x == 0) s_min = ~0ull;
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned long long mine = ~0ull;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= count; i += stride) {
        const long long cur = offsets[i];
        const bool bad = (i == 0) ? (cur < 0) : (cur < offsets[i - 1]);
        if (bad) {
            mine = (unsigned long long)i;
            break;  // later indices of this thread are larger
        }
    }
    if (mine != ~0ull) atomicMin(&s_min, mine);
    allow_next_grid();
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (s_min != ~0ull) atomicMin(&slot->min, s_min);
    if (atomic_add_acq_rel(&slot->done, 1u) == gridDim.x - 1) {
        const unsigned long long g = ld_acquire(&slot->min);
        *result = (g == ~0ull) ? -1LL : (long long)g;
        slot->min = ~0ull;
        slot->done = 0u;
    }
}

cudaError_t launch_check_offsets(const long long *offsets, long long count, Slot *slot, long long *result,
                                 int max_blocks, cudaStream_t stream) {
    long long blocks = (count + 1 + kBlockThreads - 1) / kBlockThreads;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    void *args[] = {(void *)&offsets, (void *)&count, (void *)&slot, (void *)&result};
    return launch_kernel((const void *)check_offsets_kernel, dim3((unsigned)blocks), dim3(kBlockThreads), args, 0,
                         stream);
}

}  // namespace u16wf
