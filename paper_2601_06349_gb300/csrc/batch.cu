// Ragged-batch entry points' launch logic (the kernels are in batch.cuh):
// the lengths kernel for the per-string forms, the choice of kernel by form,
// chunk width, vector width and store class, and the launch.
#include <cuda_runtime.h>

#include "batch.cuh"

namespace u16wf {

// first_bad[s] = length of string s (the value for a well-formed string).
// The next grid (the check) may start as soon as this one has waited for
// its own predecessors: it reads only what those wrote before its first
// atomic on first_bad, where it waits for this grid, so this grid's
// duration is on the check's path.  Each thread takes kLengthsPerThread
// strings (a block stride apart, so that every load is coalesced) and issues
// all their loads before its first store: one memory latency per pass
// instead of one per string (1M strings: the check 43.1 -> 41.8 us; one
// string per thread in 4x the blocks 44.7).
constexpr int kLengthsPerThread = 4;
__global__ void batch_lengths_kernel(const long long *offsets, long long count, long long *first_bad) {
    wait_prior_grids();
    allow_next_grid();
    constexpr int K = kLengthsPerThread;
    const long long stride = (long long)gridDim.x * blockDim.x * K;
    for (long long b = (long long)blockIdx.x * blockDim.x * K + threadIdx.x; b < count; b += stride) {
        long long s[K], e[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const long long i = b + (long long)k * blockDim.x;
            s[k] = 0;
            e[k] = 0;
            if (i < count) {
                s[k] = offsets[i];
                e[k] = offsets[i + 1];
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const long long i = b + (long long)k * blockDim.x;
            if (i < count) first_bad[i] = e[k] - s[k];
        }
    }
}

// Chunk width of each form when the configuration leaves it open (0):
// 1024 units out of place (1M strings: 69.5 against 72.8 us), 2048 for the
// rest (in place 66 against 69 us, check 43 against 50 us).
static int batch_u(int mode, int u) { return u == 2 || u == 4 ? u : mode == kModeOut ? 2 : 4; }
static int batch_vb(int vb) { return vb == 8 || vb == 32 ? vb : 16; }

static const void *pick_batch(int mode, int st, int nw, int vb, bool pf) {
    switch (mode) {
        case kModeCheck: return words_kernel_ptr<kModeCheck, 8>(nw, vb, pf);
        case kModeInPlaceFirst: return words_kernel_ptr<kModeInPlaceFirst, 8>(nw, vb, pf);
        case kModeInPlace: return words_kernel_ptr<kModeInPlace, 8>(nw, vb, pf);
        default: return batch_out_kernel(st, nw, vb, pf);
    }
}

cudaError_t launch_batch(const BatchLaunch &L, cudaStream_t stream) {
    const int vb = batch_vb(L.vector_bytes);
    const int nw = batch_u(L.mode, L.units_per_thread) == 2 ? 1 : 2;
    const int bt = L.block_threads;
    if (bt < 32 || bt > kMaxBlockThreads || bt % 32) return cudaErrorInvalidValue;
    BatchArgs A;
    A.in = L.in;
    A.out = L.out;
    A.offsets = L.offsets;
    A.count = L.count;
    A.first_bad = L.first_bad;
    A.a = (int)(((uintptr_t)L.in & (uintptr_t)(vb - 1)) >> 1);
    const int st = L.mode == kModeOut ? lv_store_class(L.in, L.out, vb) : 8;
    const void *fn = pick_batch(L.mode, st, nw, vb, L.prefetch);
    if (!fn) return cudaErrorInvalidValue;
    if (L.mode == kModeCheck || L.mode == kModeInPlaceFirst) {
        // One pass over the strings where it fits in four times the batch
        // kernel's grid.
        long long blocks = (L.count + kBlockThreads * kLengthsPerThread - 1) / (kBlockThreads * kLengthsPerThread);
        if (blocks > 4LL * L.blocks) blocks = 4LL * L.blocks;
        if (blocks < 1) blocks = 1;
        const long long *offsets = L.offsets;
        long long count = L.count;
        long long *first_bad = L.first_bad;
        void *largs[] = {(void *)&offsets, (void *)&count, (void *)&first_bad};
        cudaError_t e = launch_kernel((const void *)batch_lengths_kernel, dim3((unsigned)blocks), dim3(kBlockThreads),
                                      largs, 0, stream);
        if (e != cudaSuccess) return e;
    }
    void *args[] = {(void *)&A};
    const long long warps = (long long)L.blocks * (bt / 32);
    const long long chunk_units = 1024LL * nw;
    // The per-string forms overlap the lengths kernel before them (they wait
    // only before their first atomic), which needs the attribute.
    const bool pdl = L.mode == kModeCheck || L.mode == kModeInPlaceFirst || L.full_occupancy ||
                     (L.units_hint > 0 && pdl_fits((L.units_hint / chunk_units + warps) / warps, false));
    return launch_kernel(fn, dim3((unsigned)L.blocks), dim3((unsigned)bt), args, 0, stream, pdl);
}

const void *batch_kernel_for_occupancy(int mode, int u, bool prefetch, int vector_bytes) {
    const int vb = batch_vb(vector_bytes);
    return pick_batch(mode, mode == kModeOut ? vb : 8, batch_u(mode, u) == 2 ? 1 : 2, vb, prefetch);
}

// ---------------------------------------------------------------------------
__global__ void init_slots_kernel(Slot *slots, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        slots[i].min = ~0ull;
        slots[i].done = 0u;
        slots[i].pad0 = 0u;
        slots[i].result = 0;
        slots[i].pad1 = 0;
    }
}

cudaError_t init_slots(Slot *slots, int count, cudaStream_t stream) {
    init_slots_kernel<<<(count + 255) / 256, 256, 0, stream>>>(slots, count);
    return cudaGetLastError();
}

}  // namespace u16wf
