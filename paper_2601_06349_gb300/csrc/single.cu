// Single-string toWellFormed / isWellFormed kernels (Section 1 rule,
// Section 3.1 block algorithm recast for a warp).
//
// Data layout: the string in[0..n) is viewed as 16-byte vectors from the
// aligned address in - a (a = misalignment of `in` in units, 0..7); vector v
// holds units [8v - a, 8v - a + 8).  A warp chunk is U slices of 32
// consecutive vectors; chunk c starts at unit c * 256U - a.  Warps take
// chunks in grid-stride order, so a block of W warps streams 16*32*U*W
// contiguous bytes per step.
//
// Per chunk (Section 3.1, recast):
//   1. load the U vectors of each lane (128-bit loads; with PF the next
//      chunk's vectors are requested before this chunk is processed);
//   2. fast test: does any unit of the warp's chunk lie in 0xD800-0xDFFF?  If
//      not the chunk is well formed: out of place it is stored unchanged, in
//      place and read-only nothing is stored (Section 3.1: "the copy is
//      omitted" in place; the branchy design of the Discussion paragraph);
//   3. otherwise classify every unit high / low, take the neighbours from the
//      same vector, the adjacent lane (shuffle) or the units just outside the
//      chunk (halo), and replace mismatched units by U+FFFD.
// Chunks never depend on each other (no loop-carried state, as in the
// paper's Discussion of overlapping loads).
#include <cuda_runtime.h>
#include <limits.h>
#include <stdlib.h>

#include "device.cuh"
#include "internal.h"
#include "single.cuh"

namespace u16wf {

// The smallest mismatch index known so far (lane 0 returns it, ~0 if none),
// for the check's early exit.  Warp 0 of each block reads the global minimum
// and folds it into the block's shared best; every warp reads the shared
// best.  One global load per block per chunk step instead of one per warp:
// thousands of warps polling one word made a hot spot in L2 (the 1 GiB check
// at all resident blocks: 0.163 ms per pass without the poll, 0.20 with it).
__device__ __forceinline__ unsigned long long poll_known_mismatch(const SingleArgs &A, unsigned long long *blk_best,
                                                                  int lane) {
    if (lane != 0) return ~0ull;
    if ((threadIdx.x >> 5) == 0) {
        const unsigned long long g = *((volatile unsigned long long *)&A.slot->min);
        if (g != ~0ull) atomicMin(blk_best, g);
    }
    return *((volatile unsigned long long *)blk_best);
}

template <int MODE, bool FB, int ST, int U, bool PF>
__global__ void __launch_bounds__(kMaxBlockThreads) single_kernel(const SingleArgs A) {
    constexpr long long CU = (long long)U * kWarpSliceUnits;
    const int lane = threadIdx.x & 31;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const uint4 *vin = reinterpret_cast<const uint4 *>(A.in - A.a);
    long long my_first = LLONG_MAX;
    int filter = 0;                        // repair: step-two test on (see process_chunk)
    __shared__ unsigned long long s_best;  // check: this block's smallest published mismatch
    wait_prior_grids();
    if constexpr (MODE == kModeCheck) {
        if (threadIdx.x == 0) s_best = ~0ull;
        __syncthreads();
    }

    if constexpr (PF) {
        Chunk<U> nv;
        long long c = gwarp;
        if (c < A.chunks) load_chunk<MODE, U>(A, vin, c, lane, nv);
        while (c < A.chunks) {
            const Chunk<U> v = nv;
            const long long cur = c;
            c += nwarps;
            unsigned long long g = ~0ull;
            if constexpr (MODE == kModeCheck) {
                if (!A.full_pass) g = poll_known_mismatch(A, &s_best, lane);
            }
            if (c < A.chunks) load_chunk<MODE, U>(A, vin, c, lane, nv);
            const long long cfirst = cur * CU - A.a;
            if constexpr (MODE == kModeCheck) {
                // Early exit: a smaller error index is already known.
                g = __shfl_sync(kFull, g, 0);
                if (g != ~0ull && (long long)g < cfirst) break;
            }
            process_chunk<MODE, FB, ST, U>(A, cfirst, v, lane, my_first, &s_best, &filter);
        }
    } else {
        for (long long c = gwarp; c < A.chunks; c += nwarps) {
            const long long cfirst = c * CU - A.a;
            unsigned long long g = ~0ull;
            if constexpr (MODE == kModeCheck) {
                if (!A.full_pass) g = poll_known_mismatch(A, &s_best, lane);
            }
            Chunk<U> v;
            load_chunk<MODE, U>(A, vin, c, lane, v);
            if constexpr (MODE == kModeCheck) {
                g = __shfl_sync(kFull, g, 0);
                if (g != ~0ull && (long long)g < cfirst) break;
            }
            process_chunk<MODE, FB, ST, U>(A, cfirst, v, lane, my_first, &s_best, &filter);
        }
    }

    allow_next_grid();
    if constexpr (FB) finish_first_bad(A, my_first, lane);
    if constexpr (MODE == kModeList) finish_list(A);
}

template <int MODE, bool FB, int ST>
static const void *single_kernel_ptr(int u, bool pf) {
    if (pf) {
        switch (u) {
            case 2: return (const void *)single_kernel<MODE, FB, ST, 2, true>;
            default: return (const void *)single_kernel<MODE, FB, ST, 4, true>;
        }
    }
    switch (u) {
        case 2: return (const void *)single_kernel<MODE, FB, ST, 2, false>;
        default: return (const void *)single_kernel<MODE, FB, ST, 4, false>;
    }
}

static const void *pick_single(int mode, bool fb, int st, int u, bool pf) {
    if (mode == kModeCheck) return single_kernel_ptr<kModeCheck, true, 16>(u, pf);
    if (mode == kModeList) return single_kernel_ptr<kModeList, false, 16>(u, pf);
    if (mode == kModeInPlace)
        return fb ? single_kernel_ptr<kModeInPlace, true, 16>(u, pf) : single_kernel_ptr<kModeInPlace, false, 16>(u, pf);
    switch (st) {
        case 16: return fb ? single_kernel_ptr<kModeOut, true, 16>(u, pf) : single_kernel_ptr<kModeOut, false, 16>(u, pf);
        case 8: return fb ? single_kernel_ptr<kModeOut, true, 8>(u, pf) : single_kernel_ptr<kModeOut, false, 8>(u, pf);
        case 4: return fb ? single_kernel_ptr<kModeOut, true, 4>(u, pf) : single_kernel_ptr<kModeOut, false, 4>(u, pf);
        default: return fb ? single_kernel_ptr<kModeOut, true, 2>(u, pf) : single_kernel_ptr<kModeOut, false, 2>(u, pf);
    }
}

static int store_width(const SingleLaunch &L) {
    if (L.mode != kModeOut) return 16;
    const unsigned rel = (unsigned)(((uintptr_t)L.out - (uintptr_t)L.in) & 15u);
    return (rel == 0) ? 16 : (rel == 8) ? 8 : (rel % 4 == 0) ? 4 : 2;
}

SingleArgs make_single_args(const SingleLaunch &L, int units_per_chunk) {
    SingleArgs A;
    A.in = L.in;
    A.out = L.out;
    A.n = L.n;
    A.a = (int)(((uintptr_t)L.in & 15u) >> 1);
    A.chunks = (L.n + A.a + units_per_chunk - 1) / units_per_chunk;
    A.slot = L.slot;
    A.result = L.result;
    A.lead = L.lead;
    A.trail = L.trail;
    A.unit_stores = L.unit_stores ? 1 : 0;
    A.positions = L.positions;
    A.capacity = L.capacity;
    A.full_pass = L.full_pass ? 1 : 0;
    return A;
}

// In place with 4-vector chunks and 128-bit loads: the bit-word kernel
// (single_words.cu) on 2048-unit chunks.  On 1 GiB at 1e-2 lone surrogates,
// with the next chunk in flight: 225-232 us against 236 us, 28 M against
// 43 M warp-instructions (256 MiB case); error-free strings run as before.
constexpr int kWordsU = 8;
static bool use_words(const SingleLaunch &L) {
    return L.mode == kModeInPlace && L.variant != kVariantTma && L.units_per_thread != 2;
}

cudaError_t launch_single(const SingleLaunch &L, cudaStream_t stream) {
    if (L.variant == kVariantTma && store_width(L) == 16 && L.mode != kModeList)
        return launch_single_tma(L, stream);
    const bool words = use_words(L);
    const int U = words ? kWordsU : L.units_per_thread == 2 ? 2 : 4;
    const bool pf = L.variant == kVariantLdgPrefetch;
    const SingleArgs A = make_single_args(L, U * kWarpSliceUnits);
    const bool fb = (L.first_bad || L.mode == kModeCheck) && L.mode != kModeList;
    const void *fn = words ? inplace_words_kernel_for(fb, U, pf) : pick_single(L.mode, fb, store_width(L), U, pf);
    const int bt = L.block_threads;
    if (bt < 32 || bt > kMaxBlockThreads || bt % 32) return cudaErrorInvalidValue;
    const long long warps_per_block = bt / 32;
    long long blocks = (A.chunks + warps_per_block - 1) / warps_per_block;
    if (blocks > (long long)L.max_blocks) blocks = L.max_blocks;
    if (blocks < 1) blocks = 1;
    void *args[] = {(void *)&A};
    const long long warps = blocks * warps_per_block;
    return launch_kernel(fn, dim3((unsigned)blocks), dim3((unsigned)bt), args, 0, stream,
                         pdl_fits((A.chunks + warps - 1) / warps, L.full_occupancy));
}

bool g_pdl = false;
static thread_local bool t_pdl_off = false;
PdlOffScope::PdlOffScope() : saved(t_pdl_off) { t_pdl_off = true; }
PdlOffScope::~PdlOffScope() { t_pdl_off = saved; }

cudaError_t launch_kernel(const void *fn, dim3 grid, dim3 block, void **args, size_t smem, cudaStream_t stream,
                          bool pdl) {
    if (!g_pdl || !pdl || t_pdl_off) return cudaLaunchKernel(fn, grid, block, args, smem, stream);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

const void *single_kernel_for_occupancy(int mode, bool fb, int u, int variant) {
    if (variant == kVariantTma && mode != kModeList) return single_tma_kernel_for_occupancy(mode, fb);
    if (mode == kModeInPlace && u != 2) return inplace_words_kernel_for(fb, kWordsU, variant == kVariantLdgPrefetch);
    return pick_single(mode, fb, 16, u == 2 ? 2 : 4, variant == kVariantLdgPrefetch);
}

}  // namespace u16wf
