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
//   1. load the U vectors of each lane (128-bit loads);
//   2. fast test: does any unit of the warp's chunk lie in 0xD800-0xDFFF?  If
//      not the chunk is well formed: out of place it is stored unchanged, in
//      place and read-only nothing is stored (Section 3.1: "the copy is
//      omitted" in place; the branchy design of the Discussion paragraph);
//   3. otherwise classify every unit high / low, take the neighbours from the
//      same vector, the adjacent lane (shuffle) or the units just outside the
//      chunk (halo loads), and replace mismatched units by U+FFFD.
// Chunks never depend on each other (no loop-carried state, as in the
// paper's Discussion of overlapping loads).
#include <cuda_runtime.h>
#include <limits.h>

#include "device.cuh"
#include "internal.h"

namespace u16wf {

struct SingleArgs {
    const uint16_t *in;
    uint16_t *out;
    long long n;
    long long chunks;
    Slot *slot;          // first-error reduction state (FB only)
    long long *result;   // where the last block stores the first-error index (FB only)
    int a;               // misalignment of `in` in units
    uint32_t lead;       // unit just before in[0] (0 = none); a chunk of a longer string passes its neighbour
    uint32_t trail;      // unit just after in[n-1] (0 = none)
};

// Unit p of the string, with the outside neighbours and zero elsewhere.
__device__ __forceinline__ uint32_t unit_at(const SingleArgs &A, long long p) {
    if (p >= 0 && p < A.n) return A.in[p];
    if (p == -1) return A.lead;
    if (p == A.n) return A.trail;
    return 0u;
}

template <int MODE, bool FB, int ST, int U>
__global__ void __launch_bounds__(kBlockThreads) single_kernel(const SingleArgs A) {
    constexpr long long CU = (long long)U * kWarpSliceUnits;  // units per warp chunk
    const int lane = threadIdx.x & 31;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const uint4 *vin = reinterpret_cast<const uint4 *>(A.in - A.a);
    long long my_first = LLONG_MAX;

    for (long long c = gwarp; c < A.chunks; c += nwarps) {
        const long long cfirst = c * CU - A.a;  // unit index of the chunk's first unit
        if constexpr (MODE == kModeCheck) {
            // Early exit: a smaller error index is already known.
            unsigned long long g = 0;
            if (lane == 0) g = *((volatile unsigned long long *)&A.slot->min);
            g = __shfl_sync(kFull, g, 0);
            if (g != ~0ull && (long long)g < cfirst) break;
        }
        const bool edge = (cfirst < 0) || (cfirst + CU > A.n);
        uint4 v[U];
        uint32_t valid = 0xFFFFFFFFu;
        if (!edge) {
            const uint4 *p = vin + c * (32LL * U) + lane;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if constexpr (MODE == kModeInPlace)
                    v[u] = ld_plain(p + 32 * u);
                else
                    v[u] = ld_stream(p + 32 * u);
            }
        } else {
            valid = 0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long p0 = cfirst + u * kWarpSliceUnits + lane * kUnitsPerVec;
                v[u] = make_uint4(0, 0, 0, 0);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const long long p = p0 + k;
                    vec_set_unit(v[u], k, unit_at(A, p));
                    if (p >= 0 && p < A.n) valid |= 1u << (8 * u + k);
                }
            }
        }

        uint32_t surr = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) surr |= any_surrogate(v[u]);

        if (!__any_sync(kFull, surr != 0)) {
            // Well-formed chunk: copy out of place, nothing otherwise.
            if constexpr (MODE == kModeOut) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long p0 = cfirst + u * kWarpSliceUnits + lane * kUnitsPerVec;
                    if (!edge) {
                        store_vec<ST>(A.out + p0, v[u]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            if (valid & (1u << (8 * u + k))) A.out[p0 + k] = (uint16_t)vec_unit(v[u], k);
                    }
                }
            }
            continue;
        }

        // Slow path: locate the mismatched units.
        uint32_t h = 0, l = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            uint32_t hu, lu;
            classify8(v[u], hu, lu);
            h |= hu << (8 * u);
            l |= lu << (8 * u);
        }
        uint32_t halo_prev = 0, halo_next = 0;
        if (lane == 0) halo_prev = unit_is_high(unit_at(A, cfirst - 1));
        if (lane == 31) halo_next = unit_is_low(unit_at(A, cfirst + CU));
        const uint32_t bad = mismatch_mask<U>(h, l, halo_prev, halo_next, 0u, 0u, lane) & valid;

        if constexpr (MODE != kModeCheck) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t b8 = (bad >> (8 * u)) & 0xFFu;
                if (MODE == kModeInPlace && b8 == 0) continue;
                const long long p0 = cfirst + u * kWarpSliceUnits + lane * kUnitsPerVec;
                const uint4 f = fix_vec(v[u], b8);
                if (!edge) {
                    if constexpr (MODE == kModeInPlace)
                        *reinterpret_cast<uint4 *>(A.out + p0) = f;
                    else
                        store_vec<ST>(A.out + p0, f);
                } else {
                    const uint32_t w8 = (MODE == kModeInPlace) ? b8 : ((valid >> (8 * u)) & 0xFFu);
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (w8 & (1u << k)) A.out[p0 + k] = (uint16_t)vec_unit(f, k);
                }
            }
        }
        if constexpr (FB) {
            if (bad) {
                const int b = __ffs(bad) - 1;
                const long long p = cfirst + (b >> 3) * kWarpSliceUnits + lane * kUnitsPerVec + (b & 7);
                my_first = p < my_first ? p : my_first;
            }
            if constexpr (MODE == kModeCheck) {
                // Publish early so that other warps can stop.
                const long long wmin = warp_min_ll(my_first);
                if (lane == 0 && wmin != LLONG_MAX) atomicMin(&A.slot->min, (unsigned long long)wmin);
            }
        }
    }

    if constexpr (FB) {
        // Block minimum, one atomic per block, last block publishes and resets.
        __shared__ long long s_min[kBlockThreads / 32];
        __shared__ bool s_last;
        const long long wmin = warp_min_ll(my_first);
        if (lane == 0) s_min[threadIdx.x >> 5] = wmin;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long m = LLONG_MAX;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = s_min[w] < m ? s_min[w] : m;
            if (m != LLONG_MAX) atomicMin(&A.slot->min, (unsigned long long)m);
            __threadfence();
            const unsigned prev = atomicAdd(&A.slot->done, 1u);
            s_last = (prev == gridDim.x - 1);
        }
        __syncthreads();
        if (s_last && threadIdx.x == 0) {
            __threadfence();
            const unsigned long long g = atomicAdd(&A.slot->min, 0ull);
            *A.result = (g < (unsigned long long)A.n) ? (long long)g : A.n;
            A.slot->min = ~0ull;
            A.slot->done = 0u;
            __threadfence();
        }
    }
}

template <int MODE, bool FB, int ST>
static const void *single_kernel_ptr(int u) {
    switch (u) {
        case 1: return (const void *)single_kernel<MODE, FB, ST, 1>;
        case 2: return (const void *)single_kernel<MODE, FB, ST, 2>;
        default: return (const void *)single_kernel<MODE, FB, ST, 4>;
    }
}

static const void *pick_single(int mode, bool fb, int st, int u) {
    if (mode == kModeCheck) return single_kernel_ptr<kModeCheck, true, 16>(u);
    if (mode == kModeInPlace) return fb ? single_kernel_ptr<kModeInPlace, true, 16>(u)
                                        : single_kernel_ptr<kModeInPlace, false, 16>(u);
    switch (st) {
        case 16: return fb ? single_kernel_ptr<kModeOut, true, 16>(u) : single_kernel_ptr<kModeOut, false, 16>(u);
        case 8: return fb ? single_kernel_ptr<kModeOut, true, 8>(u) : single_kernel_ptr<kModeOut, false, 8>(u);
        case 4: return fb ? single_kernel_ptr<kModeOut, true, 4>(u) : single_kernel_ptr<kModeOut, false, 4>(u);
        default: return fb ? single_kernel_ptr<kModeOut, true, 2>(u) : single_kernel_ptr<kModeOut, false, 2>(u);
    }
}

cudaError_t launch_single(const SingleLaunch &L, cudaStream_t stream) {
    const int a = (int)(((uintptr_t)L.in & 15u) >> 1);
    int st = 16;
    if (L.mode == kModeOut) {
        const unsigned rel = (unsigned)(((uintptr_t)L.out - (uintptr_t)L.in) & 15u);
        st = (rel == 0) ? 16 : (rel == 8) ? 8 : (rel % 4 == 0) ? 4 : 2;
    }
    const int U = L.units_per_thread;
    const long long CU = (long long)U * kWarpSliceUnits;
    SingleArgs A;
    A.in = L.in;
    A.out = L.out;
    A.n = L.n;
    A.chunks = (L.n + a + CU - 1) / CU;
    A.slot = L.slot;
    A.result = L.result;
    A.a = a;
    A.lead = L.lead;
    A.trail = L.trail;
    const bool fb = L.first_bad || L.mode == kModeCheck;
    const void *fn = pick_single(L.mode, fb, st, U);
    const long long warps_per_block = kBlockThreads / 32;
    long long blocks = (A.chunks + warps_per_block - 1) / warps_per_block;
    const long long cap = (long long)L.max_blocks;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    void *args[] = {(void *)&A};
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(kBlockThreads), args, 0, stream);
}

const void *single_kernel_for_occupancy(int mode, bool fb, int u) { return pick_single(mode, fb, 16, u); }

}  // namespace u16wf
