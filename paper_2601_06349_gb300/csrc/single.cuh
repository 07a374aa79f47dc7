// Per-chunk work of the single-string kernels, shared by the 128-bit-load
// kernel (single.cu) and the TMA-staged kernel (single_tma.cu).
#pragma once

#include <cuda_runtime.h>
#include <limits.h>

#include "device.cuh"
#include "internal.h"

namespace u16wf {

struct SingleArgs {
    const uint16_t *in;
    uint16_t *out;
    long long n;
    long long chunks;    // warp chunks of U*256 units covering [-a, n)
    Slot *slot;          // first-error reduction state (first-error kernels only)
    long long *result;   // where the last block stores the first-error index
    int a;               // misalignment of `in` in units
    uint32_t lead;       // unit just before in[0] (0 = none); a chunk of a longer string passes its neighbour
    uint32_t trail;      // unit just after in[n-1] (0 = none)
};

SingleArgs make_single_args(const SingleLaunch &L, int units_per_chunk);

// Unit p of the string, with the outside neighbours and zero elsewhere.
__device__ __forceinline__ uint32_t unit_at(const SingleArgs &A, long long p) {
    if (p >= 0 && p < A.n) return A.in[p];
    if (p == -1) return A.lead;
    if (p == A.n) return A.trail;
    return 0u;
}

// Load warp chunk c: 128-bit loads inside the string, unit loads at its ends.
template <int MODE, int U>
__device__ __forceinline__ void load_chunk(const SingleArgs &A, const uint4 *vin, long long c, int lane,
                                           uint4 (&v)[U]) {
    constexpr long long CU = (long long)U * kWarpSliceUnits;
    const long long cfirst = c * CU - A.a;
    if (cfirst >= 0 && cfirst + CU <= A.n) {
        const uint4 *p = vin + c * (32LL * U) + lane;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if constexpr (MODE == kModeInPlace)
                v[u] = ld_plain(p + 32 * u);
            else
                v[u] = ld_stream(p + 32 * u);
        }
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long p0 = cfirst + u * kWarpSliceUnits + lane * kUnitsPerVec;
            v[u] = make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int k = 0; k < 8; ++k) vec_set_unit(v[u], k, unit_at(A, p0 + k));
        }
    }
}

// Units of vector u of this lane that lie in [0, n), as an 8-bit mask.
__device__ __forceinline__ uint32_t valid_bits8(long long p0, long long n) {
    const long long lo = p0 < 0 ? -p0 : 0;
    const long long hi = n - p0 < 8 ? n - p0 : 8;
    if (hi <= lo) return 0u;
    return ((1u << hi) - 1u) & ~((1u << lo) - 1u);
}

// Steps 2-5 of the chunk starting at unit cfirst whose vectors are in v.
// `halo(p)` returns unit p for the two units just outside the chunk.
template <int MODE, bool FB, int ST, int U, class Halo>
__device__ __forceinline__ void process_chunk(const SingleArgs &A, long long cfirst, const uint4 (&v)[U], int lane,
                                              long long &my_first, Halo halo) {
    constexpr long long CU = (long long)U * kWarpSliceUnits;
    const bool edge = (cfirst < 0) || (cfirst + CU > A.n);
    const uint32_t surr = any_surrogate<U>(v);

    if (!__any_sync(kFull, surr != 0)) {
        // Well-formed chunk: copy out of place, nothing otherwise.
        if constexpr (MODE == kModeOut) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long p0 = cfirst + u * kWarpSliceUnits + lane * kUnitsPerVec;
                if (!edge) {
                    store_vec<ST>(A.out + p0, v[u]);
                } else {
                    const uint32_t w8 = valid_bits8(p0, A.n);
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (w8 & (1u << k)) A.out[p0 + k] = (uint16_t)vec_unit(v[u], k);
                }
            }
        }
        return;
    }

    // Slow path: locate the mismatched units, one vector at a time.
    uint32_t hp = 0, hn = 0;
    if (lane == 0) hp = unit_is_high(halo(cfirst - 1));
    if (lane == 31) hn = unit_is_low(halo(cfirst + CU));
    uint32_t from_prev, from_next;
    neighbour_bits<U>(v, hp, hn, lane, from_prev, from_next);
    bool found = false;
    uint32_t any_bad = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const long long p0 = cfirst + u * kWarpSliceUnits + lane * kUnitsPerVec;
        uint32_t bad_lo, bad_hi;
        vec_mismatch(v[u], (from_prev >> u) & 1u, (from_next >> u) & 1u, 0u, 0u, 0u, bad_lo, bad_hi);
        if (edge) {
            uint32_t vlo, vhi;
            bits_to_flags(valid_bits8(p0, A.n), vlo, vhi);
            bad_lo &= vlo;
            bad_hi &= vhi;
        }
        const bool vb = (bad_lo | bad_hi) != 0;
        any_bad |= bad_lo | bad_hi;
        if constexpr (MODE != kModeCheck) {
            if (MODE == kModeOut || vb) {
                const uint4 f = vb ? fix_vec(v[u], bad_lo, bad_hi) : v[u];
                if (!edge) {
                    if constexpr (MODE == kModeInPlace)
                        *reinterpret_cast<uint4 *>(A.out + p0) = f;
                    else
                        store_vec<ST>(A.out + p0, f);
                } else {
                    const uint32_t w8 = (MODE == kModeInPlace) ? (gather4(bad_lo) | (gather4(bad_hi) << 4))
                                                               : valid_bits8(p0, A.n);
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (w8 & (1u << k)) A.out[p0 + k] = (uint16_t)vec_unit(f, k);
                }
            }
        }
        if constexpr (FB) {
            if (vb && !found) {
                found = true;
                const long long p = p0 + first_flag(bad_lo, bad_hi);
                my_first = p < my_first ? p : my_first;
            }
        }
    }
    if constexpr (FB && MODE == kModeCheck) {
        // Publish early so that other warps can stop.
        if (__any_sync(kFull, any_bad != 0)) {
            const long long wmin = warp_min_ll(my_first);
            if (lane == 0) atomicMin(&A.slot->min, (unsigned long long)wmin);
        }
    }
}

// Block minimum, one atomic per block; the last block to finish publishes
// the first-error index and resets the slot for the next launch.
__device__ __forceinline__ void finish_first_bad(const SingleArgs &A, long long my_first, int lane) {
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

cudaError_t launch_single_tma(const SingleLaunch &L, cudaStream_t stream);
const void *single_tma_kernel_for_occupancy(int mode, bool fb);

}  // namespace u16wf
