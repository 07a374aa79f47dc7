// Ragged-batch toWellFormed / isWellFormed: many strings of uneven length in
// one launch.  String s is in[offsets[s] .. offsets[s+1]); every string end is
// a hard boundary (Section 3.1: a string that starts with a low or ends with a
// high surrogate has that unit replaced, whatever lies next to it in memory).
//
// The flattened unit range [offsets[0], offsets[count]) is read from the
// device and cut into warp chunks exactly as in the single-string kernel
// (U slices of 32 vectors of 8 units).  The grid is persistent and each warp
// owns a contiguous run of chunks, so consecutive chunks of a warp need
// consecutive entries of `offsets`.
//
// Per chunk:
//   - fast path: no surrogate in the chunk means nothing can be mismatched,
//     whatever the string boundaries; out of place the chunk is copied;
//   - slow path: the warp finds the first string starting at or after the
//     chunk by a 32-way search over `offsets` (a window of 32 consecutive
//     entries from the previous chunk's answer first), marks every string
//     start inside the chunk in a per-warp bitmask in shared memory, and
//     applies the pairing rule with "no left neighbour" at a start and "no
//     right neighbour" just before one.
#include <cuda_runtime.h>
#include <limits.h>

#include "device.cuh"
#include "internal.h"

namespace u16wf {

struct BatchArgs {
    const uint16_t *in;
    uint16_t *out;
    const long long *offsets;
    long long count;
    long long *first_bad;
    int a;  // misalignment of `in` in units
};

// Smallest s in [from, count] with offsets[s] >= key, or count + 1.
// Requires from == 0 or offsets[from - 1] < key.  Warp-collective.
__device__ __forceinline__ long long lower_bound_warp(const long long *offsets, long long count, long long from,
                                                      long long key, int lane) {
    long long lo = from, hi = count + 1;  // the answer lies in [lo, hi]
    long long stride = 1;                 // first a window of 32 consecutive entries
    while (lo < hi) {
        const long long idx = lo + stride * lane;
        const bool ge = (idx >= hi) || (offsets[idx] >= key);
        const unsigned m = __ballot_sync(kFull, ge);
        if (m == 0) {
            lo = lo + stride * 31 + 1;
        } else {
            const int j = __ffs(m) - 1;
            if (j == 0) return lo;
            const long long nlo = lo + stride * (j - 1) + 1;
            long long nhi = lo + stride * j;
            nhi = nhi < hi ? nhi : hi;
            if (stride == 1) return nhi;
            lo = nlo;
            hi = nhi;
        }
        stride = (hi - lo + 32) / 32;
    }
    return lo;
}

template <int MODE, int ST, int U>
__global__ void __launch_bounds__(kBlockThreads) batch_kernel(const BatchArgs A) {
    constexpr long long CU = (long long)U * kWarpSliceUnits;
    constexpr int kWords = (int)(CU / 32) + 1;  // bit CU marks a start just past the chunk
    __shared__ uint32_t s_bits[kBlockThreads / 32][kWords];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t *bits = s_bits[wib];

    const long long lo = A.offsets[0];
    const long long hi = A.offsets[A.count];
    if (lo < 0 || hi <= lo) return;
    const long long vbeg = (lo + A.a) >> 3;
    const long long vend = (hi + A.a + 7) >> 3;
    const long long chunks = (vend - vbeg + 32LL * U - 1) / (32LL * U);
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long c_begin = gwarp * chunks / nwarps;
    const long long c_end = (gwarp + 1) * chunks / nwarps;
    const uint4 *vin = reinterpret_cast<const uint4 *>(A.in - A.a);

    long long hint = 0;
    for (long long c = c_begin; c < c_end; ++c) {
        const long long vfirst = vbeg + c * (32LL * U);
        const long long cfirst = vfirst * 8 - A.a;
        const bool edge = (cfirst < lo) || (cfirst + CU > hi);
        uint4 v[U];
        uint32_t valid = 0xFFFFFFFFu;
        if (!edge) {
            const uint4 *p = vin + vfirst + lane;
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
                    if (p >= lo && p < hi) {
                        vec_set_unit(v[u], k, A.in[p]);
                        valid |= 1u << (8 * u + k);
                    }
                }
            }
        }
        if constexpr (U < 4) valid &= (1u << (8 * U)) - 1u;

        uint32_t surr = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) surr |= any_surrogate(v[u]);

        if (!__any_sync(kFull, surr != 0)) {
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

        // String starts in [cfirst, cfirst + CU].
        for (int i = lane; i < kWords; i += 32) bits[i] = 0u;
        __syncwarp();
        const long long s_first = lower_bound_warp(A.offsets, A.count, hint, cfirst, lane);
        hint = s_first;
        long long s_last = s_first - 1;  // last string index starting in the chunk
        for (long long base = s_first;; base += 32) {
            const long long idx = base + lane;
            const long long off = idx <= A.count ? A.offsets[idx] : LLONG_MAX;
            const bool inside = off >= cfirst && off <= cfirst + CU;
            if (inside) {
                const long long r = off - cfirst;
                atomicOr(&bits[r >> 5], 1u << (r & 31));
            }
            const unsigned m = __ballot_sync(kFull, inside);
            s_last = base + __popc(m) - 1 > s_last ? base + __popc(m) - 1 : s_last;
            if (m != kFull) break;
        }
        __syncwarp();
        uint32_t no_prev = 0, no_next = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r0 = u * kWarpSliceUnits + lane * kUnitsPerVec;
            const unsigned long long w2 =
                (unsigned long long)bits[r0 >> 5] | ((unsigned long long)bits[(r0 >> 5) + 1] << 32);
            const uint32_t s9 = (uint32_t)(w2 >> (r0 & 31)) & 0x1FFu;  // starts at units r0 .. r0+8
            no_prev |= (s9 & 0xFFu) << (8 * u);
            no_next |= ((s9 >> 1) & 0xFFu) << (8 * u);
        }

        uint32_t h = 0, l = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            uint32_t hu, lu;
            classify8(v[u], hu, lu);
            h |= hu << (8 * u);
            l |= lu << (8 * u);
        }
        uint32_t halo_prev = 0, halo_next = 0;
        if (lane == 0) {
            const long long p = cfirst - 1;
            halo_prev = (p >= lo && p < hi) ? unit_is_high(A.in[p]) : 0u;
        }
        if (lane == 31) {
            const long long p = cfirst + CU;
            halo_next = (p >= lo && p < hi) ? unit_is_low(A.in[p]) : 0u;
        }
        const uint32_t bad = mismatch_mask<U>(h, l, halo_prev, halo_next, no_prev, no_next, lane) & valid;

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
        } else {
            // Per-string first-error index: the first bad unit of each string
            // within this thread's units, one atomic per (thread, string).
            uint32_t rest = bad;
            long long prev_s = -1;
            const long long s_lo = hint > 0 ? hint - 1 : 0;
            while (rest) {
                const int b = __ffs(rest) - 1;
                rest &= rest - 1;
                const long long p = cfirst + (b >> 3) * kWarpSliceUnits + lane * kUnitsPerVec + (b & 7);
                long long a_i = s_lo, b_i = s_last > s_lo ? s_last : s_lo;
                while (a_i < b_i) {  // largest index with offsets[index] <= p
                    const long long mid = (a_i + b_i + 1) >> 1;
                    if (A.offsets[mid] <= p)
                        a_i = mid;
                    else
                        b_i = mid - 1;
                }
                a_i = a_i < A.count - 1 ? a_i : A.count - 1;
                if (a_i != prev_s) {
                    prev_s = a_i;
                    atomicMin(&A.first_bad[a_i], p - A.offsets[a_i]);
                }
            }
        }
    }
}

// first_bad[s] = length of string s (the value for a well-formed string).
__global__ void batch_lengths_kernel(const long long *offsets, long long count, long long *first_bad) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        first_bad[i] = offsets[i + 1] - offsets[i];
}

template <int MODE, int ST>
static const void *batch_ptr(int u) {
    switch (u) {
        case 1: return (const void *)batch_kernel<MODE, ST, 1>;
        case 2: return (const void *)batch_kernel<MODE, ST, 2>;
        default: return (const void *)batch_kernel<MODE, ST, 4>;
    }
}

static const void *pick_batch(int mode, int st, int u) {
    if (mode == kModeCheck) return batch_ptr<kModeCheck, 16>(u);
    if (mode == kModeInPlace) return batch_ptr<kModeInPlace, 16>(u);
    switch (st) {
        case 16: return batch_ptr<kModeOut, 16>(u);
        case 8: return batch_ptr<kModeOut, 8>(u);
        case 4: return batch_ptr<kModeOut, 4>(u);
        default: return batch_ptr<kModeOut, 2>(u);
    }
}

cudaError_t launch_batch(const BatchLaunch &L, cudaStream_t stream) {
    BatchArgs A;
    A.in = L.in;
    A.out = L.out;
    A.offsets = L.offsets;
    A.count = L.count;
    A.first_bad = L.first_bad;
    A.a = (int)(((uintptr_t)L.in & 15u) >> 1);
    int st = 16;
    if (L.mode == kModeOut) {
        const unsigned rel = (unsigned)(((uintptr_t)L.out - (uintptr_t)L.in) & 15u);
        st = (rel == 0) ? 16 : (rel == 8) ? 8 : (rel % 4 == 0) ? 4 : 2;
    }
    if (L.mode == kModeCheck) {
        long long blocks = (L.count + kBlockThreads - 1) / kBlockThreads;
        if (blocks > L.blocks) blocks = L.blocks;
        if (blocks < 1) blocks = 1;
        batch_lengths_kernel<<<(unsigned)blocks, kBlockThreads, 0, stream>>>(L.offsets, L.count, L.first_bad);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const void *fn = pick_batch(L.mode, st, L.units_per_thread);
    void *args[] = {(void *)&A};
    return cudaLaunchKernel(fn, dim3((unsigned)L.blocks), dim3(kBlockThreads), args, 0, stream);
}

const void *batch_kernel_for_occupancy(int mode, int u) { return pick_batch(mode, 16, u); }

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
