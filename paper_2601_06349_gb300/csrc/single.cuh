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
    int unit_stores;     // in place: store replaced units one by one (2 bytes) instead of their 16-byte block
    long long *positions;  // list mode: positions of mismatched units (unordered), `capacity` entries
    long long capacity;
    int full_pass;         // check: no early exit (the autotuner times a whole pass)
};

SingleArgs make_single_args(const SingleLaunch &L, int units_per_chunk);

// Unit p of the string, with the outside neighbours and zero elsewhere.
__device__ __forceinline__ uint32_t unit_at(const SingleArgs &A, long long p) {
    if (p >= 0 && p < A.n) return A.in[p];
    if (p == -1) return A.lead;
    if (p == A.n) return A.trail;
    return 0u;
}

// A loaded warp chunk: this lane's U vectors, and (lanes 0 and 31) the units
// just before and after the chunk, which the slow path needs as neighbours.
template <int U>
struct Chunk {
    uint4 v[U];
    uint32_t halo;
};

// Load warp chunk c: 128-bit loads inside the string, unit loads at its ends.
template <int MODE, int U>
__device__ __forceinline__ void load_chunk(const SingleArgs &A, const uint4 *vin, long long c, int lane,
                                           Chunk<U> &ch) {
    constexpr long long CU = (long long)U * kWarpSliceUnits;
    const long long cfirst = c * CU - A.a;
    if (cfirst >= 0 && cfirst + CU <= A.n) {
        const uint4 *p = vin + c * (32LL * U) + lane;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if constexpr (MODE == kModeInPlace)
                ch.v[u] = ld_plain(p + 32 * u);
            else
                ch.v[u] = ld_stream(p + 32 * u);
        }
    } else if constexpr (MODE == kModeCheck && U == 4) {
        // The check on 4-vector chunks (strings from about 6.2M units, where
        // one end chunk is a small share of the call) keeps unit loads: either
        // whole-vector form costs its kernel 9 registers (40 -> 49: 6 -> 4
        // resident blocks of 256 threads, 1 GiB well formed 176 -> 187 us).
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long p0 = cfirst + u * kWarpSliceUnits + lane * kUnitsPerVec;
            ch.v[u] = make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int k = 0; k < 8; ++k) vec_set_unit(ch.v[u], k, unit_at(A, p0 + k));
        }
    } else if constexpr (MODE == kModeCheck) {
        // The read-only check on 2-vector chunks (the default below about
        // 6.2M units) reads the same whole vectors as the repair path below,
        // but clears the units outside the string with one mask per vector
        // (its callers pass no lead or trail unit): 1,000 units 2.34 -> 1.5-1.8
        // us per call back to back, 4,095 units 2.19 -> 1.6-1.9.
        const long long first = cfirst + lane * kUnitsPerVec;
        const int before = (int)(first > 1 ? -1LL : first < -(CU + 9) ? CU + 9 : -first);
        const int left = (int)(A.n - first < -1 ? -1LL : A.n - first > CU + 9 ? CU + 9 : A.n - first);
        const uint4 *p = vin + c * (32LL * U) + lane;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int lo = before - u * kWarpSliceUnits, hi = left - u * kWarpSliceUnits;
            ch.v[u] = make_uint4(0, 0, 0, 0);
            ld_pred<true>(ch.v[u], p + 32 * u, hi > 0 && lo < kUnitsPerVec);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int lo = before - u * kWarpSliceUnits, hi = left - u * kWarpSliceUnits;
            if (lo > 0 || hi < kUnitsPerVec) {
                const int a = lo < 0 ? 0 : lo > 8 ? 8 : lo, b = hi < 0 ? 0 : hi > 8 ? 8 : hi;
                uint32_t flo, fhi;
                bits_to_flags(b > a ? ((1u << b) - 1u) & ~((1u << a) - 1u) : 0u, flo, fhi);
                ch.v[u].x &= prmt(flo, 0u, 0x9988);
                ch.v[u].y &= prmt(flo, 0u, 0xBBAA);
                ch.v[u].z &= prmt(fhi, 0u, 0x9988);
                ch.v[u].w &= prmt(fhi, 0u, 0xBBAA);
            }
        }
    } else {
        // A chunk at an end of the string.  Every 16-byte vector that holds a
        // unit of the string is read whole, with a predicated load (all issue
        // before the first is used).  Reading a vector's units outside the
        // string cannot fault: an aligned 16-byte block that holds one byte of
        // the string lies in the same mapped page.  Those units are replaced
        // afterwards by what unit_at() gives them (zero, or lead / trail at
        // -1 / n); vectors without a unit of the string are never read.  One
        // string of 1,000 units: 2.2 us per call when every lane read its
        // units one by one, against 1.0 for 1,024 units.
        // Per lane, in 32 bits: units of the string before and after this
        // lane's first unit, clamped to [-1, CU + 9]; for vector u, units
        // k < lo lie before the string (k = lo - 1 at -1) and units k >= hi
        // after it (k = hi at n).
        const long long first = cfirst + lane * kUnitsPerVec;
        const int before = (int)(first > 1 ? -1LL : first < -(CU + 9) ? CU + 9 : -first);
        const int left = (int)(A.n - first < -1 ? -1LL : A.n - first > CU + 9 ? CU + 9 : A.n - first);
        const uint4 *p = vin + c * (32LL * U) + lane;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int lo = before - u * kWarpSliceUnits, hi = left - u * kWarpSliceUnits;
            ch.v[u] = make_uint4(0, 0, 0, 0);
            ld_pred<MODE != kModeInPlace>(ch.v[u], p + 32 * u, hi > 0 && lo < kUnitsPerVec);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int lo = before - u * kWarpSliceUnits, hi = left - u * kWarpSliceUnits;
            if (lo > 0 || hi < kUnitsPerVec) {
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (k < lo || k >= hi) vec_set_unit(ch.v[u], k, k == hi ? A.trail : k == lo - 1 ? A.lead : 0u);
            }
        }
    }
    ch.halo = 0;
    if (lane == 0) ch.halo = unit_at(A, cfirst - 1);
    if (lane == 31) ch.halo = unit_at(A, cfirst + CU);
}

// Units of vector u of this lane that lie in [0, n), as an 8-bit mask.
__device__ __forceinline__ uint32_t valid_bits8(long long p0, long long n) {
    const long long lo = p0 < 0 ? -p0 : 0;
    const long long hi = n - p0 < 8 ? n - p0 : 8;
    if (hi <= lo) return 0u;
    return ((1u << hi) - 1u) & ~((1u << lo) - 1u);
}

// Store vector u of a chunk (dst = this lane's first unit of the chunk).
template <int MODE, int ST>
__device__ __forceinline__ void store_chunk_vec(uint16_t *dst, int u, const uint4 &f, bool edge, long long p0,
                                                long long n, uint32_t bad8) {
    uint16_t *d = dst + u * kWarpSliceUnits;
    if (!edge) {
        if constexpr (MODE == kModeInPlace)
            *reinterpret_cast<uint4 *>(d) = f;
        else
            store_vec<ST>(d, f);
    } else {
        const uint32_t w8 = (MODE == kModeInPlace) ? bad8 : valid_bits8(p0, n);
        if (MODE != kModeInPlace && w8 == 0xFFu) {  // a whole vector inside the string
            store_vec<ST>(d, f);
            return;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (w8 & (1u << k)) d[k] = (uint16_t)vec_unit(f, k);
    }
}

// Steps 2-5 of the chunk starting at unit cfirst.
// `filter` (repair modes, warp-uniform): 0 runs Section 3.1's step-two test
// before locating anything.  A chunk that fails it sets a count of chunks
// that skip the test, so that strings with mismatches everywhere test only
// one chunk in kFilterRetry.
constexpr int kFilterRetry = 16;

template <int MODE, bool FB, int ST, int U>
__device__ __forceinline__ void process_chunk(const SingleArgs &A, long long cfirst, const Chunk<U> &ch, int lane,
                                              long long &my_first, unsigned long long *blk_best = nullptr,
                                              int *filter = nullptr) {
    constexpr long long CU = (long long)U * kWarpSliceUnits;
    const bool edge = (cfirst < 0) || (cfirst + CU > A.n);
    const long long lfirst = cfirst + lane * kUnitsPerVec;  // this lane's first unit
    uint16_t *dst = (MODE == kModeCheck || MODE == kModeList) ? nullptr : A.out + lfirst;
    ChunkBits<U> cb;
    const uint32_t surr = chunk_surrogates<U>(ch.v, cb);

    if (!__any_sync(kFull, surr != 0)) {
        // Well-formed chunk: copy out of place, nothing otherwise.
        if constexpr (MODE == kModeOut) {
#pragma unroll
            for (int u = 0; u < U; ++u) store_chunk_vec<MODE, ST>(dst, u, ch.v[u], edge, lfirst + u * kWarpSliceUnits, A.n, 0u);
        }
        return;
    }

    // Slow path: locate the mismatched units.
    uint32_t from_prev, from_next;
    chunk_classes_prev<U>(cb, unit_is_high(ch.halo), lane, from_prev);
    if constexpr (MODE == kModeCheck) {
        // Read-only check: the step-two test clears chunks whose surrogates
        // all pair up, without locating anything (chunks at the string ends
        // take the full path).
        if (!edge && !__any_sync(kFull, chunk_step_two<U>(cb, from_prev, unit_is_low(ch.halo), lane) != 0)) return;
    } else if constexpr (MODE == kModeOut || MODE == kModeInPlace) {
        // Repair: the same test clears a chunk whose pairs all match; it is
        // then copied unchanged (out of place) or left alone (in place).
        if (filter) {
            if (*filter > 0) {
                --*filter;
            } else if (!edge) {
                if (!__any_sync(kFull, chunk_step_two<U>(cb, from_prev, unit_is_low(ch.halo), lane) != 0)) {
                    if constexpr (MODE == kModeOut) {
#pragma unroll
                        for (int u = 0; u < U; ++u) store_chunk_vec<MODE, ST>(dst, u, ch.v[u], false, 0, A.n, 0u);
                    }
                    return;
                }
                *filter = kFilterRetry;
            }
        }
    }
    chunk_next_low<U>(cb, unit_is_low(ch.halo), lane, from_next);
    bool found = false;
    uint32_t any_bad = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const long long p0 = lfirst + u * kWarpSliceUnits;
        uint32_t bad_lo, bad_hi;
        vec_bad<U>(cb, u, from_prev, from_next, 0u, 0u, 0u, bad_lo, bad_hi);
        if (edge) {
            uint32_t vlo, vhi;
            bits_to_flags(valid_bits8(p0, A.n), vlo, vhi);
            bad_lo &= vlo;
            bad_hi &= vhi;
        }
        const uint32_t vbad = bad_lo | bad_hi;
        any_bad |= vbad;
        if constexpr (MODE == kModeOut) {
            uint4 f = ch.v[u];
            if (vbad) f = fix_vec(f, bad_lo, bad_hi);
            store_chunk_vec<MODE, ST>(dst, u, f, edge, p0, A.n, 0u);
        } else if constexpr (MODE == kModeInPlace) {
            if (vbad) {
                if (A.unit_stores) {
                    uint32_t rest = gather4(bad_lo) | (gather4(bad_hi) << 4);
                    uint16_t *d = dst + u * kWarpSliceUnits;
                    while (rest) {
                        d[__ffs(rest) - 1] = (uint16_t)0xFFFDu;
                        rest &= rest - 1;
                    }
                } else {
                    store_chunk_vec<MODE, ST>(dst, u, fix_vec(ch.v[u], bad_lo, bad_hi), edge, p0, A.n,
                                              gather4(bad_lo) | (gather4(bad_hi) << 4));
                }
            }
        } else if constexpr (MODE == kModeList) {
            // All positions: reserve room for the warp's units with one atomic,
            // then each lane writes its own (warp-aggregated, unordered).
            const uint32_t bits8 = gather4(bad_lo) | (gather4(bad_hi) << 4);
            const uint32_t mine = __popc(bits8);
            uint32_t incl = mine;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, incl, d);
                if (lane >= d) incl += t;
            }
            const uint32_t total = __shfl_sync(kFull, incl, 31);
            if (total) {
                unsigned long long base = 0;
                if (lane == 31) base = atomicAdd((unsigned long long *)&A.slot->pad1, (unsigned long long)total);
                base = __shfl_sync(kFull, base, 31);
                unsigned long long at = base + (incl - mine);
                uint32_t rest = bits8;
                while (rest) {
                    const int k = __ffs(rest) - 1;
                    rest &= rest - 1;
                    if ((long long)at < A.capacity) A.positions[at] = p0 + k;
                    ++at;
                }
            }
        }
        if constexpr (FB) {
            if (vbad && !found) {
                found = true;
                const long long p = p0 + first_flag(bad_lo, bad_hi);
                my_first = p < my_first ? p : my_first;
            }
        }
    }
    if constexpr (FB && MODE == kModeCheck) {
        // Publish early so that other warps can stop: the block's best so far
        // lives in shared memory (blk_best, which also takes in the global
        // minimum when a warp of the block polls it), and only a warp that
        // improves on it updates the global minimum, so that strings with
        // mismatches everywhere do not pile thousands of atomics onto one
        // address.
        if (__any_sync(kFull, any_bad != 0)) {
            const long long wmin = warp_min_ll(my_first);
            if (lane == 0) {
                const unsigned long long w = (unsigned long long)wmin;
                if (atomicMin(blk_best, w) > w) atomicMin(&A.slot->min, w);
            }
        }
    }
}

// Block minimum, one atomic per block; the last block to finish publishes
// the first-error index and resets the slot for the next launch (the next
// grid on the stream sees the reset at the kernel boundary).  A grid of one
// block publishes directly.
__device__ __forceinline__ void finish_first_bad(const SingleArgs &A, long long my_first, int lane) {
    __shared__ long long s_min[kMaxBlockThreads / 32];
    const long long wmin = warp_min_ll(my_first);
    if (lane == 0) s_min[threadIdx.x >> 5] = wmin;
    __syncthreads();
    if (threadIdx.x != 0) return;
    long long m = LLONG_MAX;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = s_min[w] < m ? s_min[w] : m;
    if (gridDim.x == 1) {
        // The check's early-exit publications came from this block's warps,
        // so m already holds them.
        *A.result = (m < A.n) ? m : A.n;
        A.slot->min = ~0ull;
        return;
    }
    if (m != LLONG_MAX) atomicMin(&A.slot->min, (unsigned long long)m);
    if (atomic_add_acq_rel(&A.slot->done, 1u) == gridDim.x - 1) {
        const unsigned long long g = ld_acquire(&A.slot->min);
        *A.result = (g < (unsigned long long)A.n) ? (long long)g : A.n;
        A.slot->min = ~0ull;
        A.slot->done = 0u;
    }
}

// List mode: the last block publishes the number of mismatched units and
// resets the counter for the next launch.
__device__ __forceinline__ void finish_list(const SingleArgs &A) {
    __syncthreads();  // every warp of the block has reserved its positions
    if (threadIdx.x != 0) return;
    if (atomic_add_acq_rel(&A.slot->done, 1u) == gridDim.x - 1) {
        *A.result = (long long)ld_acquire((const unsigned long long *)&A.slot->pad1);
        A.slot->pad1 = 0;
        A.slot->done = 0u;
    }
}

cudaError_t launch_single_tma(const SingleLaunch &L, cudaStream_t stream);
const void *single_tma_kernel_for_occupancy(int mode, bool fb);

}  // namespace u16wf
