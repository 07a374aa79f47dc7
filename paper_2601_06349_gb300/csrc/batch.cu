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
//     start inside the chunk in a per-warp byte map in shared memory, and
//     applies the pairing rule with "no left neighbour" at a start and "no
//     right neighbour" just before one;
//   - per-string first-error index: the chunk's mismatch bits go to shared
//     memory (one byte per vector, plus a one-bit-per-byte summary from a
//     ballot), then each lane takes one string of the offsets window and
//     finds the first set bit from its start.
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

// This lane's U vectors of a chunk, and (lanes 0 and 31) the units just
// before and after the chunk (0 outside [lo, hi)).
template <int U>
struct BatchChunk {
    uint4 v[U];
    uint32_t halo;
};

template <int MODE, int U>
__device__ __forceinline__ void load_batch_chunk(const BatchArgs &A, const uint4 *vin, long long vfirst, long long lo,
                                                 long long hi, int lane, BatchChunk<U> &ch) {
    constexpr long long CU = (long long)U * kWarpSliceUnits;
    const long long cfirst = vfirst * 8 - A.a;
    if (cfirst >= lo && cfirst + CU <= hi) {
        const uint4 *p = vin + vfirst + lane;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if constexpr (MODE == kModeInPlace || MODE == kModeInPlaceFirst)
                ch.v[u] = ld_plain(p + 32 * u);
            else
                ch.v[u] = ld_stream(p + 32 * u);
        }
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long p0 = cfirst + u * kWarpSliceUnits + lane * kUnitsPerVec;
            ch.v[u] = make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const long long p = p0 + k;
                if (p >= lo && p < hi) vec_set_unit(ch.v[u], k, A.in[p]);
            }
        }
    }
    ch.halo = 0;
    const long long hp = (lane == 0) ? cfirst - 1 : cfirst + CU;
    if ((lane == 0 || lane == 31) && hp >= lo && hp < hi) ch.halo = A.in[hp];
}

__device__ __forceinline__ uint32_t batch_valid_bits8(long long p0, long long lo, long long hi) {
    const long long a = lo - p0 > 0 ? lo - p0 : 0;
    const long long b = hi - p0 < 8 ? hi - p0 : 8;
    if (b <= a) return 0u;
    return ((1u << b) - 1u) & ~((1u << a) - 1u);
}

template <int MODE, int ST>
__device__ __forceinline__ void batch_store_vec(uint16_t *d, const uint4 &f, bool edge, long long p0, long long lo,
                                                long long hi, uint32_t bad8) {
    if (!edge) {
        if constexpr (MODE == kModeInPlace || MODE == kModeInPlaceFirst)
            *reinterpret_cast<uint4 *>(d) = f;
        else
            store_vec<ST>(d, f);
    } else {
        const uint32_t w8 = (MODE == kModeInPlace || MODE == kModeInPlaceFirst) ? bad8 : batch_valid_bits8(p0, lo, hi);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (w8 & (1u << k)) d[k] = (uint16_t)vec_unit(f, k);
    }
}

// Per-warp shared scratch of the slow path.
template <int U>
struct __align__(16) WarpScratch {
    uint8_t starts[U * kWarpSliceUnits + 16];  // 0x80 at r when a string starts at unit cfirst + r (r <= CU)
    uint8_t bad[U * 32];                        // per-string first-error modes: mismatch bits of vector 32u + lane
};

// Per-string first-error modes: the chunk's mismatched units as one bit per
// unit (ws.bad, byte 32u + lane = vector u of that lane, bit k = unit k)
// plus a summary with one bit per byte (bit lane of nz[u]).  Returns the
// first unit index >= r (0 <= r < CU) of the chunk with its bit set, or CU.
template <int U>
__device__ __forceinline__ int first_mismatch_from(const WarpScratch<U> &ws, const uint32_t (&nz)[U], int r) {
    const int b0 = r >> 3;
    const uint32_t m0 = ws.bad[b0] & (0xFFu << (r & 7));
    if (m0) return (b0 << 3) + __ffs(m0) - 1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int from = b0 + 1 - 32 * u;  // first byte of word u after byte b0
        uint32_t m = from >= 32 ? 0u : from > 0 ? nz[u] & (0xFFFFFFFFu << from) : nz[u];
        if (m) {
            const int b = 32 * u + __ffs(m) - 1;
            return (b << 3) + __ffs(ws.bad[b]) - 1;
        }
    }
    return U * kWarpSliceUnits;
}

// A window of 32 consecutive entries of `offsets` (one per lane), loaded
// while the previous chunk of the warp was processed (base < 0: none).
struct OffsetsWindow {
    long long base = -1;
    long long off = LLONG_MAX;
};

template <int MODE, int ST, int U>
__device__ __forceinline__ void process_batch_chunk(const BatchArgs &A, long long cfirst, long long lo, long long hi,
                                                    const BatchChunk<U> &ch, int lane, WarpScratch<U> &ws,
                                                    long long &hint, OffsetsWindow &next_win) {
    constexpr long long CU = (long long)U * kWarpSliceUnits;
    const bool edge = (cfirst < lo) || (cfirst + CU > hi);
    const long long lfirst = cfirst + lane * kUnitsPerVec;
    uint16_t *dst = (MODE == kModeCheck) ? nullptr : A.out + lfirst;
    ChunkBits<U> cb;
    const uint32_t surr = chunk_surrogates<U>(ch.v, cb);

    if (!__any_sync(kFull, surr != 0)) {
        if constexpr (MODE == kModeOut) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                batch_store_vec<MODE, ST>(dst + u * kWarpSliceUnits, ch.v[u], edge, lfirst + u * kWarpSliceUnits, lo,
                                          hi, 0u);
        }
        return;
    }

    // String starts in [cfirst, cfirst + CU] as a byte map (0x80 per start).
    // The barrier orders the previous chunk's reads of the scratch before
    // these writes.
    constexpr int kStartVecs = (int)(CU + 16) / 16;
    __syncwarp();
    for (int i = lane; i < kStartVecs; i += 32) reinterpret_cast<uint4 *>(ws.starts)[i] = make_uint4(0, 0, 0, 0);
    const long long cend = cfirst + CU;
    // One window of 32 offsets usually covers both the search and the
    // collection: the one the previous chunk requested for this one (from the
    // string just before this chunk's first start), else one from the
    // previous chunk's first string.  Any window whose first entry starts at
    // or before this chunk's first string will do.
    // (The check only: in the repair kernels the window's registers cost a
    // resident block per SM, 70 -> 85 us on 1M strings; the check gains,
    // 78 -> 76 us.)
    constexpr bool kWindowAhead = MODE == kModeCheck;
    long long base, off;
    if (kWindowAhead && next_win.base >= 0) {
        base = next_win.base;
        off = next_win.off;
    } else {
        base = hint;
        off = base + lane <= A.count ? A.offsets[base + lane] : LLONG_MAX;
    }
    long long idx = base + lane;
    unsigned ge = __ballot_sync(kFull, off >= cfirst);
    if (ge == 0) {  // the chunk's strings start beyond this window: search
        base = lower_bound_warp(A.offsets, A.count, base + 32, cfirst, lane);
        idx = base + lane;
        off = idx <= A.count ? A.offsets[idx] : LLONG_MAX;
        ge = __ballot_sync(kFull, off >= cfirst);
    }
    const int fs_lane = __ffs(ge) - 1;
    const long long s_first = base + fs_lane;  // first string starting at or after cfirst
    const long long base_first = base;
    const long long off_first = off;           // offsets[base_first + lane]
    hint = s_first;
    // Request the next chunk's window now, so that its latency hides behind
    // this chunk's work: from the string before the first one starting at or
    // after this chunk's end (known when this window reaches that far).
    if constexpr (kWindowAhead) {
        const unsigned ge_end = __ballot_sync(kFull, off >= cfirst + CU);
        if (ge_end) {
            const long long s_next = base + __ffs(ge_end) - 1;
            next_win.base = s_next > 0 ? s_next - 1 : 0;
            next_win.off = next_win.base + lane <= A.count ? A.offsets[next_win.base + lane] : LLONG_MAX;
        } else {
            next_win.base = -1;
        }
    }
    bool simple = true;  // all starts of the chunk lie in the first window
    __syncwarp();
    for (;;) {
        const bool inside = off >= cfirst && off <= cend;
        if (inside) ws.starts[off - cfirst] = 0x80;
        const unsigned m = __ballot_sync(kFull, inside);
        // continue while the window's last entry still starts inside the chunk
        if (!(m >> 31)) break;
        simple = false;
        base += 32;
        idx = base + lane;
        off = idx <= A.count ? A.offsets[idx] : LLONG_MAX;
    }
    __syncwarp();
    uint32_t from_prev, from_next;
    chunk_classes<U>(cb, unit_is_high(ch.halo), unit_is_low(ch.halo), lane, from_prev, from_next);
    uint32_t nz[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int r0 = u * kWarpSliceUnits + lane * kUnitsPerVec;
        const long long p0 = cfirst + r0;
        const uint2 st = *reinterpret_cast<const uint2 *>(ws.starts + r0);  // starts at units r0 .. r0+7
        const uint32_t st_next = ws.starts[r0 + 8] >> 7;                   // a start at unit r0+8
        uint32_t bad_lo, bad_hi;
        vec_bad<U>(cb, u, from_prev, from_next, st.x, st.y, st_next, bad_lo, bad_hi);
        if (edge) {
            uint32_t vlo, vhi;
            bits_to_flags(batch_valid_bits8(p0, lo, hi), vlo, vhi);
            bad_lo &= vlo;
            bad_hi &= vhi;
        }
        const uint32_t vbad = bad_lo | bad_hi;
        if constexpr (MODE == kModeOut) {
            uint4 f = ch.v[u];
            if (vbad) f = fix_vec(f, bad_lo, bad_hi);
            batch_store_vec<MODE, ST>(dst + u * kWarpSliceUnits, f, edge, p0, lo, hi, 0u);
        } else if constexpr (MODE == kModeInPlace || MODE == kModeInPlaceFirst) {
            if (vbad)
                batch_store_vec<MODE, ST>(dst + u * kWarpSliceUnits, fix_vec(ch.v[u], bad_lo, bad_hi), edge, p0, lo,
                                          hi, gather4(bad_lo) | (gather4(bad_hi) << 4));
        }
        if constexpr (MODE == kModeCheck || MODE == kModeInPlaceFirst) {
            const uint32_t bits8 = gather4(bad_lo) | (gather4(bad_hi) << 4);
            ws.bad[u * 32 + lane] = (uint8_t)bits8;
            nz[u] = __ballot_sync(kFull, bits8 != 0);
        }
    }
    if constexpr (MODE == kModeCheck || MODE == kModeInPlaceFirst) {
        uint32_t any = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) any |= nz[u];
        if (any == 0) return;
        __syncwarp();
        // Per-string first-error index, one lane per string: the string of
        // window entry `lane` starts at `off` and ends at the next entry; its
        // first mismatched unit in this chunk is the first set bit from its
        // start.  Strings that start in this chunk take the window entries in
        // [cfirst, cend); the string holding the chunk's first units (it
        // started earlier) takes the units before the first of them.
        const int q0 = first_mismatch_from<U>(ws, nz, 0);
        const long long first_start = __shfl_sync(kFull, off_first, fs_lane);  // offsets[s_first]
        const long long before = __shfl_sync(kFull, off_first, fs_lane >= 1 ? fs_lane - 1 : 0);
        if (lane == 0 && s_first >= 1 && s_first <= A.count && q0 < (int)CU && cfirst + q0 < first_start) {
            const long long start = fs_lane >= 1 ? before : A.offsets[s_first - 1];
            atomicMin(&A.first_bad[s_first - 1], cfirst + q0 - start);
        }
        long long wbase = base_first;
        long long woff = off_first;
        for (;;) {
            const long long wnext = __shfl_down_sync(kFull, woff, 1);
            const long long widx = wbase + lane;
            const bool starts_here = woff >= cfirst && woff < cend && widx < A.count;
            if (starts_here) {
                const long long end = lane < 31 ? wnext : A.offsets[widx + 1];
                const int q = first_mismatch_from<U>(ws, nz, (int)(woff - cfirst));
                if (cfirst + q < end && q < (int)CU) atomicMin(&A.first_bad[widx], cfirst + q - woff);
            }
            if (simple || !__shfl_sync(kFull, starts_here ? 1 : 0, 31)) break;
            wbase += 32;
            const long long ni = wbase + lane;
            woff = ni <= A.count ? A.offsets[ni] : LLONG_MAX;
        }
    }
}

template <int MODE, int ST, int U, bool PF>
__global__ void __launch_bounds__(kBlockThreads) batch_kernel(const BatchArgs A) {
    __shared__ WarpScratch<U> s_scratch[kBlockThreads / 32];

    const int lane = threadIdx.x & 31;
    WarpScratch<U> &ws = s_scratch[threadIdx.x >> 5];
    wait_prior_grids();

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
    OffsetsWindow next_win;
    if constexpr (PF) {
        BatchChunk<U> nv;
        if (c_begin < c_end) load_batch_chunk<MODE, U>(A, vin, vbeg + c_begin * (32LL * U), lo, hi, lane, nv);
        for (long long c = c_begin; c < c_end; ++c) {
            const BatchChunk<U> v = nv;
            if (c + 1 < c_end) load_batch_chunk<MODE, U>(A, vin, vbeg + (c + 1) * (32LL * U), lo, hi, lane, nv);
            const long long cfirst = (vbeg + c * (32LL * U)) * 8 - A.a;
            process_batch_chunk<MODE, ST, U>(A, cfirst, lo, hi, v, lane, ws, hint, next_win);
        }
    } else {
        for (long long c = c_begin; c < c_end; ++c) {
            const long long vfirst = vbeg + c * (32LL * U);
            BatchChunk<U> v;
            load_batch_chunk<MODE, U>(A, vin, vfirst, lo, hi, lane, v);
            process_batch_chunk<MODE, ST, U>(A, vfirst * 8 - A.a, lo, hi, v, lane, ws, hint, next_win);
        }
    }
    allow_next_grid();
}

// first_bad[s] = length of string s (the value for a well-formed string).
__global__ void batch_lengths_kernel(const long long *offsets, long long count, long long *first_bad) {
    wait_prior_grids();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        first_bad[i] = offsets[i + 1] - offsets[i];
}

template <int MODE, int ST>
static const void *batch_ptr(int u, bool pf) {
    if (pf) return u == 2 ? (const void *)batch_kernel<MODE, ST, 2, true> : (const void *)batch_kernel<MODE, ST, 4, true>;
    return u == 2 ? (const void *)batch_kernel<MODE, ST, 2, false> : (const void *)batch_kernel<MODE, ST, 4, false>;
}

static const void *pick_batch(int mode, int st, int u, bool pf) {
    if (mode == kModeCheck) return batch_ptr<kModeCheck, 16>(u, pf);
    if (mode == kModeInPlaceFirst) return batch_ptr<kModeInPlaceFirst, 16>(u, pf);
    if (mode == kModeInPlace) return batch_ptr<kModeInPlace, 16>(u, pf);
    switch (st) {
        case 16: return batch_ptr<kModeOut, 16>(u, pf);
        case 8: return batch_ptr<kModeOut, 8>(u, pf);
        case 4: return batch_ptr<kModeOut, 4>(u, pf);
        default: return batch_ptr<kModeOut, 2>(u, pf);
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
    if (L.mode == kModeCheck || L.mode == kModeInPlaceFirst) {
        long long blocks = (L.count + kBlockThreads - 1) / kBlockThreads;
        if (blocks > L.blocks) blocks = L.blocks;
        if (blocks < 1) blocks = 1;
        const long long *offsets = L.offsets;
        long long count = L.count;
        long long *first_bad = L.first_bad;
        void *largs[] = {(void *)&offsets, (void *)&count, (void *)&first_bad};
        cudaError_t e = launch_kernel((const void *)batch_lengths_kernel, dim3((unsigned)blocks), dim3(kBlockThreads),
                                      largs, 0, stream);
        if (e != cudaSuccess) return e;
    }
    const void *fn = pick_batch(L.mode, st, L.units_per_thread == 2 ? 2 : 4, L.prefetch);
    void *args[] = {(void *)&A};
    const long long warps = (long long)L.blocks * (kBlockThreads / 32);
    const long long chunk_units = (L.units_per_thread == 2 ? 2 : 4) * (long long)kWarpSliceUnits;
    const bool pdl = L.full_occupancy ||
                     (L.units_hint > 0 && pdl_fits((L.units_hint / chunk_units + warps) / warps, false));
    return launch_kernel(fn, dim3((unsigned)L.blocks), dim3(kBlockThreads), args, 0, stream, pdl);
}

const void *batch_kernel_for_occupancy(int mode, int u, bool prefetch) {
    return pick_batch(mode, 16, u == 2 ? 2 : 4, prefetch);
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
