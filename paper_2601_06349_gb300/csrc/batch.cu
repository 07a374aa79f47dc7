// Ragged-batch toWellFormed / isWellFormed: many strings of uneven length in
// one launch.  String s is in[offsets[s] .. offsets[s+1]); every string end is
// a hard boundary (Section 3.1: a string that starts with a low or ends with a
// high surrogate has that unit replaced, whatever lies next to it in memory).
//
// The flattened unit range [offsets[0], offsets[count]) is read from the
// device and cut into warp chunks of U slices of 32 vectors of 8 units
// (U = 4 or 8: 1024 or 2048 units).  The grid is persistent and each warp
// owns a contiguous run of chunks, so consecutive chunks of a warp need
// consecutive entries of `offsets`.  One kernel (batch_words_kernel) serves
// every form: out of place, in place, the per-string first-error index (the
// check), and in place with the per-string index (the serving engine); the
// per-chunk steps are described above words_chunk() below.
#include <cuda_runtime.h>
#include <limits.h>
#include <stdlib.h>

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

// ---------------------------------------------------------------------------
// Per chunk, on bit words.
//
// After classification each lane packs, per vector, the surrogate bits and
// the low-surrogate bits of its 8 units (bit k = unit k) into one 16-bit
// entry of a per-warp table.  Read back four entries at a time, the table
// gives lane l the units [1024 j + 32 l, +32) of the chunk as 32-bit words,
// one per 1024 units of chunk (j = 0 for U = 4, j = 0, 1 for U = 8): H (high
// surrogates) and L (low surrogates).  A chunk without any surrogate is done
// at once (out of place it is copied).  The string starts inside the chunk
// become a third word S (one shared atomic OR per start, from a window of the
// offsets).  The Section 1 rule with every string end as a boundary (Section
// 3.1) is then word logic in each lane:
//   Hprev  = H one unit up (bit 31 of the lane before; lane 0: the unit
//            before the chunk),  Lnext = L one unit down;
//   a unit that starts a string has no left neighbour, the unit before it no
//   right neighbour:  NoRight = S one unit down;
//   bad    = H & ~(Lnext & ~NoRight) | L & ~(Hprev & ~S).
// Then, by form:
//   - out of place: each lane takes its vectors' 8 bits from the lane word
//     that holds them (one shuffle per vector), replaces in registers and
//     stores each vector once;
//   - in place: one 2-byte store of U+FFFD per bad unit, or for a dense chunk
//     the bad words back through shared memory to one byte per vector and a
//     16-byte block per vector that holds one (no ordering between warps is
//     needed: a replacement never changes a neighbour's verdict);
//   - per-string first-error index: each lane of the offsets window takes one
//     string that meets the chunk and finds its first bad unit from
//     max(start, chunk start) in constant time: the word holding that unit
//     (one shuffle), else the first later word with a bad unit (a ballot
//     summary and one more shuffle).  Results go to first_bad with an atomic
//     minimum, over the string lengths a small kernel writes first.
// The 2048-unit chunk halves the per-unit cost of the offsets window and the
// lookups (1M strings, check: 50 -> 43 us).

// Per-warp table, start words and dense-store bytes of the word kernels.
template <int U>
struct __align__(16) WordScratch {
    uint16_t cls[U * 32];      // vector v of the chunk: bit k = unit k is a surrogate, bit 8+k = it is a low one
    uint32_t starts[U * 8];    // word w: bit j set when a string starts at unit 32 w + j of the chunk
    uint32_t bad[U * 8];       // repair of a dense chunk: the bad words again (byte v = vector v's 8 bits)
};

// Vector u of this lane of the chunk at vector vfirst, read again for the
// dense store path (unit loads at the batch's ends, 0 outside [lo, hi)).
__device__ __forceinline__ uint4 reload_batch_vec(const BatchArgs &A, const uint4 *vin, long long vfirst, int u,
                                                  long long lo, long long hi, int lane, bool edge) {
    if (!edge) return ld_plain(vin + vfirst + 32 * u + lane);
    const long long p0 = (vfirst + 32 * u + lane) * 8 - A.a;
    uint4 v = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (p0 + k >= lo && p0 + k < hi) vec_set_unit(v, k, A.in[p0 + k]);
    return v;
}

// Above this many replaced units in one lane word (any lane of the warp) a
// repair chunk stores whole 16-byte blocks instead of single units.
constexpr int kSparseMax = 4;

// The strings base .. base+31 of the batch, one per lane: its start and end
// (kFar for lanes past the last string).  kFar stays far from overflow when
// a chunk position is subtracted from it.
constexpr long long kFar = LLONG_MAX / 4;
struct Window {
    long long base = 0;
    long long start = kFar;
    long long end = kFar;
};

__device__ __forceinline__ void load_window(const BatchArgs &A, long long base, int lane, Window &w) {
    const long long s = base + lane;
    w.base = base;
    w.start = s < A.count ? A.offsets[s] : kFar;
    w.end = s < A.count ? A.offsets[s + 1] : kFar;
}

// Position x relative to a chunk [cfirst, cfirst + CU), saturated: -1 before
// the chunk, CU at its end (the unit after it), CU + 1 beyond.
template <int CU>
__device__ __forceinline__ int rel_pos(long long x, long long cfirst) {
    const long long d = x - cfirst;
    return d < 0 ? -1 : d > CU ? CU + 1 : (int)d;
}

// Per-warp state carried from chunk to chunk: a string index at or before the
// first string of the next chunk, and (when `have_nw`) the window prefetched
// for the next chunk, which starts with the string holding its first unit.
struct CheckState {
    long long hint = 0;
    Window nw;
    bool have_nw = false;
    bool waited = false;
};

template <int MODE, int ST, int U>
__device__ __forceinline__ void words_chunk(const BatchArgs &A, const uint4 *vin, long long vfirst, long long lo,
                                            long long hi, const BatchChunk<U> &ch, int lane, WordScratch<U> &ws,
                                            CheckState &st) {
    constexpr int NW = U / 4;            // 32-unit words per lane
    constexpr int CU = U * kWarpSliceUnits;
    constexpr bool kOut = MODE == kModeOut;
    constexpr bool kRepair = MODE != kModeCheck;
    constexpr bool kLookup = MODE == kModeCheck || MODE == kModeInPlaceFirst;
    static_assert(NW == 1 || NW == 2, "chunk width");
    const long long cfirst = vfirst * 8 - A.a;
    const bool edge = (cfirst < lo) || (cfirst + CU > hi);
    const long long lfirst = cfirst + lane * kUnitsPerVec;

    // Classification (high byte only, Section 3.3), packed to the table one
    // vector at a time so that its registers free at once, and the fast
    // test.  The barrier after the previous chunk's last reads of the scratch
    // orders these writes.
    uint32_t acc = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t hb0 = prmt(ch.v[u].x, ch.v[u].y, 0x7531);
        const uint32_t hb1 = prmt(ch.v[u].z, ch.v[u].w, 0x7531);
        const uint32_t sf0 = surrogate_flags(hb0);
        const uint32_t sf1 = surrogate_flags(hb1);
        acc |= sf0 | sf1;
        const uint32_t s8 = pack_flags8(sf0, sf1);
        const uint32_t l8 = pack_flags8(sf0 & (hb0 << 5), sf1 & (hb1 << 5));
        ws.cls[32 * u + lane] = (uint16_t)prmt(s8, l8, 0x0073);
    }
    if (!__any_sync(kFull, acc != 0)) {  // no surrogate: nothing in the chunk is mismatched
        if constexpr (kOut) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                batch_store_vec<kModeOut, ST>(A.out + lfirst + u * kWarpSliceUnits, ch.v[u], edge,
                                              lfirst + u * kWarpSliceUnits, lo, hi, 0u);
        }
        if (st.have_nw) st.hint = st.nw.base;  // the window was for this chunk
        st.have_nw = false;
        return;
    }
#pragma unroll
    for (int j = 0; j < NW; ++j) ws.starts[32 * j + lane] = 0u;

    // The chunk's first window: the one prefetched for it, else a search for
    // the string holding the chunk's first unit.
    Window w;
    if (st.have_nw) {
        w = st.nw;
    } else {
        const long long s0 = lower_bound_warp(A.offsets, A.count, st.hint, cfirst + 1, lane) - 1;
        load_window(A, s0 > 0 ? s0 : 0, lane, w);
    }
    st.hint = w.base;
    st.have_nw = false;
    const int relS = rel_pos<CU>(w.start, cfirst);
    const int relE = rel_pos<CU>(w.end, cfirst);
    __syncwarp();

    // Lane word j covers units [1024 j + 32 lane, +32) of the chunk: table
    // entries 128 j + 4 lane .. +3.
    uint32_t H[NW], L[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const uint2 t = *reinterpret_cast<const uint2 *>(&ws.cls[128 * j + 4 * lane]);
        const uint32_t s32 = prmt(t.x, t.y, 0x6420);
        L[j] = prmt(t.x, t.y, 0x7531);
        H[j] = s32 & ~L[j];
    }

    // String starts in [cfirst, cend) into the start words; a start at cend
    // (the unit after the chunk) is kept aside.  A chunk whose window's last
    // string starts inside it walks further windows.  On the way, the first
    // string that ends beyond cend holds the next chunk's first unit: its
    // window is requested now, so that its latency hides behind this chunk.
    uint32_t at_end = 0;
    int nwin = 1;
    long long nb = -1;
    {
        Window m = w;
        int mS = relS, mE = relE;
        for (;;) {
            if ((unsigned)mS < (unsigned)CU) atomicOr(&ws.starts[mS >> 5], 1u << (mS & 31));
            at_end |= __ballot_sync(kFull, mS == CU);
            const unsigned beyond = __ballot_sync(kFull, mE > CU);
            if (nb < 0 && beyond) nb = m.base + (__ffs(beyond) - 1);
            if (!(__ballot_sync(kFull, mS < CU) >> 31)) break;
            load_window(A, m.base + 32, lane, m);
            mS = rel_pos<CU>(m.start, cfirst);
            mE = rel_pos<CU>(m.end, cfirst);
            ++nwin;
        }
    }
    if (nb >= 0) {
        load_window(A, nb, lane, st.nw);
        st.have_nw = true;
    }
    __syncwarp();

    // Section 1 rule with the string ends, per lane word.  The word before
    // word j of lane 0 is word j-1 of lane 31 (or the unit before the chunk),
    // the word after word j of lane 31 is word j+1 of lane 0 (or the unit
    // after the chunk): a source lane sends the word its destination needs.
    uint32_t S[NW], bad[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) S[j] = ws.starts[32 * j + lane];
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const uint32_t h_up = __shfl_sync(kFull, (j > 0 && lane == 31) ? H[j > 0 ? j - 1 : 0] : H[j], (lane + 31) & 31);
        const uint32_t l_dn =
            __shfl_sync(kFull, (j < NW - 1 && lane == 0) ? L[j < NW - 1 ? j + 1 : j] : L[j], (lane + 1) & 31);
        const uint32_t s_dn =
            __shfl_sync(kFull, (j < NW - 1 && lane == 0) ? S[j < NW - 1 ? j + 1 : j] : S[j], (lane + 1) & 31);
        const uint32_t h_in =
            (j == 0 && lane == 0) ? (unit_is_high(ch.halo) ? 1u : 0u) : (h_up >> 31);
        const uint32_t l_in = (j == NW - 1 && lane == 31) ? (unit_is_low(ch.halo) ? 1u : 0u) : l_dn & 1u;
        const uint32_t s_in = (j == NW - 1 && lane == 31) ? (at_end ? 1u : 0u) : s_dn & 1u;
        const uint32_t hprev = (H[j] << 1) | h_in;
        const uint32_t lnext = (L[j] >> 1) | (l_in << 31);
        const uint32_t noright = (S[j] >> 1) | (s_in << 31);
        bad[j] = (H[j] & ~(lnext & ~noright)) | (L[j] & ~(hprev & ~S[j]));
    }
    // Summary: bit w set when word w (lane w & 31, word w >> 5) has a bad unit.
    unsigned long long nz = __ballot_sync(kFull, bad[0] != 0);
    if constexpr (NW == 2) nz |= (unsigned long long)__ballot_sync(kFull, bad[1] != 0) << 32;
    if constexpr (kOut) {
        // Out of place: each vector's 8 bits from the lane word that holds
        // them (vector 32u + lane is byte lane & 3 of word 8u + lane / 4),
        // replaced in registers, stored once.
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t wsrc = __shfl_sync(kFull, bad[u >> 2], 8 * (u & 3) + (lane >> 2));
            const uint32_t bits8 = (wsrc >> (8 * (lane & 3))) & 0xFFu;
            uint4 f = ch.v[u];
            if (bits8) {
                uint32_t flo, fhi;
                bits_to_flags(bits8, flo, fhi);
                f = fix_vec(f, flo, fhi);
            }
            batch_store_vec<kModeOut, ST>(A.out + lfirst + u * kWarpSliceUnits, f, edge, lfirst + u * kWarpSliceUnits,
                                          lo, hi, 0u);
        }
        return;
    }
    if (nz == 0) return;

    if constexpr (kRepair) {
        // Replacements: one 2-byte store per bad unit, or for a dense chunk
        // the bad bits back to one byte per vector (the byte order of the
        // words makes byte v of ws.bad vector v's 8 bits) and a 16-byte block
        // per vector holding one.  Units outside [lo, hi) are never bad.
        int pop = 0;
#pragma unroll
        for (int j = 0; j < NW; ++j) pop += __popc(bad[j]);
        if (__reduce_max_sync(kFull, (unsigned)pop) <= (unsigned)kSparseMax) {
            if constexpr (kOut) __syncwarp();  // this chunk's copies (other lanes' too) before the replacements
#pragma unroll
            for (int j = 0; j < NW; ++j) {
                uint16_t *base = A.out + cfirst + 1024 * j + 32 * lane;
                uint32_t rest = bad[j];
                while (rest) {
                    base[__ffs(rest) - 1] = (uint16_t)0xFFFDu;
                    rest &= rest - 1;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < NW; ++j) ws.bad[32 * j + lane] = bad[j];
            __syncwarp();
            const uint8_t *bytes = reinterpret_cast<const uint8_t *>(ws.bad);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t bits8 = bytes[32 * u + lane];
                if (bits8) {
                    uint32_t flo, fhi;
                    bits_to_flags(bits8, flo, fhi);
                    const uint4 v = reload_batch_vec(A, vin, vfirst, u, lo, hi, lane, edge);
                    batch_store_vec<MODE, ST>(A.out + lfirst + u * kWarpSliceUnits, fix_vec(v, flo, fhi), edge,
                                              lfirst + u * kWarpSliceUnits, lo, hi, bits8);
                }
            }
        }
    }
    if constexpr (kLookup) {
        // first_bad holds the lengths once the grid before this one is done.
        if (!st.waited) {
            wait_prior_grids();
            st.waited = true;
        }
        // Each lane's string: its first bad unit from max(start, cfirst) within
        // the chunk, if that lies before the string's end.
        Window m = w;
        int mS = relS, mE = relE;
        for (int k = 0;;) {
            const unsigned r = mS > 0 ? (unsigned)mS : 0u;
            const unsigned wi = (r >> 5) & (32 * NW - 1);  // lanes that take nothing read any word
            uint32_t b1 = __shfl_sync(kFull, bad[0], wi & 31u);
            if constexpr (NW == 2) {
                const uint32_t x = __shfl_sync(kFull, bad[1], wi & 31u);
                b1 = (wi >> 5) ? x : b1;
            }
            b1 &= 0xFFFFFFFFu << (r & 31);
            const unsigned long long later = wi < 32 * NW - 1 ? nz & (~0ull << (wi + 1)) : 0ull;
            const unsigned w2 = later ? (unsigned)(__ffsll((long long)later) - 1) : 0u;
            uint32_t b2 = __shfl_sync(kFull, bad[0], w2 & 31u);
            if constexpr (NW == 2) {
                const uint32_t x = __shfl_sync(kFull, bad[1], w2 & 31u);
                b2 = (w2 >> 5) ? x : b2;
            }
            const int q = b1 ? (int)(wi << 5) + __ffs(b1) - 1 : later ? (int)(w2 << 5) + __ffs(b2) - 1 : CU + 2;
            // (The index is never negative: the unsigned minimum is the same, and
            // a native reduction.)
            if (mS < CU && q < mE)
                atomicMin(reinterpret_cast<unsigned long long *>(&A.first_bad[m.base + lane]),
                          (unsigned long long)((long long)q - (m.start - cfirst)));
            if (++k >= nwin) break;
            load_window(A, m.base + 32, lane, m);
            mS = rel_pos<CU>(m.start, cfirst);
            mE = rel_pos<CU>(m.end, cfirst);
        }
    }
}

// At least 4 resident blocks per SM: without the bound the 2048-unit check
// takes 79 registers and 3 blocks; with it 63 and no spills.
template <int MODE, int ST, int U, bool PF>
__global__ void __launch_bounds__(kBlockThreads, 4) batch_words_kernel(const BatchArgs A) {
    constexpr bool kLookup = MODE == kModeCheck || MODE == kModeInPlaceFirst;
    __shared__ WordScratch<U> s_scratch[kBlockThreads / 32];
    const int lane = threadIdx.x & 31;
    WordScratch<U> &ws = s_scratch[threadIdx.x >> 5];
    // With per-string results the grid before this one is the lengths
    // kernel, which writes only first_bad and lets this grid start once it
    // has waited for its own predecessors, so `in` and `offsets` are final:
    // the wait comes before the first atomic on first_bad (and before the
    // exit).  The repairs wait here.
    if constexpr (!kLookup) wait_prior_grids();
    const long long lo = A.offsets[0];
    const long long hi = A.offsets[A.count];
    if (lo >= 0 && hi > lo) {
        const long long vbeg = (lo + A.a) >> 3;
        const long long vend = (hi + A.a + 7) >> 3;
        const long long chunks = (vend - vbeg + 32LL * U - 1) / (32LL * U);
        const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
        const long long c_begin = gwarp * chunks / nwarps;
        const long long c_end = (gwarp + 1) * chunks / nwarps;
        const uint4 *vin = reinterpret_cast<const uint4 *>(A.in - A.a);
        CheckState st;
        if constexpr (PF) {
            BatchChunk<U> nv;
            if (c_begin < c_end) load_batch_chunk<MODE, U>(A, vin, vbeg + c_begin * (32LL * U), lo, hi, lane, nv);
            for (long long c = c_begin; c < c_end; ++c) {
                const BatchChunk<U> v = nv;
                if (c + 1 < c_end) load_batch_chunk<MODE, U>(A, vin, vbeg + (c + 1) * (32LL * U), lo, hi, lane, nv);
                words_chunk<MODE, ST, U>(A, vin, vbeg + c * (32LL * U), lo, hi, v, lane, ws, st);
            }
        } else {
            for (long long c = c_begin; c < c_end; ++c) {
                const long long vfirst = vbeg + c * (32LL * U);
                BatchChunk<U> v;
                load_batch_chunk<MODE, U>(A, vin, vfirst, lo, hi, lane, v);
                words_chunk<MODE, ST, U>(A, vin, vfirst, lo, hi, v, lane, ws, st);
            }
        }
    }
    allow_next_grid();
    if constexpr (kLookup) wait_prior_grids();
}

// first_bad[s] = length of string s (the value for a well-formed string).
// The next grid (the check) may start as soon as this one has waited for
// its own predecessors: it reads only what those wrote before its first
// atomic on first_bad, where it waits for this grid.
__global__ void batch_lengths_kernel(const long long *offsets, long long count, long long *first_bad) {
    wait_prior_grids();
    allow_next_grid();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        first_bad[i] = offsets[i + 1] - offsets[i];
}

template <int MODE, int ST>
static const void *words_ptr(int u, bool pf) {
    if (pf)
        return u == 2 ? (const void *)batch_words_kernel<MODE, ST, 4, true>
                      : (const void *)batch_words_kernel<MODE, ST, 8, true>;
    return u == 2 ? (const void *)batch_words_kernel<MODE, ST, 4, false>
                  : (const void *)batch_words_kernel<MODE, ST, 8, false>;
}

// Chunk width of each mode when the configuration leaves it open (0):
// 1024 units out of place (1M strings: 69.5 against 72.8 us), 2048 for the
// rest (in place 66 against 69 us, check 43 against 50 us).
static int batch_u(int mode, int u) { return u == 2 || u == 4 ? u : mode == kModeOut ? 2 : 4; }

static const void *pick_batch(int mode, int st, int u, bool pf) {
    if (mode == kModeCheck) return words_ptr<kModeCheck, 16>(u, pf);
    if (mode == kModeInPlaceFirst) return words_ptr<kModeInPlaceFirst, 16>(u, pf);
    if (mode == kModeInPlace) return words_ptr<kModeInPlace, 16>(u, pf);
    switch (st) {
        case 16: return words_ptr<kModeOut, 16>(u, pf);
        case 8: return words_ptr<kModeOut, 8>(u, pf);
        case 4: return words_ptr<kModeOut, 4>(u, pf);
        default: return words_ptr<kModeOut, 2>(u, pf);
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
    const int u = batch_u(L.mode, L.units_per_thread);
    const void *fn = pick_batch(L.mode, st, u, L.prefetch);
    void *args[] = {(void *)&A};
    const long long warps = (long long)L.blocks * (kBlockThreads / 32);
    const long long chunk_units = u == 2 ? 1024 : 2048;
    // The per-string forms overlap the lengths kernel before them (they wait
    // only before their first atomic), which needs the attribute.
    const bool pdl = L.mode == kModeCheck || L.mode == kModeInPlaceFirst || L.full_occupancy ||
                     (L.units_hint > 0 && pdl_fits((L.units_hint / chunk_units + warps) / warps, false));
    return launch_kernel(fn, dim3((unsigned)L.blocks), dim3(kBlockThreads), args, 0, stream, pdl);
}

const void *batch_kernel_for_occupancy(int mode, int u, bool prefetch) {
    return pick_batch(mode, 16, batch_u(mode, u), prefetch);
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
