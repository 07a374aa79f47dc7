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
#pragma once

#include <cuda_runtime.h>
#include <limits.h>

#include "device.cuh"
#include "internal.h"
#include "lanevec.cuh"

namespace u16wf {

struct BatchArgs {
    const uint16_t *in;
    uint16_t *out;
    const long long *offsets;
    long long count;
    long long *first_bad;
    int a;  // misalignment of `in` in units, modulo the vector width
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


// Chunk geometry: NW 32-unit words per lane, a chunk of CU = 1024 NW units,
// read with loads of VB bytes (E = VB / 2 units): NL = 64 NW / VB loads per
// lane; load k of lane l covers units [32 E k + E l, +E) of the chunk and is
// entry 32 k + l of the per-warp table.
template <int NW, int VB>
struct Geo {
    static constexpr int E = VB / 2;
    static constexpr int NL = 64 * NW / VB;
    static constexpr int CU = 1024 * NW;
};

// This lane's loads of a chunk, and (lanes 0 and 31) the units just before
// and after the chunk (0 outside [lo, hi)).
template <int NW, int VB>
struct BatchChunk {
    LaneVec<VB> v[Geo<NW, VB>::NL];
    uint32_t halo;
};

// Unit loads of load k of a chunk that touches an end of the batch.
template <int VB>
__device__ __forceinline__ LaneVec<VB> load_units(const BatchArgs &A, long long p0, long long lo, long long hi) {
    LaneVec<VB> v;
#pragma unroll
    for (int i = 0; i < VB / 4; ++i) v.w[i] = 0;
#pragma unroll
    for (int k = 0; k < VB / 2; ++k)
        if (p0 + k >= lo && p0 + k < hi) lv_set_unit(v, k, A.in[p0 + k]);
    return v;
}

// The chunk whose first vector is vector vfirst of `vin` (the VB-aligned
// address at or below in[0]; vector v holds units [E v - a, E v - a + E)).
template <int MODE, int NW, int VB>
__device__ __forceinline__ void load_batch_chunk(const BatchArgs &A, const char *vin, long long vfirst, long long lo,
                                                 long long hi, int lane, BatchChunk<NW, VB> &ch) {
    using G = Geo<NW, VB>;
    constexpr bool kPlain = MODE == kModeInPlace || MODE == kModeInPlaceFirst;  // stores follow: keep in L2
    const long long cfirst = vfirst * G::E - A.a;
    if (cfirst >= lo && cfirst + G::CU <= hi) {
        const char *p = vin + (vfirst + lane) * VB;
#pragma unroll
        for (int k = 0; k < G::NL; ++k) ch.v[k] = lv_load<VB, !kPlain>(p + 32 * k * VB);
    } else {
#pragma unroll
        for (int k = 0; k < G::NL; ++k) ch.v[k] = load_units<VB>(A, cfirst + 32 * G::E * k + lane * G::E, lo, hi);
    }
    ch.halo = 0;
    const long long hp = (lane == 0) ? cfirst - 1 : cfirst + G::CU;
    if ((lane == 0 || lane == 31) && hp >= lo && hp < hi) ch.halo = A.in[hp];
}

// Units [p0, p0 + E) that lie in [lo, hi), as an E-bit mask.
template <int E>
__device__ __forceinline__ uint32_t batch_valid_bits(long long p0, long long lo, long long hi) {
    const long long a = lo - p0 > 0 ? lo - p0 : 0;
    const long long b = hi - p0 < E ? hi - p0 : E;
    if (b <= a) return 0u;
    return (uint32_t)(((1ull << b) - 1ull) & ~((1ull << a) - 1ull));
}

// Store load v at d (units p0 ..): whole out of place, or at the batch's
// ends only the units inside it (out of place) or only the replaced ones
// (`bad`, in place).
template <int MODE, int ST, int VB>
__device__ __forceinline__ void batch_store(uint16_t *d, const LaneVec<VB> &v, bool edge, long long p0, long long lo,
                                            long long hi, uint32_t bad) {
    constexpr bool kInPlace = MODE == kModeInPlace || MODE == kModeInPlaceFirst;
    if (!edge) {
        lv_store<VB, kInPlace ? VB : ST>(d, v);
    } else {
        const uint32_t w = kInPlace ? bad : batch_valid_bits<VB / 2>(p0, lo, hi);
#pragma unroll
        for (int k = 0; k < VB / 2; ++k)
            if (w & (1u << k)) d[k] = (uint16_t)lv_unit(v, k);
    }
}

// Per-warp table, start words and dense-store words of the word kernels.
template <int NW>
struct __align__(16) WordScratch {
    uint32_t cls[64 * NW];     // the table: 8 bytes per lane word (entry 32 k + lane of each load)
    uint32_t starts[32 * NW];  // word w: bit j set when a string starts at unit 32 w + j of the chunk
    uint32_t bad[32 * NW];     // repair of a dense chunk: the bad words again
};

// Bits of load k of this lane in a set of lane words (bad words in
// registers via a shuffle, or in shared memory): word E k + E lane / 32,
// from bit E lane mod 32.  The word is in the same half (j) for every lane.
template <int VB>
__device__ __forceinline__ uint32_t load_bits_mask() {
    return VB == 32 ? 0xFFFFu : VB == 16 ? 0xFFu : 0xFu;
}

// Above this many replaced units in one lane word (any lane of the warp) a
// repair chunk stores whole vectors instead of single units.
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

template <int MODE, int ST, int NW, int VB>
__device__ __forceinline__ void words_chunk(const BatchArgs &A, const char *vin, long long vfirst, long long lo,
                                            long long hi, const BatchChunk<NW, VB> &ch, int lane,
                                            WordScratch<NW> &ws, CheckState &st) {
    using G = Geo<NW, VB>;
    constexpr int CU = G::CU;
    constexpr int E = G::E;
    constexpr bool kOut = MODE == kModeOut;
    constexpr bool kRepair = MODE != kModeCheck;
    constexpr bool kLookup = MODE == kModeCheck || MODE == kModeInPlaceFirst;
    static_assert(NW == 1 || NW == 2, "chunk width");
    const long long cfirst = vfirst * E - A.a;
    const bool edge = (cfirst < lo) || (cfirst + CU > hi);
    const long long lfirst = cfirst + lane * E;  // this lane's first unit of load 0

    // Classification (high byte only, Section 3.3), one table entry per load
    // (its registers free at once), and the fast test.  The barrier after the
    // previous chunk's last reads of the scratch orders these writes.
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < G::NL; ++k) lv_store_entry<VB>(ws.cls, 32 * k + lane, lv_classify<VB>(ch.v[k], acc));
    if (!__any_sync(kFull, acc != 0)) {  // no surrogate: nothing in the chunk is mismatched
        if constexpr (kOut) {
#pragma unroll
            for (int k = 0; k < G::NL; ++k)
                batch_store<kModeOut, ST, VB>(A.out + lfirst + 32 * E * k, ch.v[k], edge, lfirst + 32 * E * k, lo,
                                              hi, 0u);
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

    // Lane word j covers units [1024 j + 32 lane, +32) of the chunk: 8 bytes
    // of the table.
    uint32_t H[NW], L[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const uint2 t = reinterpret_cast<const uint2 *>(ws.cls)[32 * j + lane];
        uint32_t s32;
        lv_word_bits<VB>(t.x, t.y, s32, L[j]);
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
        // Out of place: each load's E bits from the lane word that holds them
        // (load k of lane l is bits E l mod 32 .. of word E k + E l / 32, in
        // the same half j for every lane), replaced in registers, stored once.
#pragma unroll
        for (int k = 0; k < G::NL; ++k) {
            const int j = (E * k) >> 5;
            const uint32_t src = (uint32_t)((E * k) & 31) + (((uint32_t)lane * E) >> 5);
            const uint32_t bits = (__shfl_sync(kFull, bad[j], src) >> ((lane * E) & 31)) & load_bits_mask<VB>();
            LaneVec<VB> f = ch.v[k];
            if (bits) lv_fix<VB>(f, bits);
            batch_store<kModeOut, ST, VB>(A.out + lfirst + 32 * E * k, f, edge, lfirst + 32 * E * k, lo, hi, 0u);
        }
        return;
    }
    if (nz == 0) return;

    if constexpr (kRepair) {
        // In place: one 2-byte store per bad unit, or for a dense chunk the
        // bad words back through shared memory and a whole vector per load
        // holding one.  Units outside [lo, hi) are never bad.
        int pop = 0;
#pragma unroll
        for (int j = 0; j < NW; ++j) pop += __popc(bad[j]);
        if (__reduce_max_sync(kFull, (unsigned)pop) <= (unsigned)kSparseMax) {
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
#pragma unroll
            for (int k = 0; k < G::NL; ++k) {
                const int word = E * k + ((lane * E) >> 5);
                const uint32_t bits = (ws.bad[word] >> ((lane * E) & 31)) & load_bits_mask<VB>();
                if (bits) {
                    const long long p0 = lfirst + 32 * E * k;
                    LaneVec<VB> v = edge ? load_units<VB>(A, p0, lo, hi)
                                         : lv_load<VB, false>(vin + (vfirst + 32 * k + lane) * VB);
                    lv_fix<VB>(v, bits);
                    batch_store<MODE, ST, VB>(A.out + p0, v, edge, p0, lo, hi, bits);
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

// Every form's kernel.  Blocks of up to kMaxBlockThreads threads (the block
// size is chosen at launch); at least 2 such blocks per SM, i.e. at most 64
// registers, which the 2048-unit check needs to keep 4 blocks of 256 threads
// (79 registers and 3 blocks without the bound).
template <int MODE, int ST, int NW, int VB, bool PF>
__global__ void __launch_bounds__(kMaxBlockThreads, 2) batch_words_kernel(const BatchArgs A) {
    using G = Geo<NW, VB>;
    constexpr bool kLookup = MODE == kModeCheck || MODE == kModeInPlaceFirst;
    __shared__ WordScratch<NW> s_scratch[kMaxBlockThreads / 32];
    const int lane = threadIdx.x & 31;
    WordScratch<NW> &ws = s_scratch[threadIdx.x >> 5];
    // With per-string results the grid before this one is the lengths
    // kernel, which writes only first_bad and lets this grid start once it
    // has waited for its own predecessors, so `in` and `offsets` are final:
    // the wait comes before the first atomic on first_bad (and before the
    // exit).  The repairs wait here.
    if constexpr (!kLookup) wait_prior_grids();
    const long long lo = A.offsets[0];
    const long long hi = A.offsets[A.count];
    if (lo >= 0 && hi > lo) {
        const long long vbeg = (lo + A.a) / G::E;
        const long long vend = (hi + A.a + G::E - 1) / G::E;
        const long long chunks = (vend - vbeg + 32LL * G::NL - 1) / (32LL * G::NL);
        const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
        const long long c_begin = gwarp * chunks / nwarps;
        const long long c_end = (gwarp + 1) * chunks / nwarps;
        const char *vin = reinterpret_cast<const char *>(A.in - A.a);
        CheckState st;
        if constexpr (PF) {
            BatchChunk<NW, VB> nv;
            if (c_begin < c_end) load_batch_chunk<MODE, NW, VB>(A, vin, vbeg + c_begin * (32LL * G::NL), lo, hi, lane, nv);
            for (long long c = c_begin; c < c_end; ++c) {
                const BatchChunk<NW, VB> v = nv;
                if (c + 1 < c_end)
                    load_batch_chunk<MODE, NW, VB>(A, vin, vbeg + (c + 1) * (32LL * G::NL), lo, hi, lane, nv);
                words_chunk<MODE, ST, NW, VB>(A, vin, vbeg + c * (32LL * G::NL), lo, hi, v, lane, ws, st);
            }
        } else {
            for (long long c = c_begin; c < c_end; ++c) {
                const long long vfirst = vbeg + c * (32LL * G::NL);
                BatchChunk<NW, VB> v;
                load_batch_chunk<MODE, NW, VB>(A, vin, vfirst, lo, hi, lane, v);
                words_chunk<MODE, ST, NW, VB>(A, vin, vfirst, lo, hi, v, lane, ws, st);
            }
        }
    }
    allow_next_grid();
    if constexpr (kLookup) wait_prior_grids();
}

// Pointer to the kernel of a form and launch shape (nullptr if not built):
// nw 32-unit words per lane, vb-byte loads, pf next chunk in flight (built
// for nw = 1, vb = 16 only), st the store class of `out` (out of place).
template <int MODE, int ST>
const void *words_kernel_ptr(int nw, int vb, bool pf) {
    if (pf && nw == 1 && vb == 16) return (const void *)batch_words_kernel<MODE, ST, 1, 16, true>;
    if (vb == 8) {
        if constexpr (ST <= 8)
            return nw == 1 ? (const void *)batch_words_kernel<MODE, ST, 1, 8, false>
                           : (const void *)batch_words_kernel<MODE, ST, 2, 8, false>;
        return nullptr;
    }
    if (vb == 32)
        return nw == 1 ? (const void *)batch_words_kernel<MODE, ST, 1, 32, false>
                       : (const void *)batch_words_kernel<MODE, ST, 2, 32, false>;
    if constexpr (ST <= 16)
        return nw == 1 ? (const void *)batch_words_kernel<MODE, ST, 1, 16, false>
                       : (const void *)batch_words_kernel<MODE, ST, 2, 16, false>;
    return nullptr;
}

const void *batch_out_kernel(int st, int nw, int vb, bool pf);  // batch_out.cu

}  // namespace u16wf
