// Device helpers shared by the single-string and ragged-batch kernels.
//
// A thread owns runs of 8 code units held in one 16-byte vector (uint4).  A
// warp covers 32 consecutive vectors (512 bytes) per "slice"; a warp "chunk"
// is U consecutive slices (U <= 4).
//
// Classification follows Section 3.1 of the paper (mask with 0xFC00, compare
// with 0xD800 / 0xDC00), applied to the high byte only as in the paper's NEON
// variant (Section 3.3: the more significant byte decides high / low /
// neither).  The 8 high bytes of a vector are gathered into two 32-bit words
// (units 0..3 and 4..7) and every per-unit property is kept as a "byte-lane
// flag": bit 8k+7 of the word is set when unit k has the property.  Then
//   surrogate  : high byte & 0xF8 == 0xD8   (exact zero-byte test)
//   low        : surrogate and bit 2 of the high byte set (0xDC..0xDF)
//   high       : surrogate and bit 2 clear   (0xD8..0xDB)
// and the neighbours of Section 3.1's step three are 8-bit funnel shifts of
// these words: flag of unit k-1 at bit 8k+7, flag of unit k+1 at bit 8k+7.
#pragma once

#include <stdint.h>

namespace u16wf {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kUnitsPerVec = 8;
constexpr int kWarpSliceUnits = 32 * kUnitsPerVec;  // 256 units = 512 bytes
constexpr uint32_t kFlagBits = 0x80808080u;

// Scratch slot used by first-error reductions (one per stream).  `min` holds
// the smallest bad index seen so far (all ones = none), `done` counts
// finished blocks; the last block publishes the result and resets both.
struct Slot {
    unsigned long long min;
    unsigned int done;
    unsigned int pad0;
    long long result;
    long long pad1;
};
static_assert(sizeof(Slot) == 32, "slot size");

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
    return r;
}

// High bytes of the 8 units of v: units 0..3 in `lo`, 4..7 in `hi`.
__device__ __forceinline__ void high_bytes(const uint4 &v, uint32_t &lo, uint32_t &hi) {
    lo = prmt(v.x, v.y, 0x7531);
    hi = prmt(v.z, v.w, 0x7531);
}

// Bit 8k+7 set iff byte k of x is zero.  Exact per byte: the low seven bits
// plus 0x7F never carry out of the byte.
__device__ __forceinline__ uint32_t zero_byte_flags(uint32_t x) {
    return ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & kFlagBits;
}

__device__ __forceinline__ uint32_t surrogate_flags(uint32_t hb) {
    return zero_byte_flags((hb & 0xF8F8F8F8u) ^ 0xD8D8D8D8u);
}

// Bit 2 of every high byte moved to bit 7: set for 0xDC..0xDF among surrogates.
__device__ __forceinline__ uint32_t low_half_flags(uint32_t hb) { return (hb << 5) & kFlagBits; }

// Bit u (u < 4) moved to bit 8u.
__device__ __forceinline__ uint32_t spread4(uint32_t x) { return (x * 0x00204081u) & 0x01010101u; }

// Bits 8k+7 (k < 4) gathered to bits 0..3.
__device__ __forceinline__ uint32_t gather4(uint32_t flags) { return (((flags >> 7) * 0x00204081u) >> 21) & 0xFu; }

// The byte-lane flags of a vector's 8 units (lo: units 0..3, hi: units 4..7,
// flag of unit k at bit 8k+7) as byte 3 of the result, bit 24+k = unit k.
// In (lo >> 4 | hi) units 0..3 sit at bits 3, 11, 19, 27 and units 4..7 at
// 7, 15, 23, 31; the multiplier 2^0 + 2^7 + 2^14 + 2^21 adds four shifted
// copies, which put unit k on bit 24+k.  Every partial product lands on a
// different bit, so the sum has no carries and the other bits of byte 3 stay
// clear.
__device__ __forceinline__ uint32_t pack_flags8(uint32_t lo, uint32_t hi) { return ((lo >> 4) | hi) * 0x00204081u; }

// Replace by U+FFFD every unit whose byte-lane flag is set (lo: units 0..3,
// hi: units 4..7).  prmt with a selector nibble 8+k replicates the sign bit
// of byte k, so each unit gets an all-ones or all-zeros 16-bit mask.
__device__ __forceinline__ uint4 fix_vec(uint4 v, uint32_t bad_lo, uint32_t bad_hi) {
    uint32_t m;
    m = prmt(bad_lo, 0u, 0x9988);
    v.x = (v.x & ~m) | (0xFFFDFFFDu & m);
    m = prmt(bad_lo, 0u, 0xBBAA);
    v.y = (v.y & ~m) | (0xFFFDFFFDu & m);
    m = prmt(bad_hi, 0u, 0x9988);
    v.z = (v.z & ~m) | (0xFFFDFFFDu & m);
    m = prmt(bad_hi, 0u, 0xBBAA);
    v.w = (v.w & ~m) | (0xFFFDFFFDu & m);
    return v;
}

// Index (0..7) of the first flagged unit; requires bad_lo | bad_hi != 0.
__device__ __forceinline__ int first_flag(uint32_t bad_lo, uint32_t bad_hi) {
    return bad_lo ? ((__ffs(bad_lo) - 1) >> 3) : 4 + ((__ffs(bad_hi) - 1) >> 3);
}

__device__ __forceinline__ uint32_t vec_unit(const uint4 &v, int k) {
    const uint32_t w = (k < 2) ? v.x : (k < 4) ? v.y : (k < 6) ? v.z : v.w;
    return (k & 1) ? (w >> 16) : (w & 0xFFFFu);
}

__device__ __forceinline__ void vec_set_unit(uint4 &v, int k, uint32_t u) {
    uint32_t *w = (k < 2) ? &v.x : (k < 4) ? &v.y : (k < 6) ? &v.z : &v.w;
    *w = (k & 1) ? ((*w & 0x0000FFFFu) | (u << 16)) : ((*w & 0xFFFF0000u) | u);
}

__device__ __forceinline__ bool unit_is_high(uint32_t u) { return (u & 0xFC00u) == 0xD800u; }
__device__ __forceinline__ bool unit_is_low(uint32_t u) { return (u & 0xFC00u) == 0xDC00u; }

// Byte-lane flags of 8 per-unit bits (bit k = unit k).
__device__ __forceinline__ void bits_to_flags(uint32_t bits8, uint32_t &lo, uint32_t &hi) {
    lo = spread4(bits8 & 0xFu) << 7;
    hi = spread4((bits8 >> 4) & 0xFu) << 7;
}

// Per-lane flags of a warp chunk of U vectors (two words per vector: units
// 0..3 and 4..7).  chunk_surrogates() fills `a` with the gathered high bytes
// and `b` with the surrogate flags; chunk_classes() turns them, in place,
// into high-surrogate flags (`a`) and low-surrogate flags (`b`).
template <int U>
struct ChunkBits {
    uint32_t a[2 * U];
    uint32_t b[2 * U];
};

// Returns nonzero iff some unit of the chunk's U vectors is a surrogate.
template <int U>
__device__ __forceinline__ uint32_t chunk_surrogates(const uint4 (&v)[U], ChunkBits<U> &cb) {
    uint32_t acc = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        cb.a[2 * u] = prmt(v[u].x, v[u].y, 0x7531);
        cb.a[2 * u + 1] = prmt(v[u].z, v[u].w, 0x7531);
        cb.b[2 * u] = surrogate_flags(cb.a[2 * u]);
        cb.b[2 * u + 1] = surrogate_flags(cb.a[2 * u + 1]);
        acc |= cb.b[2 * u] | cb.b[2 * u + 1];
    }
    return acc;
}

// High / low flags in place, and the cross-lane neighbour flags: bit 8u+7 of
// `from_prev` is set when the unit just before this lane's vector u is a high
// surrogate, bit 8u+7 of `from_next` when the unit just after it is a low
// surrogate.  That unit is the last (first) unit of the adjacent lane's
// vector, or for lane 0 (31) the last unit of lane 31's vector in the previous
// slice (lane 0's in the next slice), or the halo unit just outside the chunk:
//   halo_prev   lane 0: the unit before the chunk is a high surrogate
//   halo_next   lane 31: the unit after the chunk is a low surrogate
// chunk_classes_prev() does the first half (classes and from_prev),
// chunk_next_low() the second.
template <int U>
__device__ __forceinline__ void chunk_classes_prev(ChunkBits<U> &cb, uint32_t halo_prev, int lane,
                                                   uint32_t &from_prev) {
#pragma unroll
    for (int i = 0; i < 2 * U; ++i) {
        const uint32_t lowhalf = low_half_flags(cb.a[i]);
        const uint32_t sur = cb.b[i];
        cb.a[i] = sur & ~lowhalf;
        cb.b[i] = sur & lowhalf;
    }
    // Byte u of last_h: byte 3 of h_hi[u] (flag of unit 7 of vector u at its bit 7).
    uint32_t last_h;
    if constexpr (U == 4) {
        last_h = prmt(prmt(cb.a[1], cb.a[3], 0x0073), prmt(cb.a[5], cb.a[7], 0x0073), 0x5410);
    } else if constexpr (U == 2) {
        last_h = prmt(cb.a[1], cb.a[3], 0x0073) & 0xFFFFu;  // bytes 2, 3 are copies, not flags
    } else {
        last_h = cb.a[2 * U - 1] >> 24;
    }
    from_prev = __shfl_sync(kFull, last_h, (lane + 31) & 31);
    // lane 0: vector u's left neighbour is lane 31's vector u-1, or the halo
    if (lane == 0) from_prev = (from_prev << 8) | ((halo_prev & 1u) << 7);
}

template <int U>
__device__ __forceinline__ void chunk_next_low(const ChunkBits<U> &cb, uint32_t halo_next, int lane,
                                               uint32_t &from_next) {
    // Byte u of first_l: byte 0 of l_lo[u] (flag of unit 0 of vector u).
    uint32_t first_l;
    if constexpr (U == 4) {
        first_l = prmt(prmt(cb.b[0], cb.b[2], 0x0040), prmt(cb.b[4], cb.b[6], 0x0040), 0x5410);
    } else if constexpr (U == 2) {
        first_l = prmt(cb.b[0], cb.b[2], 0x0040) & 0xFFFFu;
    } else {
        first_l = cb.b[0] & 0xFFu;
    }
    from_next = __shfl_sync(kFull, first_l, (lane + 1) & 31);
    // lane 31: vector u's right neighbour is lane 0's vector u+1, or the halo
    if (lane == 31) from_next = (from_next >> 8) | ((halo_next & 1u) << (8 * U - 1));
}

template <int U>
__device__ __forceinline__ void chunk_classes(ChunkBits<U> &cb, uint32_t halo_prev, uint32_t halo_next, int lane,
                                              uint32_t &from_prev, uint32_t &from_next) {
    chunk_classes_prev<U>(cb, halo_prev, lane, from_prev);
    chunk_next_low<U>(cb, halo_next, lane, from_next);
}

// Section 3.1 step two for a whole chunk: in a well-formed run every unit's
// "left neighbour is high" equals its own "is low".  Returns nonzero in some
// lane iff that fails at a unit of the chunk or at the unit just after it
// (the halo, whose left neighbour is the chunk's last unit), i.e. iff the
// chunk holds a mismatched unit or its first unit is low without a high
// before it (the mismatch then belongs to the previous chunk).
template <int U>
__device__ __forceinline__ uint32_t chunk_step_two(const ChunkBits<U> &cb, uint32_t from_prev, uint32_t halo_next,
                                                   int lane) {
    uint32_t x = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t h_lo = cb.a[2 * u], h_hi = cb.a[2 * u + 1];
        const uint32_t pin = (from_prev << (24 - 8 * u)) & 0x80000000u;
        x |= (__funnelshift_l(pin, h_lo, 8) ^ cb.b[2 * u]) | (__funnelshift_l(h_lo, h_hi, 8) ^ cb.b[2 * u + 1]);
    }
    if (lane == 31) x |= (cb.a[2 * U - 1] >> 31) ^ (halo_next & 1u);
    return x;
}

// Mismatch flags of vector u of the chunk (Section 1 rule, Section 3.1 step
// three): a high surrogate whose right neighbour is not low, or a low one
// whose left neighbour is not high.
//   st_lo/hi  byte-lane flags of units that start a string (no left
//             neighbour); st_next: bit 0 set when the unit after the vector
//             starts one.  Zero for a single string.
template <int U>
__device__ __forceinline__ void vec_bad(const ChunkBits<U> &cb, int u, uint32_t from_prev, uint32_t from_next,
                                        uint32_t st_lo, uint32_t st_hi, uint32_t st_next, uint32_t &bad_lo,
                                        uint32_t &bad_hi) {
    const uint32_t h_lo = cb.a[2 * u], h_hi = cb.a[2 * u + 1];
    const uint32_t l_lo = cb.b[2 * u], l_hi = cb.b[2 * u + 1];
    // from_prev / from_next hold one flag per vector at bit 8u+7
    const uint32_t pin = (from_prev << (24 - 8 * u)) & 0x80000000u;  // left neighbour of unit 0, at bit 31
    const uint32_t nin = (from_next >> (8 * u)) & 0x80u;              // right neighbour of unit 7, at bit 7
    // flag of unit k-1 / unit k+1 at bit 8k+7
    const uint32_t ph_lo = __funnelshift_l(pin, h_lo, 8) & ~st_lo;
    const uint32_t ph_hi = __funnelshift_l(h_lo, h_hi, 8) & ~st_hi;
    const uint32_t nl_lo = __funnelshift_r(l_lo, l_hi, 8) & ~__funnelshift_r(st_lo, st_hi, 8);
    const uint32_t nl_hi = __funnelshift_r(l_hi, nin, 8) & ~__funnelshift_r(st_hi, st_next << 7, 8);
    bad_lo = (h_lo & ~nl_lo) | (l_lo & ~ph_lo);
    bad_hi = (h_hi & ~nl_hi) | (l_hi & ~ph_hi);
}

// Warp-wide minimum of a 64-bit value.
__device__ __forceinline__ long long warp_min_ll(long long v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const long long o = __shfl_xor_sync(kFull, v, off);
        v = o < v ? o : v;
    }
    return v;
}

// Completion counters of the last-block pattern.  The add has acquire and
// release semantics at GPU scope: it orders this thread's earlier writes (its
// block's atomicMin) before the count, and the block that brings the count to
// the grid size sees every other block's earlier writes, with no separate
// fence on either side.
__device__ __forceinline__ unsigned atomic_add_acq_rel(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// 16-byte loads / stores.
// Programmatic dependent launch.  wait_prior_grids(): wait for the grids this
// one depends on (a no-op when it was launched without the attribute); called
// first in every kernel, before any global memory access.
// allow_next_grid(): this block's main work is done, the next launch on the
// stream may start placing its blocks (which wait in turn).  Called after the
// main loop, not at the start: blocks of the next launch that become resident
// early sit in the SM slots a reduced persistent grid leaves free, and slowed
// the read-only check (0.81 -> 0.56 of the peak at 3 blocks per SM).
__device__ __forceinline__ void wait_prior_grids() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_next_grid() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint4 ld_stream(const uint4 *p) { return __ldcs(p); }
__device__ __forceinline__ uint4 ld_plain(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_stream(uint4 *p, const uint4 &v) { __stcs(p, v); }

// 128-bit load under a predicate instead of a branch: v keeps its value where
// `take` is false (no memory is touched then).  Loads of several vectors thus
// all issue before the first is used, where a branch around each would make
// the merge after it wait for that load.  STREAM: evict-first.
template <bool STREAM>
__device__ __forceinline__ void ld_pred(uint4 &v, const uint4 *p, bool take) {
    if constexpr (STREAM)
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t@q ld.global.cs.v4.u32 {%0,%1,%2,%3}, [%4];\n\t}"
            : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w)
            : "l"(p), "r"((unsigned)take));
    else
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t@q ld.global.v4.u32 {%0,%1,%2,%3}, [%4];\n\t}"
            : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w)
            : "l"(p), "r"((unsigned)take));
}

// Store the 8 units of v at dst, whose alignment is implied by ST (16, 8 or
// 4 bytes, or 2 = an odd unit index relative to 4 bytes).
template <int ST>
__device__ __forceinline__ void store_vec(uint16_t *dst, const uint4 &v) {
    if constexpr (ST == 16) {
        st_stream(reinterpret_cast<uint4 *>(dst), v);
    } else if constexpr (ST == 8) {
        uint2 *d = reinterpret_cast<uint2 *>(dst);
        __stcs(d, make_uint2(v.x, v.y));
        __stcs(d + 1, make_uint2(v.z, v.w));
    } else if constexpr (ST == 4) {
        uint32_t *d = reinterpret_cast<uint32_t *>(dst);
        __stcs(d, v.x);
        __stcs(d + 1, v.y);
        __stcs(d + 2, v.z);
        __stcs(d + 3, v.w);
    } else {
        static_assert(ST == 2, "store width");
        dst[0] = (uint16_t)(v.x & 0xFFFFu);
        uint32_t *d = reinterpret_cast<uint32_t *>(dst + 1);
        __stcs(d, __byte_perm(v.x, v.y, 0x5432));
        __stcs(d + 1, __byte_perm(v.y, v.z, 0x5432));
        __stcs(d + 2, __byte_perm(v.z, v.w, 0x5432));
        dst[7] = (uint16_t)(v.w >> 16);
    }
}

}  // namespace u16wf
