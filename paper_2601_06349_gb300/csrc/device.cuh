// Device helpers shared by the single-string and ragged-batch kernels.
//
// A thread owns runs of 8 code units held in one 16-byte vector (uint4).  A
// warp covers 32 consecutive vectors (512 bytes) per "slice"; a warp "chunk"
// is U consecutive slices.  Per thread, the units of its U vectors are
// described by 32-bit masks with bit 8*u + k for unit k of slice u (U <= 4).
//
// Classification follows Section 3.1 of the paper (mask with 0xFC00, compare
// with 0xD800 / 0xDC00), applied to the high byte only as in the paper's NEON
// variant (Section 3.3: the more significant byte decides high / low /
// neither): byte & 0xFC == 0xD8 is high, == 0xDC is low, byte & 0xF8 == 0xD8
// is any surrogate.
#pragma once

#include <stdint.h>

namespace u16wf {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kUnitsPerVec = 8;
constexpr int kWarpSliceUnits = 32 * kUnitsPerVec;  // 256 units = 512 bytes
constexpr uint16_t kReplacement = 0xFFFD;

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

// High bytes of the 8 units of v: units 0..3 in b03, 4..7 in b47.
__device__ __forceinline__ void high_bytes(const uint4 &v, uint32_t &b03, uint32_t &b47) {
    b03 = __byte_perm(v.x, v.y, 0x7531);
    b47 = __byte_perm(v.z, v.w, 0x7531);
}

// Nonzero iff some unit of v is a surrogate.  (x - 0x01..) & ~x & 0x80..
// is nonzero exactly when x has a zero byte.
__device__ __forceinline__ uint32_t any_surrogate(const uint4 &v) {
    uint32_t b03, b47;
    high_bytes(v, b03, b47);
    const uint32_t x0 = (b03 & 0xF8F8F8F8u) ^ 0xD8D8D8D8u;
    const uint32_t x1 = (b47 & 0xF8F8F8F8u) ^ 0xD8D8D8D8u;
    return ((x0 - 0x01010101u) & ~x0 & 0x80808080u) | ((x1 - 0x01010101u) & ~x1 & 0x80808080u);
}

// 4-bit mask, bit k set iff byte k of x is zero (exact per byte: no borrow
// crosses bytes because the low seven bits plus 0x7F stay below 0x100).
__device__ __forceinline__ uint32_t zero_bytes4(uint32_t x) {
    const uint32_t nonzero = ((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x;
    const uint32_t z = (~nonzero & 0x80808080u) >> 7;  // bits 0, 8, 16, 24
    return ((z * 0x00204081u) >> 21) & 0xFu;          // gathers them to bits 0..3
}

// 8-bit masks (bit k = unit k) of high and low surrogates in v.
__device__ __forceinline__ void classify8(const uint4 &v, uint32_t &h, uint32_t &l) {
    uint32_t b03, b47;
    high_bytes(v, b03, b47);
    const uint32_t m03 = b03 & 0xFCFCFCFCu, m47 = b47 & 0xFCFCFCFCu;
    h = zero_bytes4(m03 ^ 0xD8D8D8D8u) | (zero_bytes4(m47 ^ 0xD8D8D8D8u) << 4);
    l = zero_bytes4(m03 ^ 0xDCDCDCDCu) | (zero_bytes4(m47 ^ 0xDCDCDCDCu) << 4);
}

__device__ __forceinline__ bool unit_is_high(uint32_t u) { return (u & 0xFC00u) == 0xD800u; }
__device__ __forceinline__ bool unit_is_low(uint32_t u) { return (u & 0xFC00u) == 0xDC00u; }

// Bit u (u < 4) moved to bit 8*u.
__device__ __forceinline__ uint32_t spread4(uint32_t x) { return (x * 0x00204081u) & 0x01010101u; }

// Replace the units of a 32-bit word (2 units) flagged in bad2 (bits 0, 1).
__device__ __forceinline__ uint32_t fix_word(uint32_t w, uint32_t bad2) {
    const uint32_t m = ((bad2 & 1u) ? 0x0000FFFFu : 0u) | ((bad2 & 2u) ? 0xFFFF0000u : 0u);
    return (w & ~m) | (0xFFFDFFFDu & m);
}

__device__ __forceinline__ uint4 fix_vec(uint4 v, uint32_t bad8) {
    v.x = fix_word(v.x, bad8);
    v.y = fix_word(v.y, bad8 >> 2);
    v.z = fix_word(v.z, bad8 >> 4);
    v.w = fix_word(v.w, bad8 >> 6);
    return v;
}

__device__ __forceinline__ uint32_t vec_unit(const uint4 &v, int k) {
    const uint32_t w = (k < 2) ? v.x : (k < 4) ? v.y : (k < 6) ? v.z : v.w;
    return (k & 1) ? (w >> 16) : (w & 0xFFFFu);
}

__device__ __forceinline__ void vec_set_unit(uint4 &v, int k, uint32_t u) {
    uint32_t *w = (k < 2) ? &v.x : (k < 4) ? &v.y : (k < 6) ? &v.z : &v.w;
    *w = (k & 1) ? ((*w & 0x0000FFFFu) | (u << 16)) : ((*w & 0xFFFF0000u) | u);
}

// Mismatch mask for a warp chunk of U slices (Section 1 rule).
//   h, l       this lane's high / low masks (bit 8u+k)
//   halo_prev  1 if the unit just before the chunk is a high surrogate that
//              may pair with the chunk's first unit (only lane 0's value is used)
//   halo_next  1 if the unit just after the chunk is a low surrogate that may
//              pair with the chunk's last unit (only lane 31's value is used)
//   no_prev    bit 8u+k set: unit k of slice u has no left neighbour (string start)
//   no_next    bit 8u+k set: unit k of slice u has no right neighbour (string end)
// A unit's left neighbour is the previous unit of the same vector, the last
// unit of the previous lane's vector, or (lane 0) the last unit of lane 31's
// vector in the previous slice; symmetrically on the right.
template <int U>
__device__ __forceinline__ uint32_t mismatch_mask(uint32_t h, uint32_t l, uint32_t halo_prev, uint32_t halo_next,
                                                  uint32_t no_prev, uint32_t no_next, int lane) {
    static_assert(U >= 1 && U <= 4, "masks hold at most 4 slices");
    constexpr uint32_t kSliceMask = (U == 4) ? 0xFFFFFFFFu : ((1u << (8 * U)) - 1u);
    uint32_t last_h = 0, first_l = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        last_h |= ((h >> (8 * u + 7)) & 1u) << u;
        first_l |= ((l >> (8 * u)) & 1u) << u;
    }
    uint32_t from_prev = __shfl_sync(kFull, last_h, (lane + 31) & 31);
    uint32_t from_next = __shfl_sync(kFull, first_l, (lane + 1) & 31);
    if (lane == 0) from_prev = ((from_prev << 1) | (halo_prev & 1u)) & ((1u << U) - 1u);
    if (lane == 31) from_next = (from_next >> 1) | ((halo_next & 1u) << (U - 1));
    // bit 8u+k: unit k-1 (or the neighbour) is high / unit k+1 (or the neighbour) is low
    const uint32_t prev_is_high = (((h << 1) & ~0x01010101u) | spread4(from_prev)) & ~no_prev & kSliceMask;
    const uint32_t next_is_low = (((l >> 1) & ~0x80808080u) | (spread4(from_next) << 7)) & ~no_next & kSliceMask;
    return ((h & ~next_is_low) | (l & ~prev_is_high)) & kSliceMask;
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

// Streaming 16-byte loads / stores.
__device__ __forceinline__ uint4 ld_stream(const uint4 *p) { return __ldcs(p); }
__device__ __forceinline__ uint4 ld_nc(const uint4 *p) { return __ldg(p); }
__device__ __forceinline__ uint4 ld_plain(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}
__device__ __forceinline__ void st_stream(uint4 *p, const uint4 &v) { __stcs(p, v); }

// Store the 8 units of v at out + p0, where out + p0 has the alignment
// implied by ST (16, 8, 4 bytes, or 2 = odd unit index relative to 4 bytes).
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
