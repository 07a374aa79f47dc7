// One lane's load of VB bytes (E = VB / 2 code units; VB = 8, 16 or 32) and
// what the bit-word kernels do with it: classify its units into surrogate and
// low-surrogate bits, store them as one table entry, replace units by U+FFFD
// and store it back.  The bit-word layout (32-unit words per lane, built from
// a per-warp table of 64 bits per word) is the same for every width, so the
// width only changes these steps: each load instruction moves 32 * VB bytes
// per warp (8-byte loads: 256 B, 16-byte: 512 B, 32-byte: 1 KiB).
#pragma once

#include <stdint.h>

#include "device.cuh"

namespace u16wf {

template <int VB>
struct LaneVec {
    static_assert(VB == 8 || VB == 16 || VB == 32, "vector width");
    static constexpr int kUnits = VB / 2;
    uint32_t w[VB / 4];
};

// Aligned load of one lane vector; STREAM: evict-first (.cs).
template <int VB, bool STREAM>
__device__ __forceinline__ LaneVec<VB> lv_load(const void *p) {
    LaneVec<VB> v;
    if constexpr (VB == 8) {
        if constexpr (STREAM)
            asm volatile("ld.global.cs.v2.u32 {%0,%1}, [%2];" : "=r"(v.w[0]), "=r"(v.w[1]) : "l"(p));
        else
            asm volatile("ld.global.v2.u32 {%0,%1}, [%2];" : "=r"(v.w[0]), "=r"(v.w[1]) : "l"(p));
    } else if constexpr (VB == 16) {
        if constexpr (STREAM)
            asm volatile("ld.global.cs.v4.u32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(v.w[0]), "=r"(v.w[1]), "=r"(v.w[2]), "=r"(v.w[3])
                         : "l"(p));
        else
            asm volatile("ld.global.v4.u32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(v.w[0]), "=r"(v.w[1]), "=r"(v.w[2]), "=r"(v.w[3])
                         : "l"(p));
    } else {
        if constexpr (STREAM)
            asm volatile("ld.global.cs.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v.w[0]), "=r"(v.w[1]), "=r"(v.w[2]), "=r"(v.w[3]), "=r"(v.w[4]), "=r"(v.w[5]),
                           "=r"(v.w[6]), "=r"(v.w[7])
                         : "l"(p));
        else
            asm volatile("ld.global.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v.w[0]), "=r"(v.w[1]), "=r"(v.w[2]), "=r"(v.w[3]), "=r"(v.w[4]), "=r"(v.w[5]),
                           "=r"(v.w[6]), "=r"(v.w[7])
                         : "l"(p));
    }
    return v;
}

template <int VB>
__device__ __forceinline__ uint32_t lv_unit(const LaneVec<VB> &v, int k) {
    const uint32_t w = v.w[k >> 1];
    return (k & 1) ? (w >> 16) : (w & 0xFFFFu);
}

template <int VB>
__device__ __forceinline__ void lv_set_unit(LaneVec<VB> &v, int k, uint32_t u) {
    uint32_t &w = v.w[k >> 1];
    w = (k & 1) ? ((w & 0x0000FFFFu) | (u << 16)) : ((w & 0xFFFF0000u) | u);
}

// Classification on the high byte (Section 3.3): the table entry of the
// vector -- its E surrogate bits in bits 0..E-1 and its E low-surrogate bits
// in bits E..2E-1 (bit k = unit k) -- and, ORed into acc, the surrogate
// byte-lane flags (nonzero iff some unit is a surrogate).
template <int VB>
__device__ __forceinline__ uint32_t lv_classify(const LaneVec<VB> &v, uint32_t &acc) {
    if constexpr (VB == 8) {
        const uint32_t hb = prmt(v.w[0], v.w[1], 0x7531);
        const uint32_t sf = surrogate_flags(hb);
        acc |= sf;
        const uint32_t s4 = pack_flags8(sf, 0u) >> 24;                // units 0..3 at bits 0..3
        const uint32_t l4 = pack_flags8(sf & (hb << 5), 0u) >> 24;
        return s4 | (l4 << 4);
    } else {
        uint32_t s[VB / 16], l[VB / 16];
#pragma unroll
        for (int h = 0; h < VB / 16; ++h) {
            const uint32_t hb0 = prmt(v.w[4 * h], v.w[4 * h + 1], 0x7531);
            const uint32_t hb1 = prmt(v.w[4 * h + 2], v.w[4 * h + 3], 0x7531);
            const uint32_t sf0 = surrogate_flags(hb0);
            const uint32_t sf1 = surrogate_flags(hb1);
            acc |= sf0 | sf1;
            s[h] = pack_flags8(sf0, sf1);  // byte 3: units 8h..8h+7
            l[h] = pack_flags8(sf0 & (hb0 << 5), sf1 & (hb1 << 5));
        }
        if constexpr (VB == 16) return prmt(s[0], l[0], 0x0073);  // S8 | L8 << 8
        // S16 | L16 << 16
        return prmt(prmt(s[0], s[1], 0x0073), prmt(l[0], l[1], 0x0073), 0x5410);
    }
}

template <int VB>
__device__ __forceinline__ void lv_store_entry(void *table, int idx, uint32_t entry) {
    if constexpr (VB == 8)
        reinterpret_cast<uint8_t *>(table)[idx] = (uint8_t)entry;
    else if constexpr (VB == 16)
        reinterpret_cast<uint16_t *>(table)[idx] = (uint16_t)entry;
    else
        reinterpret_cast<uint32_t *>(table)[idx] = entry;
}

// A lane word's 32 units from its 8 bytes of table (x: the first four bytes,
// y: the last four): surrogate bits S and low-surrogate bits L, bit j = unit j.
template <int VB>
__device__ __forceinline__ void lv_word_bits(uint32_t x, uint32_t y, uint32_t &S, uint32_t &L) {
    if constexpr (VB == 16) {
        S = prmt(x, y, 0x6420);
        L = prmt(x, y, 0x7531);
    } else if constexpr (VB == 32) {
        S = prmt(x, y, 0x5410);
        L = prmt(x, y, 0x7632);
    } else {
        // Eight entries of one byte each, S in the low nibble: compact the
        // nibbles of each word into 16 bits, in order.
        auto compact = [](uint32_t t) {
            t &= 0x0F0F0F0Fu;
            t = (t | (t >> 4)) & 0x00FF00FFu;
            return (t | (t >> 8)) & 0x0000FFFFu;
        };
        S = compact(x) | (compact(y) << 16);
        L = compact(x >> 4) | (compact(y >> 4) << 16);
    }
}

// Replace by U+FFFD every unit k of v with bit k of `bits` set.  Per group of
// four units the bits become byte-lane flags (bit k to bit 8k+7), and prmt
// with a selector nibble 8+k replicates byte k's top bit into a 16-bit mask.
template <int VB>
__device__ __forceinline__ void lv_fix(LaneVec<VB> &v, uint32_t bits) {
#pragma unroll
    for (int g = 0; g < VB / 8; ++g) {
        const uint32_t f = spread4((bits >> (4 * g)) & 0xFu) << 7;
        uint32_t m = prmt(f, 0u, 0x9988);
        v.w[2 * g] = (v.w[2 * g] & ~m) | (0xFFFDFFFDu & m);
        m = prmt(f, 0u, 0xBBAA);
        v.w[2 * g + 1] = (v.w[2 * g + 1] & ~m) | (0xFFFDFFFDu & m);
    }
}

// Store the E units of v at d (streaming), whose alignment in bytes is at
// least ST (32, 16, 8, 4, or 2 for an odd unit address relative to 4 bytes).
template <int VB, int ST>
__device__ __forceinline__ void lv_store(uint16_t *d, const LaneVec<VB> &v) {
    if constexpr (VB == 32 && ST == 32) {
        asm volatile("st.global.cs.v8.u32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(d), "r"(v.w[0]), "r"(v.w[1]),
                     "r"(v.w[2]), "r"(v.w[3]), "r"(v.w[4]), "r"(v.w[5]), "r"(v.w[6]), "r"(v.w[7])
                     : "memory");
    } else if constexpr (VB >= 16) {
        constexpr int S16 = ST > 16 ? 16 : ST;
#pragma unroll
        for (int h = 0; h < VB / 16; ++h)
            store_vec<S16>(d + 8 * h, make_uint4(v.w[4 * h], v.w[4 * h + 1], v.w[4 * h + 2], v.w[4 * h + 3]));
    } else if constexpr (ST >= 8) {
        __stcs(reinterpret_cast<uint2 *>(d), make_uint2(v.w[0], v.w[1]));
    } else if constexpr (ST == 4) {
        __stcs(reinterpret_cast<uint32_t *>(d), v.w[0]);
        __stcs(reinterpret_cast<uint32_t *>(d) + 1, v.w[1]);
    } else {
        d[0] = (uint16_t)(v.w[0] & 0xFFFFu);
        __stcs(reinterpret_cast<uint32_t *>(d + 1), __byte_perm(v.w[0], v.w[1], 0x5432));
        d[3] = (uint16_t)(v.w[1] >> 16);
    }
}

// Largest store alignment class of `out` relative to `in` for VB-byte
// vectors read from VB-aligned addresses of `in`.
__host__ __device__ inline int lv_store_class(const void *in, const void *out, int vb) {
    const unsigned rel = (unsigned)(((uintptr_t)out - (uintptr_t)in) & (unsigned)(vb - 1));
    if (rel == 0) return vb;
    return (rel % 16 == 0) ? 16 : (rel % 8 == 0) ? 8 : (rel % 4 == 0) ? 4 : 2;
}

}  // namespace u16wf
