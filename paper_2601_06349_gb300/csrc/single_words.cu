// In-place toWellFormed of a single string on bit words (Section 1 rule,
// Section 3.2 in-place form: only replaced units are written).
//
// Per warp chunk of U slices (U = 4 or 8: 1024 or 2048 units):
//   1. load the lane's U vectors (128-bit loads) and the units just outside
//      the chunk (lanes 0 and 31);
//   2. classify every unit on its high byte (Section 3.3) and pack, per
//      vector, its surrogate bits and low-surrogate bits (bit k = unit k) into
//      a 16-bit entry of a per-warp table; a chunk without any surrogate is
//      done;
//   3. read the table back four entries at a time: lane l then holds units
//      [1024 j + 32 l, +32) of the chunk as 32-bit words H (high) and L (low);
//   4. the rule is word logic: a high unit whose next unit is not low, a low
//      unit whose previous unit is not high; the neighbour bits across words
//      come from the adjacent lane (shuffles) or the units outside the chunk;
//   5. store 0xFFFD at every set bit of the bad words, one 2-byte store each,
//      or, when some lane has more than kSparseMax of them, write the bad
//      words back to the table (byte v of the table is then vector v's 8
//      bits) and store each 16-byte block that holds a replaced unit.
// Step 5 needs no ordering between warps or blocks: replacing a mismatched
// unit by 0xFFFD never changes a neighbour's verdict (H and FFFD are both
// non-low, L and FFFD both non-high).
#include <cuda_runtime.h>
#include <limits.h>

#include "device.cuh"
#include "internal.h"
#include "single.cuh"

namespace u16wf {

namespace {

// Above this many replaced units in one lane word (any lane of the warp) the
// chunk stores whole 16-byte blocks instead of single units.
constexpr int kSparseMax = 4;

template <int U>
struct __align__(16) WordTable {
    uint16_t cls[U * 32];   // vector v: bit k = unit k is a surrogate, bit 8+k = it is a low one
    uint32_t bad[U * 8];    // the bad words (byte v = vector v's 8 bits) for the block stores
};

// Bits of the 32-unit word whose first unit is `first` that lie in [0, n).
__device__ __forceinline__ uint32_t word_inside(long long first, long long n) {
    const int lo = first >= 0 ? 0 : first < -32 ? 32 : (int)-first;        // units before the string
    const int hi = n - first <= 0 ? 0 : n - first >= 32 ? 32 : (int)(n - first);  // units up to its end
    const uint32_t from_lo = lo >= 32 ? 0u : 0xFFFFFFFFu << lo;
    const uint32_t below_hi = hi >= 32 ? 0xFFFFFFFFu : (1u << hi) - 1u;
    return from_lo & below_hi;
}

template <bool FB, int U>
__device__ __forceinline__ void inplace_words_chunk(const SingleArgs &A, long long cfirst, const Chunk<U> &ch,
                                                    int lane, WordTable<U> &ws, long long &my_first) {
    constexpr int NW = U / 4;  // 32-unit words per lane
    constexpr long long CU = (long long)U * kWarpSliceUnits;
    static_assert(NW == 1 || NW == 2, "chunk width");

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
    if (!__any_sync(kFull, acc != 0)) return;  // no surrogate: nothing to replace
    __syncwarp();

    uint32_t H[NW], L[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const uint2 t = *reinterpret_cast<const uint2 *>(&ws.cls[128 * j + 4 * lane]);
        const uint32_t s32 = prmt(t.x, t.y, 0x6420);
        L[j] = prmt(t.x, t.y, 0x7531);
        H[j] = s32 & ~L[j];
    }
    // At an end of the string the units at -1 and n carry the lead and trail
    // units (a chunk of a longer string sees its neighbours), so the rule can
    // flag them: only units inside [0, n) are kept.
    const bool edge = (cfirst < 0) || (cfirst + CU > A.n);
    uint32_t bad[NW];
    int pop = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const uint32_t h_up = __shfl_sync(kFull, (j > 0 && lane == 31) ? H[j > 0 ? j - 1 : 0] : H[j], (lane + 31) & 31);
        const uint32_t l_dn =
            __shfl_sync(kFull, (j < NW - 1 && lane == 0) ? L[j < NW - 1 ? j + 1 : j] : L[j], (lane + 1) & 31);
        const uint32_t h_in = (j == 0 && lane == 0) ? (unit_is_high(ch.halo) ? 1u : 0u) : (h_up >> 31);
        const uint32_t l_in = (j == NW - 1 && lane == 31) ? (unit_is_low(ch.halo) ? 1u : 0u) : l_dn & 1u;
        const uint32_t hprev = (H[j] << 1) | h_in;
        const uint32_t lnext = (L[j] >> 1) | (l_in << 31);
        bad[j] = (H[j] & ~lnext) | (L[j] & ~hprev);
        if (edge) bad[j] &= word_inside(cfirst + 1024 * j + 32 * lane, A.n);
        pop += __popc(bad[j]);
    }
    const unsigned most = __reduce_max_sync(kFull, (unsigned)pop);
    if (most == 0) return;

    if constexpr (FB) {
        unsigned long long nz = __ballot_sync(kFull, bad[0] != 0);
        if constexpr (NW == 2) nz |= (unsigned long long)__ballot_sync(kFull, bad[1] != 0) << 32;
        const int w0 = __ffsll((long long)nz) - 1;
        uint32_t b = __shfl_sync(kFull, bad[0], w0 & 31);
        if constexpr (NW == 2) {
            const uint32_t x = __shfl_sync(kFull, bad[1], w0 & 31);
            b = (w0 >> 5) ? x : b;
        }
        const long long p = cfirst + 32 * w0 + __ffs(b) - 1;
        my_first = p < my_first ? p : my_first;
    }

    if (A.unit_stores || most <= (unsigned)kSparseMax) {
        // Only units inside the string are bad (above), so every store lands
        // inside it.
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            uint16_t *base = A.out + cfirst + 1024 * j + 32 * lane;
            uint32_t rest = bad[j];
            while (rest) {
                base[__ffs(rest) - 1] = (uint16_t)0xFFFDu;
                rest &= rest - 1;
            }
        }
        return;
    }
    // Dense: back to one byte per vector, then 16-byte blocks.
#pragma unroll
    for (int j = 0; j < NW; ++j) ws.bad[32 * j + lane] = bad[j];
    __syncwarp();
    const long long lfirst = cfirst + lane * kUnitsPerVec;
    uint16_t *dst = A.out + lfirst;
    const uint8_t *bytes = reinterpret_cast<const uint8_t *>(ws.bad);
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t bits8 = bytes[32 * u + lane];
        if (bits8) {
            uint32_t lo, hi;
            bits_to_flags(bits8, lo, hi);
            store_chunk_vec<kModeInPlace, 16>(dst, u, fix_vec(ch.v[u], lo, hi), edge, lfirst + u * kWarpSliceUnits,
                                              A.n, bits8);
        }
    }
}

template <bool FB, int U, bool PF>
__global__ void __launch_bounds__(kMaxBlockThreads) inplace_words_kernel(const SingleArgs A) {
    constexpr long long CU = (long long)U * kWarpSliceUnits;
    __shared__ WordTable<U> s_table[kMaxBlockThreads / 32];
    const int lane = threadIdx.x & 31;
    WordTable<U> &ws = s_table[threadIdx.x >> 5];
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const uint4 *vin = reinterpret_cast<const uint4 *>(A.in - A.a);
    long long my_first = LLONG_MAX;
    wait_prior_grids();
    if constexpr (PF) {
        Chunk<U> nv;
        long long c = gwarp;
        if (c < A.chunks) load_chunk<kModeInPlace, U>(A, vin, c, lane, nv);
        while (c < A.chunks) {
            const Chunk<U> v = nv;
            const long long cur = c;
            c += nwarps;
            if (c < A.chunks) load_chunk<kModeInPlace, U>(A, vin, c, lane, nv);
            inplace_words_chunk<FB, U>(A, cur * CU - A.a, v, lane, ws, my_first);
        }
    } else {
        for (long long c = gwarp; c < A.chunks; c += nwarps) {
            Chunk<U> v;
            load_chunk<kModeInPlace, U>(A, vin, c, lane, v);
            inplace_words_chunk<FB, U>(A, c * CU - A.a, v, lane, ws, my_first);
        }
    }
    allow_next_grid();
    if constexpr (FB) finish_first_bad(A, my_first, lane);
}

template <bool FB, int U>
const void *words_ptr(bool pf) {
    return pf ? (const void *)inplace_words_kernel<FB, U, true> : (const void *)inplace_words_kernel<FB, U, false>;
}

}  // namespace

const void *inplace_words_kernel_for(bool fb, int u, bool pf) {
    if (u == 8) return fb ? words_ptr<true, 8>(pf) : words_ptr<false, 8>(pf);
    return fb ? words_ptr<true, 4>(pf) : words_ptr<false, 4>(pf);
}

}  // namespace u16wf
