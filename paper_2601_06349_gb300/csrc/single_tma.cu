// TMA-staged single-string kernel: the same per-chunk work as single.cu, with
// the input streamed into shared memory by bulk copies (cp.async.bulk, the
// 1-D form of the Tensor Memory Accelerator) instead of per-thread 128-bit
// loads, so that the bytes in flight per SM no longer depend on registers.
//
// A block of 8 warps owns "tiles" of 8192 units (16 KiB, one warp chunk of
// 1024 units per warp).  Thread 0 copies tile t together with one 16-byte
// vector on each side (the halo: the units just before and after the tile)
// into one of S shared-memory stages, completing on that stage's mbarrier.
// Tiles go to blocks in grid-stride order; each block keeps S - 1 copies in
// flight ahead of the tile it is working on.  Warps read their vectors from
// the stage (conflict-free 16-byte shared loads), and the units just outside
// each warp's chunk from the stage as well.  Stores go from registers to
// global memory exactly as in the 128-bit-load kernel.
//
// Tiles whose halo would leave the string (the first tile and the last one or
// two) are handled per warp chunk with the 128-bit-load code path.
//
// Every wait on an mbarrier is bounded (iteration count and a 1-second
// global-timer limit).  On expiry the kernel records an error in
// g_tma_timeout, waits (bounded again) for its own copies still in flight,
// and finishes without further work; utf16_check_device_errors() reports it.
#include <cuda_runtime.h>
#include <limits.h>

#include "../../include/utf16wf.h"
#include "device.cuh"
#include "internal.h"
#include "single.cuh"

namespace u16wf {

constexpr int kTmaU = 4;
constexpr int kTileUnits = (kBlockThreads / 32) * kTmaU * kWarpSliceUnits;  // 8192
constexpr int kTileVecs = kTileUnits / kUnitsPerVec;                        // 1024
constexpr int kStageVecs = kTileVecs + 2;                                   // + halo vector on each side
constexpr unsigned kStageBytes = kStageVecs * 16u;                          // 16,416 bytes
constexpr int kTmaStages = 4;
constexpr size_t kTmaSmemBytes = (size_t)kTmaStages * kStageBytes;

__device__ unsigned int g_tma_timeout = 0;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for phase `parity` of `bar`: false after 2^22 polls or
// `limit_ns` nanoseconds (1 s by default).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  unsigned long long limit_ns = 1000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned i = 0; i < (1u << 22); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// Self-test of the bounded wait: one thread waits on a barrier that nothing
// completes; the wait must give up, record the timeout like the TMA kernel
// does, and return.
__global__ void bounded_wait_probe(unsigned long long limit_ns, unsigned int *gave_up) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const bool done = mbar_wait_bounded(&bar, 0, limit_ns);
        *gave_up = done ? 0u : 1u;
        if (!done) atomicExch(&g_tma_timeout, 1u);
    }
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

struct TmaArgs {
    SingleArgs s;
    long long tile_lo, tile_hi;  // tiles [tile_lo, tile_hi) go through shared memory
    long long edge_chunks_lo;    // warp chunks [0, edge_chunks_lo) and
    long long edge_chunks_hi;    // [edge_chunks_hi, s.chunks) use 128-bit loads
};

template <int MODE, bool FB>
__global__ void __launch_bounds__(kBlockThreads) single_tma_kernel(const TmaArgs T) {
    extern __shared__ __align__(128) uint4 stages[];
    __shared__ __align__(8) unsigned long long full[kTmaStages];
    __shared__ int s_issued;
    __shared__ int s_fault;

    const SingleArgs &A = T.s;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    long long my_first = LLONG_MAX;
    const uint4 *vin = reinterpret_cast<const uint4 *>(A.in - A.a);
    __shared__ unsigned long long s_best;  // check: this block's smallest published mismatch
    wait_prior_grids();
    if (threadIdx.x == 0) s_best = ~0ull;

    // Tiles of this block: tile_lo + blockIdx.x + k * gridDim.x.
    const long long first_tile = T.tile_lo + blockIdx.x;
    const long long my_tiles =
        first_tile < T.tile_hi ? (T.tile_hi - first_tile + gridDim.x - 1) / gridDim.x : 0;

    auto issue = [&](long long k) {
        const int s = (int)(k % kTmaStages);
        const long long t = first_tile + k * gridDim.x;
        // units [t*8192 - a - 8, (t+1)*8192 - a + 8): 16-byte aligned in global memory
        const uint4 *src = vin + t * kTileVecs - 1;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&full[s], kStageBytes);
        bulk_copy_g2s(stages + (size_t)s * kStageVecs, src, kStageBytes, &full[s]);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTmaStages; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fault = 0;
        int issued = 0;
        for (; issued < kTmaStages && issued < my_tiles; ++issued) issue(issued);
        s_issued = issued;
    }
    __syncthreads();

    // Chunks at the ends of the string, with 128-bit and unit loads, while
    // the first copies are in flight.
    {
        const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
        const long long n_lo = T.edge_chunks_lo, n_hi = A.chunks - T.edge_chunks_hi;
        for (long long e = gwarp; e < n_lo + n_hi; e += nwarps) {
            const long long c = e < n_lo ? e : T.edge_chunks_hi + (e - n_lo);
            Chunk<kTmaU> ch;
            load_chunk<MODE, kTmaU>(A, vin, c, lane, ch);
            process_chunk<MODE, FB, 16, kTmaU>(A, c * (kTmaU * kWarpSliceUnits) - A.a, ch, lane, my_first, &s_best);
        }
    }

    for (long long k = 0; k < my_tiles; ++k) {
        if (k >= s_issued) break;  // copies stopped early (first error already known)
        const int s = (int)(k % kTmaStages);
        const unsigned parity = (unsigned)((k / kTmaStages) & 1);
        // One thread polls; the others wait at the barrier and then observe
        // the completed phase themselves (one try_wait each, which acquires
        // the copied bytes).
        if (threadIdx.x == 0 && !mbar_wait_bounded(&full[s], parity)) {
            atomicExch(&g_tma_timeout, 1u);
            s_fault = 1;
        }
        __syncthreads();
        if (s_fault) break;
        if (!mbar_try_wait(&full[s], parity) && !mbar_wait_bounded(&full[s], parity)) atomicExch(&g_tma_timeout, 1u);
        const long long t = first_tile + k * gridDim.x;
        const long long tile_first = t * kTileUnits - A.a;
        const uint4 *stage = stages + (size_t)s * kStageVecs;
        const uint16_t *stage_units = reinterpret_cast<const uint16_t *>(stage);
        bool skip = false;
        if constexpr (MODE == kModeCheck) {
            if (!A.full_pass) {  // the block's shared best: thread 0 folds the global minimum into it
                const unsigned long long g = *((volatile unsigned long long *)&s_best);
                skip = (g != ~0ull && (long long)g < tile_first);
            }
        }
        if (!skip) {
            Chunk<kTmaU> ch;
#pragma unroll
            for (int u = 0; u < kTmaU; ++u) ch.v[u] = stage[1 + warp * (32 * kTmaU) + u * 32 + lane];
            // units just outside this warp's chunk, from the stage (tile halo at the tile ends)
            const int r = warp * (kTmaU * kWarpSliceUnits) + kUnitsPerVec;
            ch.halo = 0;
            if (lane == 0) ch.halo = stage_units[r - 1];
            if (lane == 31) ch.halo = stage_units[r + kTmaU * kWarpSliceUnits];
            const long long cfirst = tile_first + (long long)warp * (kTmaU * kWarpSliceUnits);
            process_chunk<MODE, FB, 16, kTmaU>(A, cfirst, ch, lane, my_first, &s_best);
        }
        __syncthreads();  // every warp is done with stage s
        if (threadIdx.x == 0) {
            const long long next = k + kTmaStages;
            bool go = next < my_tiles;
            if constexpr (MODE == kModeCheck) {
                const unsigned long long g = *((volatile unsigned long long *)&A.slot->min);
                if (g != ~0ull) atomicMin(&s_best, g);
                if (!A.full_pass && g != ~0ull && (long long)g < (first_tile + next * gridDim.x) * kTileUnits - A.a)
                    go = false;
            }
            if (go) {
                issue(next);
                s_issued = (int)(next + 1);
            }
        }
        __syncthreads();
    }

    // After a timeout, wait (bounded) for this block's copies still in flight
    // so that none lands in shared memory after the block has exited.
    if (s_fault && threadIdx.x == 0) {
        for (long long k = 0; k < s_issued; ++k) {
            const int s = (int)(k % kTmaStages);
            mbar_wait_bounded(&full[s], (unsigned)((k / kTmaStages) & 1));
        }
    }
    __syncthreads();
    allow_next_grid();
    if constexpr (FB) finish_first_bad(A, my_first, lane);
}

template <int MODE, bool FB>
static const void *tma_ptr() {
    return (const void *)single_tma_kernel<MODE, FB>;
}

const void *single_tma_kernel_for_occupancy(int mode, bool fb) {
    if (mode == kModeCheck) return tma_ptr<kModeCheck, true>();
    if (mode == kModeInPlace) return fb ? tma_ptr<kModeInPlace, true>() : tma_ptr<kModeInPlace, false>();
    return fb ? tma_ptr<kModeOut, true>() : tma_ptr<kModeOut, false>();
}

size_t single_tma_smem_bytes() { return kTmaSmemBytes; }

cudaError_t launch_single_tma(const SingleLaunch &L, cudaStream_t stream) {
    TmaArgs T;
    T.s = make_single_args(L, kTmaU * kWarpSliceUnits);
    const long long n = L.n, a = T.s.a;
    // Tile t covers units [t*8192 - a, (t+1)*8192 - a); it goes through
    // shared memory when its halo vectors lie inside the string.
    const long long tiles = (n + a + kTileUnits - 1) / kTileUnits;
    long long lo = 1;
    long long hi = (n + a - kUnitsPerVec) / kTileUnits;
    if (hi < lo) hi = lo;
    if (lo > tiles) lo = tiles;
    if (hi > tiles) hi = tiles;
    T.tile_lo = lo;
    T.tile_hi = hi;
    constexpr long long chunks_per_tile = kBlockThreads / 32;
    T.edge_chunks_lo = lo * chunks_per_tile < T.s.chunks ? lo * chunks_per_tile : T.s.chunks;
    T.edge_chunks_hi = hi * chunks_per_tile < T.s.chunks ? hi * chunks_per_tile : T.s.chunks;
    if (T.edge_chunks_hi < T.edge_chunks_lo) T.edge_chunks_hi = T.edge_chunks_lo;
    const bool fb = L.first_bad || L.mode == kModeCheck;
    const void *fn = single_tma_kernel_for_occupancy(L.mode, fb);
    const long long work_blocks = (hi - lo) > 0 ? (hi - lo) : 1;
    long long blocks = work_blocks < (long long)L.max_blocks ? work_blocks : L.max_blocks;
    if (blocks < 1) blocks = 1;
    void *args[] = {(void *)&T};
    const long long warps = blocks * (kBlockThreads / 32);
    return launch_kernel(fn, dim3((unsigned)blocks), dim3(kBlockThreads), args, kTmaSmemBytes, stream,
                         pdl_fits((T.s.chunks + warps - 1) / warps, L.full_occupancy));
}

cudaError_t prepare_single_tma() {
    const int modes[3] = {kModeOut, kModeInPlace, kModeCheck};
    for (int m : modes) {
        for (int f = 0; f < 2; ++f) {
            const void *fn = single_tma_kernel_for_occupancy(m, f != 0);
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmemBytes);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

int run_bounded_wait_probe(long long limit_ns) {
    unsigned int *d = nullptr, h = 0;
    if (cudaMalloc((void **)&d, sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    bounded_wait_probe<<<1, 32>>>((unsigned long long)limit_ns, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (int)h;
}

unsigned int read_and_clear_tma_timeout() {
    unsigned int v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_tma_timeout, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (v) cudaMemcpyToSymbol(g_tma_timeout, &z, sizeof(z));
    return v;
}

}  // namespace u16wf
