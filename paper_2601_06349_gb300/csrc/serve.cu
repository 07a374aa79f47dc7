// Serving engine: continuous batching of UTF-16 repair requests.
//
// Requests (one host string each) arrive at any time through
// utf16_server_submit.  A scheduler thread takes whatever has arrived, admits
// requests in arrival order against the device arena (a FIFO ring over one
// allocation of the HBM budget) and launches them as one ragged batch as soon
// as one of the batch slots is free: there is no waiting for a batch to fill.
// Each slot has its own stream, which carries in order:
//   - the offsets and the small requests packed in the slot's pinned staging
//     buffer (one copy), and large requests copied straight from the
//     caller's buffers;
//   - the in-place batch repair with per-string first-error index (one
//     persistent kernel, plus the lengths initialisation);
//   - one host pass per large request whose buffers kernels can reach: the
//     single-string kernel on a few SMs, reading and writing the caller's
//     buffers over the host link;
//   - the first-error indices and the packed region back to staging, large
//     copied requests straight to the caller.
// Batches on different slots overlap, so one batch's input is on its way
// while another computes and a third comes back.  A completion thread polls
// the slots' events, completes batches in the order they finish, scatters
// small results to the callers' buffers, and frees ring space in allocation
// order and the slot, which lets the scheduler admit more requests.
//
// The kernels are the library's own ragged-batch and single-string kernels,
// so a request's result does not depend on which batch or path it takes:
// every string end is a hard boundary.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/utf16wf.h"
#include "internal.h"
#include "runtime.h"

namespace u16wf {

static int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

static int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// FIFO ring allocator over [0, cap): allocations are freed in the order they
// were made, so the live region is one run (or two, once it wraps).
class FifoRing {
   public:
    explicit FifoRing(int64_t cap) : cap_(cap) {}
    int64_t alloc(int64_t size) {
        if (size <= 0 || size > cap_) return -1;
        int64_t off;
        if (live_.empty()) {
            off = 0;
        } else {
            const int64_t oldest = live_.front().first;
            const int64_t newest_end = live_.back().first + live_.back().second;
            if (live_.back().first >= oldest) {  // live: [oldest, newest_end)
                if (cap_ - newest_end >= size)
                    off = newest_end;
                else if (oldest >= size)
                    off = 0;
                else
                    return -1;
            } else {  // wrapped: live [oldest, cap) and [0, newest_end)
                if (oldest - newest_end >= size)
                    off = newest_end;
                else
                    return -1;
            }
        }
        live_.push_back({off, size});
        used_ += size;
        return off;
    }
    bool free_oldest() {
        if (live_.empty()) return false;
        used_ -= live_.front().second;
        live_.pop_front();
        return true;
    }
    int64_t used() const { return used_; }
    int64_t live() const { return (int64_t)live_.size(); }
    int64_t cap() const { return cap_; }

   private:
    int64_t cap_;
    int64_t used_ = 0;
    std::deque<std::pair<int64_t, int64_t>> live_;
};

struct Request {
    uint64_t ticket = 0;
    const uint16_t *in = nullptr;
    uint16_t *out = nullptr;
    int64_t n = 0;
    int64_t arrival_ns = 0;
    int64_t done_ns = 0;
    int64_t first_bad = -1;
    int status = UTF16_OK;
    bool large = false;
    bool direct = false;          // small request whose buffers the GPU reads / writes itself (pinned host memory)
    bool host_pass = false;       // large request repaired by one kernel in the caller's own buffers
    const uint16_t *dev_in = nullptr;   // device view of `in` (direct and host-pass requests)
    uint16_t *dev_out = nullptr;        // device view of `out` (direct and host-pass requests)
    int64_t dev_off = 0;  // unit offset inside the batch (host-pass requests: the index of their string)
};

// One direct request for the gather / scatter kernels.
struct CopyDesc {
    const uint16_t *src;  // caller's input (device view of pinned host memory)
    uint16_t *dst;        // caller's output (same)
    long long off;        // unit offset in the batch
    long long n;
};

constexpr long long kPieceUnits = 4096;  // direct requests are copied in pieces of at most 8 KiB

// Copy pieces of requests between the callers' pinned host buffers and the
// batch in device memory: one warp per piece, four 16-byte loads in flight
// per lane before the stores (the host side is a long-latency link), unit
// copies when the host side is not 16-byte aligned (the batch side always is).
template <bool GATHER>
__global__ void __launch_bounds__(256) copy_requests_kernel(const CopyDesc *descs, int count, uint16_t *units) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int i = gwarp; i < count; i += nwarps) {
        const CopyDesc c = descs[i];
        uint16_t *dev = units + c.off;
        const uint16_t *src = GATHER ? c.src : dev;
        uint16_t *dst = GATHER ? dev : c.dst;
        const bool vec = ((((uintptr_t)c.src | (uintptr_t)c.dst) & 15u) == 0);
        const int n = (int)c.n;
        const int vecs = vec ? n / 8 : 0;
        for (int base = 0; base < vecs; base += 128) {
            uint4 buf[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j = base + k * 32 + lane;
                if (j < vecs) buf[k] = reinterpret_cast<const uint4 *>(src)[j];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j = base + k * 32 + lane;
                if (j < vecs) reinterpret_cast<uint4 *>(dst)[j] = buf[k];
            }
        }
        for (int base = vecs * 8; base < n; base += 256) {
            uint16_t buf[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int j = base + k * 32 + lane;
                if (j < n) buf[k] = src[j];
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int j = base + k * 32 + lane;
                if (j < n) dst[j] = buf[k];
            }
        }
    }
}

struct BatchSlot {
    std::vector<Request> reqs;
    int64_t ring_off = -1;
    uint16_t *d_units = nullptr;
    long long *d_offsets = nullptr;
    long long *d_first = nullptr;
    CopyDesc *d_desc = nullptr;
    char *h_stage = nullptr;  // pinned: [offsets][first][descriptors][staged small units]
    int64_t h_cap = 0;
    int64_t small_units = 0;
    int64_t total_units = 0;
    int64_t head_bytes = 0;  // offsets + first-error region, 256-aligned (same on device and host)
    int64_t first_off = 0;   // byte offset of the first-error array in that region
    int64_t strings = 0;     // strings of the launched batch (requests plus padding strings)
    int64_t desc_off = 0;    // byte offset of the direct-request descriptors in the head region
    int ndirect = 0;
    int64_t unit_cap = 0;    // units the batch's arena space holds after the head region
    std::vector<int> req_of_string;  // request index of each string, -1 for padding
    cudaStream_t stream = nullptr;  // the batch's copies in, kernels and copies out, in order
    Slot *slot = nullptr;           // reduction scratch of the stream's host-pass launches
    cudaEvent_t ev_done = nullptr;
    uint64_t seq = 0;               // launch sequence number (arena space is freed in this order)
    int status = UTF16_OK;
};

// Head layout of a batch of up to `reqs` requests (at most 2*reqs strings:
// a padding string may precede each aligned large request): offsets, then
// first-error indices, each 256-byte aligned.
static void batch_head_layout(int64_t reqs, int64_t pieces, int64_t &first_off, int64_t &head_bytes,
                              int64_t *desc_off = nullptr) {
    first_off = align_up((2 * reqs + 2) * 8, 256);
    const int64_t d = first_off + align_up(2 * reqs * 8, 256);
    if (desc_off) *desc_off = d;
    head_bytes = d + align_up(pieces * (int64_t)sizeof(CopyDesc), 256);
}

static int64_t pieces_of(const Request &r) { return r.direct ? (r.n + kPieceUnits - 1) / kPieceUnits : 0; }

// Host copies between callers' buffers and a slot's pinned staging, spread
// over a few worker threads (the calling thread works too).  Copies are cut
// into pieces of at most 1 MiB so that the threads finish together; a list
// of less than 256 KiB in all is copied by the caller alone.
struct CopyJob {
    void *dst;
    const void *src;
    size_t bytes;
};

class CopyPool {
   public:
    explicit CopyPool(int workers) {
        for (int i = 0; i < workers; ++i) threads_.emplace_back([this] { loop(); });
    }
    ~CopyPool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (std::thread &t : threads_) t.join();
    }
    void run(const std::vector<CopyJob> &jobs) {
        size_t total = 0;
        for (const CopyJob &j : jobs) total += j.bytes;
        if (threads_.empty() || total < (256u << 10)) {
            for (const CopyJob &j : jobs) memcpy(j.dst, j.src, j.bytes);
            return;
        }
        std::unique_lock<std::mutex> lk(mu_);
        // a worker that woke late for the previous list may still hold it
        done_.wait(lk, [&] { return active_ == 0; });
        pieces_.clear();
        for (const CopyJob &j : jobs)
            for (size_t o = 0; o < j.bytes; o += kPiece)
                pieces_.push_back({(char *)j.dst + o, (const char *)j.src + o, std::min(kPiece, j.bytes - o)});
        next_.store(0);
        ++gen_;
        const CopyJob *list = pieces_.data();
        const size_t n = pieces_.size();
        lk.unlock();
        cv_.notify_all();
        work(list, n);
        lk.lock();
        done_.wait(lk, [&] { return active_ == 0; });
    }

   private:
    static constexpr size_t kPiece = 1u << 20;
    void work(const CopyJob *list, size_t n) {
        for (;;) {
            const size_t i = next_.fetch_add(1);
            if (i >= n) return;
            memcpy(list[i].dst, list[i].src, list[i].bytes);
        }
    }
    void loop() {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
            if (stop_) return;
            seen = gen_;
            ++active_;
            const CopyJob *list = pieces_.data();
            const size_t n = pieces_.size();
            lk.unlock();
            work(list, n);
            lk.lock();
            if (--active_ == 0) done_.notify_all();
        }
    }
    std::vector<std::thread> threads_;
    std::vector<CopyJob> pieces_;  // changed only while no worker is active
    std::atomic<size_t> next_{0};
    std::mutex mu_;
    std::condition_variable cv_, done_;
    uint64_t gen_ = 0;
    int active_ = 0;
    bool stop_ = false;
};

}  // namespace u16wf

struct utf16_server {
    utf16_server_options opt;
    int device = 0;
    u16wf::DeviceCtx *ctx = nullptr;
    char *arena = nullptr;
    std::unique_ptr<u16wf::FifoRing> ring;
    std::vector<u16wf::BatchSlot> slots;

    std::mutex mu;
    std::condition_variable cv_sched;  // new requests, freed slots / ring space, shutdown
    std::condition_variable cv_done;   // completions available
    std::deque<u16wf::Request> pending;
    std::deque<int> free_slots;
    std::vector<int> inflight;        // slots whose batch is on the GPU
    std::deque<uint64_t> arena_order;  // batches holding arena space, in allocation order
    std::vector<uint64_t> finished_seqs;  // batches done but whose space waits for an older one
    uint64_t next_seq = 1;
    std::deque<u16wf::Request> completed;
    std::condition_variable cv_inflight;
    bool stopping = false;
    uint64_t next_ticket = 1;
    int64_t submitted = 0, finished = 0;
    utf16_server_stats stats;
    std::unique_ptr<u16wf::CopyPool> pack_pool, unpack_pool;  // staging copies of the scheduler / completer
    std::thread scheduler, completer;
};

namespace u16wf {

static void complete_request(utf16_server *S, Request &r, int status) {
    r.status = status;
    r.done_ns = now_ns();
    S->completed.push_back(r);
    S->finished++;
}

// SMs a host-pass repair may occupy (environment UTF16WF_SERVE_HOST_PASS_SMS;
// 0 turns host passes off).  The kernel streams from and to host memory, so
// a small part of the GPU already keeps up with the host link and the rest
// stays free for the batches of other slots: on 4,000 mixed requests 8 SMs
// gave 814-825K requests/s and p99 0.13 ms at 10 % load, all 152 SMs 750K
// and 0.25 ms, no host passes 748K and 0.32 ms.
static int host_pass_sms() {
    const char *e = getenv("UTF16WF_SERVE_HOST_PASS_SMS");
    return (e && *e) ? atoi(e) : 8;
}

// One large request repaired in the caller's pinned buffers by the fused
// single-string kernel (out of place, or in place when in == out), its
// first-error index written into the batch's slot for its string.
static cudaError_t launch_host_pass(utf16_server *S, BatchSlot &b, const Request &r) {
    SingleLaunch L;
    L.in = r.dev_in;
    L.out = r.dev_out;
    L.n = r.n;
    L.mode = r.dev_in == r.dev_out ? kModeInPlace : kModeOut;
    L.first_bad = true;
    utf16_config cfg = S->ctx->single_config(r.n);
    cfg.single_variant = cfg.inplace_variant = kVariantLdgPrefetch;  // host memory is far: loads in flight
    configure_single(S->ctx, cfg, L);
    const int per_sm = L.max_blocks / S->ctx->sms;
    L.max_blocks = per_sm * std::min(S->ctx->sms, host_pass_sms());
    L.full_occupancy = false;
    L.slot = b.slot;
    L.result = b.d_first + r.dev_off;
    L.lead = 0;
    L.trail = 0;
    return launch_single(L, b.stream);
}

// Build and launch one batch on slot `si` from the admitted requests in it.
// Staged small requests are packed first (through the slot's pinned staging
// buffer); then direct small requests (gathered and scattered by the GPU
// from and to the callers' pinned buffers) and large ones (copy engines),
// each at a 16-byte aligned unit offset, and host-pass requests as empty
// strings (their kernels run after the batch's).  A gap before an aligned request is
// a padding string of its own, so every request is exactly one string.
static void launch_batch_slot(utf16_server *S, int si) {
    BatchSlot &b = S->slots[(size_t)si];
    std::stable_partition(b.reqs.begin(), b.reqs.end(), [](const Request &r) { return !r.large && !r.direct; });
    int64_t *h_off = (int64_t *)b.h_stage;
    int64_t *h_first = (int64_t *)(b.h_stage + b.first_off);
    CopyDesc *h_desc = (CopyDesc *)(b.h_stage + b.desc_off);
    uint16_t *h_units = (uint16_t *)(b.h_stage + b.head_bytes);
    int64_t pos = 0;
    int64_t strings = 0;
    int nd = 0;
    b.req_of_string.clear();
    b.small_units = 0;
    h_off[0] = 0;
    std::vector<CopyJob> jobs;
    for (int i = 0; i < (int)b.reqs.size(); ++i) {
        Request &r = b.reqs[(size_t)i];
        const bool staged = !r.large && !r.direct;
        if (r.host_pass) {
            r.dev_off = strings;  // its string (empty here), whose first-error slot the host pass fills
            h_off[++strings] = pos;
            b.req_of_string.push_back(i);
            continue;
        }
        if (staged) {
            jobs.push_back({h_units + pos, r.in, (size_t)r.n * 2u});
        } else if (pos % 8 != 0) {
            pos = align_up(pos, 8);
            h_off[++strings] = pos;  // padding string
            b.req_of_string.push_back(-1);
        }
        if (r.direct)
            for (int64_t j = 0; j < r.n; j += kPieceUnits)
                h_desc[nd++] = CopyDesc{r.dev_in + j, r.dev_out + j, (long long)(pos + j),
                                        (long long)std::min<int64_t>(kPieceUnits, r.n - j)};
        r.dev_off = pos;
        pos += r.n;
        if (staged) b.small_units = pos;
        h_off[++strings] = pos;
        b.req_of_string.push_back(i);
    }
    S->pack_pool->run(jobs);
    b.total_units = pos;
    b.strings = strings;
    b.ndirect = nd;
    b.status = UTF16_OK;
    if (pos > b.unit_cap) {  // admission reserves an upper bound of this layout; never launch past it
        b.status = UTF16_ENOMEM;
        return;
    }

    // Host-side fault injection of a copy step (testing): the step's copies
    // are not issued and the batch fails as if they had.
    const int64_t fail_mod = S->opt.inject_copy_fail_mod;
    const bool fail_copy = fail_mod > 0 && (int64_t)(b.seq % (uint64_t)fail_mod) == fail_mod - 1;
    const cudaError_t kInjected = cudaErrorUnknown;
    cudaError_t e = (fail_copy && S->opt.inject_copy_fail_step == 0)
                        ? kInjected
                        : cudaMemcpyAsync(b.d_offsets, h_off, (size_t)(strings + 1) * sizeof(int64_t),
                                          cudaMemcpyHostToDevice, b.stream);
    if (e == cudaSuccess && nd)
        e = cudaMemcpyAsync(b.d_desc, h_desc, (size_t)nd * sizeof(CopyDesc), cudaMemcpyHostToDevice, b.stream);
    if (e == cudaSuccess && b.small_units)
        e = cudaMemcpyAsync(b.d_units, h_units, (size_t)b.small_units * 2u, cudaMemcpyHostToDevice, b.stream);
    for (const Request &r : b.reqs)
        if (e == cudaSuccess && r.large && !r.host_pass)
            e = cudaMemcpyAsync(b.d_units + r.dev_off, r.in, (size_t)r.n * 2u, cudaMemcpyHostToDevice, b.stream);
    const int copy_blocks = std::max(1, std::min(S->ctx->sms * 8, (nd + 7) / 8));
    if (e == cudaSuccess && nd) {
        copy_requests_kernel<true><<<copy_blocks, 256, 0, b.stream>>>(b.d_desc, nd, b.d_units);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        BatchLaunch L;
        L.in = b.d_units;
        L.out = b.d_units;
        L.offsets = b.d_offsets;
        L.count = strings;
        L.first_bad = b.d_first;
        L.mode = kModeInPlaceFirst;
        configure_batch(S->ctx, S->ctx->batch_config(b.total_units, strings), L);
        L.units_hint = b.total_units;
        e = launch_batch(L, b.stream);
    }
    if (e == cudaSuccess && nd) {
        copy_requests_kernel<false><<<copy_blocks, 256, 0, b.stream>>>(b.d_desc, nd, b.d_units);
        e = cudaGetLastError();
    }
    // Host-pass requests: after the batch kernel has set their (empty)
    // strings' first-error slots, one fused pass each fills the slot.
    for (const Request &r : b.reqs)
        if (e == cudaSuccess && r.host_pass) e = launch_host_pass(S, b, r);
    if (e == cudaSuccess && fail_copy && S->opt.inject_copy_fail_step == 1) e = kInjected;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_first, b.d_first, (size_t)strings * sizeof(int64_t), cudaMemcpyDeviceToHost, b.stream);
    if (e == cudaSuccess && b.small_units)
        e = cudaMemcpyAsync(h_units, b.d_units, (size_t)b.small_units * 2u, cudaMemcpyDeviceToHost, b.stream);
    for (const Request &r : b.reqs)
        if (e == cudaSuccess && r.large && !r.host_pass)
            e = cudaMemcpyAsync(r.out, b.d_units + r.dev_off, (size_t)r.n * 2u, cudaMemcpyDeviceToHost, b.stream);
    if (e == cudaSuccess) e = cudaEventRecord(b.ev_done, b.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        // Work of this batch already on its stream may still use the slot's
        // staging and arena space, which the completer hands on at once: wait
        // for it first.
        cudaStreamSynchronize(b.stream);
        cudaGetLastError();
        b.status = UTF16_ECUDA;
    }
}

static void scheduler_main(utf16_server *S) {
    cudaSetDevice(S->device);
    const utf16_server_options &o = S->opt;
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        S->cv_sched.wait(lk, [&] { return S->stopping || (!S->pending.empty() && !S->free_slots.empty()); });
        if (S->stopping) break;
        const int si = S->free_slots.front();
        BatchSlot &b = S->slots[(size_t)si];
        b.reqs.clear();
        // Admission in arrival order: stop at the first request that does not
        // fit (keeps FIFO order; a later, smaller request does not overtake).
        // The launch packs staged requests first and then each aligned one
        // (large or direct) at a 16-byte aligned offset, so the units needed
        // are at most the staged units plus, per aligned request, its units
        // and 7 units of padding.
        int64_t nreq = 0, pieces = 0, small_units = 0, aligned_units = 0, bytes = 0, need = 0;
        int64_t first_off = 0, head = 0, desc_off = 0;
        while (!S->pending.empty()) {
            Request &r = S->pending.front();
            if (o.inject_fail_mod > 0 && (int64_t)(r.ticket % (uint64_t)o.inject_fail_mod) == o.inject_fail_mod - 1) {
                // Host-side fault injection: this request's admission fails.
                Request x = r;
                S->pending.pop_front();
                complete_request(S, x, UTF16_ENOMEM);
                S->stats.rejected++;
                S->cv_done.notify_all();
                continue;
            }
            const bool large = r.n * 2 >= o.small_request_bytes;
            // A host-pass request is an empty string of the batch (its result
            // slot); its units stay in the caller's buffers.
            const bool aligned = !r.host_pass && (large || r.direct);
            const int64_t sm2 = small_units + (aligned || r.host_pass ? 0 : r.n);
            const int64_t al2 = aligned_units + (aligned ? r.n + 7 : 0);
            const int64_t u2 = sm2 + al2;
            int64_t f2, h2, d2;
            r.large = large;
            batch_head_layout(nreq + 1, pieces + pieces_of(r), f2, h2, &d2);
            const int64_t need2 = h2 + align_up(u2 * 2, 256);
            if (2 * (nreq + 1) > o.max_batch_strings || (nreq > 0 && bytes + r.n * 2 > o.max_batch_bytes) ||
                h2 + sm2 * 2 > b.h_cap || need2 > S->ring->cap())
                break;
            nreq += 1;
            pieces += pieces_of(r);
            small_units = sm2;
            aligned_units = al2;
            bytes += r.n * 2;
            need = need2;
            first_off = f2;
            head = h2;
            desc_off = d2;
            r.large = large;
            b.reqs.push_back(r);
            S->pending.pop_front();
        }
        if (b.reqs.empty()) continue;
        // Reserve arena space; wait for completions while it does not fit.
        int64_t ring_off;
        while ((ring_off = S->ring->alloc(need)) < 0) {
            if (S->inflight.empty() || S->stopping) break;
            S->cv_sched.wait(lk);
        }
        if (ring_off < 0) {
            for (Request &r : b.reqs) complete_request(S, r, S->stopping ? UTF16_ECLOSED : UTF16_ENOMEM);
            b.reqs.clear();
            S->cv_done.notify_all();
            if (S->stopping) break;
            continue;
        }
        S->free_slots.pop_front();
        b.seq = S->next_seq++;
        S->arena_order.push_back(b.seq);
        b.ring_off = ring_off;
        b.first_off = first_off;
        b.head_bytes = head;
        b.desc_off = desc_off;
        b.small_units = 0;
        char *base = S->arena + ring_off;
        b.d_offsets = (long long *)base;
        b.d_first = (long long *)(base + first_off);
        b.d_desc = (CopyDesc *)(base + desc_off);
        b.d_units = (uint16_t *)(base + head);
        b.unit_cap = (need - head) / 2;
        S->stats.batches++;
        S->stats.max_batch_requests = std::max(S->stats.max_batch_requests, nreq);
        lk.unlock();
        launch_batch_slot(S, si);
        lk.lock();
        S->inflight.push_back(si);
        S->cv_inflight.notify_all();
    }
    // Shutdown: whatever is still pending is closed.
    while (!S->pending.empty()) {
        Request x = S->pending.front();
        S->pending.pop_front();
        complete_request(S, x, UTF16_ECLOSED);
    }
    S->cv_done.notify_all();
}

// Completes batches in the order they finish on the GPU (a batch of small
// requests does not wait behind an older one that carries a large request),
// and frees arena space in allocation order as the oldest batches finish.
static void completer_main(utf16_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    std::vector<int> polling;
    while (true) {
        S->cv_inflight.wait(lk, [&] { return !S->inflight.empty() || S->stopping; });
        if (S->inflight.empty() && S->stopping) break;
        polling = S->inflight;
        lk.unlock();
        int si = -1, status = UTF16_OK;
        for (int cand : polling) {
            const BatchSlot &c = S->slots[(size_t)cand];
            if (c.status != UTF16_OK) {
                si = cand;
                status = c.status;
                break;
            }
            const cudaError_t q = cudaEventQuery(c.ev_done);
            if (q == cudaErrorNotReady) continue;
            si = cand;
            if (q != cudaSuccess) {
                cudaGetLastError();
                status = UTF16_ECUDA;
            }
            break;
        }
        if (si < 0) {
            std::this_thread::yield();
            lk.lock();
            continue;
        }
        BatchSlot &b = S->slots[(size_t)si];
        const int64_t *h_first = (const int64_t *)(b.h_stage + b.first_off);
        const uint16_t *h_units = (const uint16_t *)(b.h_stage + b.head_bytes);
        std::vector<CopyJob> jobs;
        for (int64_t s = 0; s < b.strings; ++s) {
            const int ri = b.req_of_string[(size_t)s];
            if (ri < 0) continue;
            Request &r = b.reqs[(size_t)ri];
            if (status == UTF16_OK && !r.large && !r.direct) jobs.push_back({r.out, h_units + r.dev_off, (size_t)r.n * 2u});
            r.first_bad = h_first[s];
        }
        S->unpack_pool->run(jobs);
        const int64_t t_done = now_ns();
        lk.lock();
        for (Request &r : b.reqs) {
            r.status = status;
            r.done_ns = std::max(t_done, now_ns());
            S->completed.push_back(r);
            S->finished++;
            S->stats.completed++;
            S->stats.units += r.n;
        }
        b.reqs.clear();
        S->inflight.erase(std::find(S->inflight.begin(), S->inflight.end(), si));
        S->finished_seqs.push_back(b.seq);
        for (bool freed = true; freed && !S->arena_order.empty();) {
            auto it = std::find(S->finished_seqs.begin(), S->finished_seqs.end(), S->arena_order.front());
            freed = it != S->finished_seqs.end();
            if (freed) {
                S->finished_seqs.erase(it);
                S->arena_order.pop_front();
                S->ring->free_oldest();
            }
        }
        S->free_slots.push_back(si);
        S->cv_sched.notify_all();
        S->cv_done.notify_all();
    }
}

}  // namespace u16wf

using namespace u16wf;

extern "C" {

int utf16_server_default_options(utf16_server_options *o) {
    if (!o) return UTF16_EINVAL;
    o->hbm_budget_bytes = 4LL << 30;
    o->max_batch_strings = 1 << 16;
    // 16 MiB batches with 8 slots: on 4,000 mixed requests (1 % of them 2-32
    // MiB) 753-766K requests/s and p99 0.85-0.91 ms at 90 % of that, against
    // 628K and 1.9 ms with 256 MiB batches and 4 slots (a batch of large
    // requests no longer holds up the small ones behind it).
    o->max_batch_bytes = 16LL << 20;
    o->max_inflight_batches = 8;
    o->staging_bytes = 32LL << 20;
    o->small_request_bytes = 256LL << 10;
    o->inject_fail_mod = 0;
    o->direct_host_access = 0;
    o->inject_copy_fail_mod = 0;
    o->inject_copy_fail_step = 0;
    return UTF16_OK;
}

int utf16_server_create(const utf16_server_options *opt, utf16_server **out) {
    if (!opt || !out) return UTF16_EINVAL;
    const utf16_server_options &o = *opt;
    if (o.hbm_budget_bytes < (1 << 20) || o.max_batch_strings < 2 || o.max_batch_bytes < 1024 ||
        o.max_inflight_batches < 1 || o.max_inflight_batches > 64 || o.staging_bytes < 4096 ||
        o.small_request_bytes < 0 || o.inject_fail_mod < 0 || o.direct_host_access < 0 || o.direct_host_access > 1 ||
        o.inject_copy_fail_mod < 0 || o.inject_copy_fail_step < 0 || o.inject_copy_fail_step > 1)
        return UTF16_EINVAL;
    std::unique_ptr<utf16_server> S(new utf16_server());
    S->opt = o;
    memset(&S->stats, 0, sizeof(S->stats));
    if (cudaGetDevice(&S->device) != cudaSuccess) return UTF16_ECUDA;
    int rc = get_ctx(&S->ctx);
    if (rc) return rc;
    if (cudaMalloc((void **)&S->arena, (size_t)o.hbm_budget_bytes) != cudaSuccess) {
        cudaGetLastError();
        return UTF16_ENOMEM;
    }
    S->ring.reset(new FifoRing(o.hbm_budget_bytes));
    S->slots.resize((size_t)o.max_inflight_batches);
    for (int i = 0; i < o.max_inflight_batches; ++i) {
        BatchSlot &b = S->slots[(size_t)i];
        b.h_cap = o.staging_bytes;
        if (cudaHostAlloc((void **)&b.h_stage, (size_t)b.h_cap, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return UTF16_ENOMEM;
        }
        if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b.ev_done, cudaEventDisableTiming) != cudaSuccess)
            return UTF16_ECUDA;
        rc = S->ctx->slot_for(b.stream, &b.slot);  // allocated now, not on the scheduler's path
        if (rc) return rc;
        S->free_slots.push_back(i);
    }
    {
        const unsigned hw = std::thread::hardware_concurrency();
        const int workers = hw >= 16 ? 3 : hw >= 8 ? 1 : 0;
        S->pack_pool.reset(new CopyPool(workers));
        S->unpack_pool.reset(new CopyPool(workers));
    }
    utf16_server *raw = S.release();
    raw->scheduler = std::thread(scheduler_main, raw);
    raw->completer = std::thread(completer_main, raw);
    *out = raw;
    return UTF16_OK;
}

int64_t utf16_server_clock_ns(void) { return now_ns(); }

int utf16_server_submit(utf16_server *S, const uint16_t *host_in, uint16_t *host_out, int64_t n, int64_t arrival_ns,
                        uint64_t *ticket) {
    if (!S || n < 0 || (n > 0 && (!host_in || !host_out))) return UTF16_EINVAL;
    // Every request must fit an otherwise empty arena and staging buffer.
    const int64_t need = 1024 + align_up(n * 2, 256) + 512;
    const bool large = n * 2 >= S->opt.small_request_bytes;
    // (max_batch_bytes only bounds packing: a longer request forms a batch alone.)
    if (need > S->opt.hbm_budget_bytes || (!large && n * 2 + 1024 > S->opt.staging_bytes)) return UTF16_ENOMEM;
    // Small requests whose buffers are pinned host memory are gathered and
    // scattered by the GPU itself (no staging copies on the CPU).
    bool direct = false;
    const uint16_t *dev_in = nullptr;
    uint16_t *dev_out = nullptr;
    if (S->opt.direct_host_access && n > 0 && !large) {
        // Both ends of each range must lie in one page-locked mapping: a
        // buffer that starts in pinned memory and runs past it is staged.
        const void *vi = pinned_view(host_in, n * 2);
        const void *vo = vi ? (host_out == host_in ? vi : pinned_view(host_out, n * 2)) : nullptr;
        if (vi && vo) {
            direct = true;
            dev_in = (const uint16_t *)vi;
            dev_out = (uint16_t *)vo;
        }
    }
    // Large requests whose buffers kernels can reach (pinned host memory, or
    // pageable memory on a device that accesses it coherently; the same
    // buffer, or two that do not overlap) are repaired where they are.
    bool host_pass = false;
    if (large && n > 0 && host_pass_sms() > 0) {
        const uintptr_t x = (uintptr_t)host_in, y = (uintptr_t)host_out, bytes = (uintptr_t)n * 2u;
        const bool overlap = x != y && x < y + bytes && y < x + bytes;
        const void *vi = overlap ? nullptr : host_view(S->ctx, host_in, n * 2);
        const void *vo = vi ? (host_out == host_in ? vi : host_view(S->ctx, host_out, n * 2)) : nullptr;
        if (vi && vo) {
            host_pass = true;
            dev_in = (const uint16_t *)vi;
            dev_out = (uint16_t *)vo;
        }
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return UTF16_ECLOSED;
    Request r;
    r.ticket = S->next_ticket++;
    r.in = host_in;
    r.out = host_out;
    r.n = n;
    r.direct = direct;
    r.host_pass = host_pass;
    r.dev_in = dev_in;
    r.dev_out = dev_out;
    r.arrival_ns = arrival_ns > 0 ? arrival_ns : now_ns();
    if (n == 0) {
        r.first_bad = 0;
        complete_request(S, r, UTF16_OK);
        S->submitted++;
        S->cv_done.notify_all();
    } else {
        S->pending.push_back(r);
        S->submitted++;
        S->cv_sched.notify_all();
    }
    if (ticket) *ticket = r.ticket;
    return UTF16_OK;
}

int utf16_server_cancel(utf16_server *S, uint64_t ticket) {
    if (!S) return UTF16_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto it = S->pending.begin(); it != S->pending.end(); ++it)
        if (it->ticket == ticket) {
            Request x = *it;
            S->pending.erase(it);
            complete_request(S, x, UTF16_ECANCELED);
            S->cv_done.notify_all();
            return UTF16_OK;
        }
    return UTF16_EAGAIN;  // already admitted (or unknown): it will complete normally
}

int utf16_server_next(utf16_server *S, utf16_completion *c, int64_t timeout_us) {
    if (!S || !c) return UTF16_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto ready = [&] { return !S->completed.empty(); };
    if (timeout_us == 0) {
        if (!ready()) return UTF16_EAGAIN;
    } else {
        const int64_t t = timeout_us < 0 ? (int64_t)3600 * 1000000 : timeout_us;
        if (!S->cv_done.wait_for(lk, std::chrono::microseconds(t), ready)) return UTF16_ETIMEOUT;
    }
    const Request r = S->completed.front();
    S->completed.pop_front();
    c->ticket = r.ticket;
    c->first_bad = r.first_bad;
    c->status = r.status;
    c->n = r.n;
    c->arrival_ns = r.arrival_ns;
    c->done_ns = r.done_ns;
    return UTF16_OK;
}

int utf16_server_stats_get(utf16_server *S, utf16_server_stats *st) {
    if (!S || !st) return UTF16_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    *st = S->stats;
    st->pending = (int64_t)S->pending.size();
    st->inflight_batches = (int64_t)S->inflight.size();
    st->arena_used_bytes = S->ring->used();
    return UTF16_OK;
}

int utf16_server_destroy(utf16_server *S) {
    if (!S) return UTF16_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        S->cv_sched.notify_all();
        S->cv_inflight.notify_all();
    }
    if (S->scheduler.joinable()) S->scheduler.join();
    if (S->completer.joinable()) S->completer.join();
    for (BatchSlot &b : S->slots)
        if (b.stream) cudaStreamSynchronize(b.stream);
    for (BatchSlot &b : S->slots) {
        if (b.h_stage) cudaFreeHost(b.h_stage);
        if (b.ev_done) cudaEventDestroy(b.ev_done);
        if (b.stream) cudaStreamDestroy(b.stream);
    }
    if (S->arena) cudaFree(S->arena);
    cudaGetLastError();
    delete S;
    return UTF16_OK;
}

// ---------------------------------------------------------------- FIFO ring
struct utf16_arena {
    FifoRing ring;
    explicit utf16_arena(int64_t cap) : ring(cap) {}
};

int utf16_arena_create(int64_t capacity, utf16_arena **out) {
    if (capacity <= 0 || !out) return UTF16_EINVAL;
    *out = new utf16_arena(capacity);
    return UTF16_OK;
}
int64_t utf16_arena_alloc(utf16_arena *a, int64_t size) { return a ? a->ring.alloc(size) : -1; }
int utf16_arena_free_oldest(utf16_arena *a) { return (a && a->ring.free_oldest()) ? UTF16_OK : UTF16_EINVAL; }
int64_t utf16_arena_used(const utf16_arena *a) { return a ? a->ring.used() : -1; }
int utf16_arena_destroy(utf16_arena *a) {
    delete a;
    return UTF16_OK;
}

}  // extern "C"
