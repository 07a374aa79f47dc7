/*
 * utf16wf -- UTF-16 toWellFormed / isWellFormed on NVIDIA GB300 (sm_103a).
 *
 * C ABI of the shared library libutf16wf.so.  No C++ or framework types appear
 * in any signature: buffers are plain pointers, sizes are int64_t counts of
 * 16-bit code units, streams are CUDA stream handles.
 *
 * What is computed (Section 1 of "Fixing ill-formed UTF-16 strings with SIMD
 * instructions", Clausecker and Lemire):
 *   - a high surrogate is a unit in 0xD800-0xDBFF, a low surrogate a unit in
 *     0xDC00-0xDFFF;
 *   - a high surrogate not immediately followed by a low surrogate, and a low
 *     surrogate not immediately preceded by a high surrogate, is mismatched;
 *   - toWellFormed replaces every mismatched unit by U+FFFD (0xFFFD) and keeps
 *     every other unit, so the length never changes;
 *   - units before the first and after the last unit of a string are outside
 *     it (Section 3.1: an input that starts with a low or ends with a high
 *     surrogate has that unit replaced).  In a batch every string is on its
 *     own: a high surrogate that ends one string stays unpaired even when the
 *     next string starts with a low surrogate.
 *   - the first-error index is the index of the first unit that toWellFormed
 *     replaces, or n when the string is well formed (isWellFormed is
 *     first_bad == n).  The paper does not define an index; this one counts
 *     the unit itself, not the position of the Section 3.1 step-two flag
 *     (which is one unit late for a lone high surrogate, Fig. 3).
 *
 * Code units are native-order uint16_t values (no byte-order mark handling).
 *
 * Conventions for every entry point:
 *   - Pointers are DEVICE pointers unless the name or comment says host.  A
 *     buffer of code units must be 2-byte aligned; no other alignment is
 *     required (16-byte aligned buffers are fastest).
 *   - The caller owns every buffer.  The library never frees caller memory.
 *     It keeps a small per-device scratch area (one 32-byte slot per stream
 *     that has run a first-error computation, from a pool of 4096 slots) and,
 *     for the host-memory entry point, staging buffers; both live until
 *     process exit or utf16_release_device().
 *   - Calls are asynchronous on `stream` unless stated otherwise.  Argument
 *     errors are detected on the host before anything is launched and return
 *     a negative status; CUDA errors of the launch return UTF16_ECUDA.  Errors
 *     of the kernel itself surface at the next synchronising call, as in the
 *     CUDA runtime.
 *   - n == 0 (or an empty batch) is a valid no-op; first-error outputs are
 *     then 0.
 *   - `stream` may be NULL (the legacy default stream).  Calls that compute a
 *     first-error index on the same stream are ordered; calls on different
 *     streams use different scratch slots and may run concurrently.
 */
#ifndef UTF16WF_H
#define UTF16WF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *utf16_stream_t;

/* Status codes. */
#define UTF16_OK 0
#define UTF16_EINVAL (-1)   /* null pointer, negative size, misaligned buffer, bad offsets */
#define UTF16_EOVERLAP (-2) /* in and out overlap without being the same buffer */
#define UTF16_ECUDA (-3)    /* a CUDA call failed */
#define UTF16_ETIMEOUT (-4) /* a bounded wait gave up (serving queue) */
#define UTF16_ENOMEM (-5)   /* scratch slots, staging memory or serving budget exhausted */
#define UTF16_ECLOSED (-6)  /* the serving engine is shut down */
#define UTF16_EAGAIN (-7)   /* nothing ready yet (non-blocking poll) */
#define UTF16_ETOOBIG (-8)  /* input longer than the no-allocation entry point's stated maximum */
#define UTF16_ECANCELED (-9) /* serving request cancelled before admission */

/* Human-readable text of a status code (static storage, never NULL). */
const char *utf16_strerror(int code);

/*
 * toWellFormed, out of place (Section 1 rule; Section 3.1 string ends).
 *   in   [n] device, read.
 *   out  [n] device, written: out[i] = 0xFFFD where in[i] is mismatched,
 *        in[i] otherwise.  out == in is allowed (same as the in-place entry
 *        point); any other overlap returns UTF16_EOVERLAP.
 */
int utf16_to_well_formed(const uint16_t *in, uint16_t *out, int64_t n, utf16_stream_t stream);

/*
 * toWellFormed in place.  Only 16-byte blocks that contain a mismatched unit
 * are written; a well-formed string causes no stores at all (Section 3.1:
 * in-place operation omits the copy).  Safe without inter-block ordering
 * because replacing a mismatched unit by 0xFFFD never changes the verdict of
 * a neighbour.
 *   buf  [n] device, read and written.
 */
int utf16_to_well_formed_inplace(uint16_t *buf, int64_t n, utf16_stream_t stream);

/*
 * toWellFormed out of place (or in place when out == in) fused with the
 * first-error index in the same pass.
 *   first_bad  one int64_t, device or host pointer.  Device: written
 *              asynchronously in stream order.  Host: the call waits for the
 *              stream and returns with *first_bad set.
 */
int utf16_to_well_formed_first_bad(const uint16_t *in, uint16_t *out, int64_t n, int64_t *first_bad,
                                   utf16_stream_t stream);

/*
 * isWellFormed with the first-error index; reads the string, writes nothing
 * else.  Blocks stop early once a smaller error index is known.
 *   first_bad  one int64_t, device or host pointer (as above).  Set to the
 *              index of the first mismatched unit, or n if there is none.
 */
int utf16_is_well_formed(const uint16_t *in, int64_t n, int64_t *first_bad, utf16_stream_t stream);

/*
 * Full error report: the index of every unit that toWellFormed replaces.
 *   positions  [capacity] int64, DEVICE (may be NULL when capacity == 0):
 *              receives min(count, capacity) distinct indices, in no
 *              particular order (the GPU reserves room per warp with one
 *              atomic); when count > capacity, which indices are kept is
 *              unspecified.
 *   count      one int64_t, device or host pointer: the total number of
 *              mismatched units (host pointer: the call waits for the stream).
 */
int utf16_error_positions(const uint16_t *in, int64_t n, int64_t *positions, int64_t capacity, int64_t *count,
                          utf16_stream_t stream);

/*
 * Ragged batch forms.  String s is in[offsets[s] .. offsets[s+1]) for
 * s = 0 .. num_strings-1.
 *   offsets    [num_strings + 1] int64, DEVICE, non-decreasing, offsets[0] >= 0
 *              (it need not be 0).  The library reads the range from the
 *              device, so a call never synchronises with the host.  Offsets
 *              that decrease give unspecified (but memory-safe within
 *              [offsets[0], offsets[num_strings]) output, unless checked
 *              mode (utf16_set_checked) rejects them first.
 *   in, out    device buffers indexed by the offsets; only units in
 *              [offsets[0], offsets[num_strings]) are read or written.
 * Each string is repaired on its own: its first unit has no left neighbour
 * and its last unit no right neighbour.
 */
int utf16_to_well_formed_batch(const uint16_t *in, uint16_t *out, const int64_t *offsets, int64_t num_strings,
                               utf16_stream_t stream);
int utf16_to_well_formed_batch_inplace(uint16_t *buf, const int64_t *offsets, int64_t num_strings,
                                       utf16_stream_t stream);
/*
 *   first_bad  [num_strings] int64, DEVICE: first-error index of each string
 *              relative to its start, equal to its length when well formed.
 */
int utf16_is_well_formed_batch(const uint16_t *in, const int64_t *offsets, int64_t num_strings,
                               int64_t *first_bad, utf16_stream_t stream);

/*
 * Validates a ragged batch's offsets, which the batch entry points above
 * take on trust: *first_violation = the smallest i in [0, num_strings] with
 * offsets[0] < 0 (i = 0) or offsets[i] < offsets[i-1] (i > 0), or -1 when the
 * array is valid.  One read of the array (8 bytes per string).
 *   offsets          [num_strings + 1] int64, DEVICE, 8-byte aligned
 *   first_violation  host pointer: the call waits for the stream and returns
 *                    the value; device pointer: written in stream order
 * Returns UTF16_EINVAL for a null pointer or negative num_strings.
 */
int utf16_check_offsets(const int64_t *offsets, int64_t num_strings, int64_t *first_violation,
                        utf16_stream_t stream);

/*
 * Checked mode (process-wide; initially the value of the environment
 * variable UTF16WF_CHECKED, off when unset or 0).  When on, the three batch
 * entry points above run the utf16_check_offsets pass first and wait for it:
 * invalid offsets return UTF16_EINVAL with nothing launched.  The calls then
 * synchronise with the host, so inside a CUDA stream capture they return
 * UTF16_EINVAL.  The serving engine builds its own offsets and is not
 * affected.  utf16_set_checked returns UTF16_OK; utf16_get_checked 1 or 0.
 */
int utf16_set_checked(int on);
int utf16_get_checked(void);

/*
 * toWellFormed plus first-error index on HOST buffers.  Blocking: returns
 * when host_out holds the result.
 * When kernels can reach both buffers -- page-locked memory (cudaHostAlloc /
 * cudaHostRegister), or pageable memory on a device that accesses it
 * coherently (cudaDevAttrPageableMemoryAccess, e.g. over NVLink-C2C through
 * the host's page tables; environment UTF16WF_HOST_PAGEABLE_DIRECT=0 turns
 * this off) -- one pass of the fused kernel reads and writes them over the
 * host link directly.  Otherwise the string is cut into chunks that are
 * copied to the device, repaired and copied back on three library-owned
 * streams so that the two copy directions and the kernel overlap; each chunk
 * receives its outside neighbours from the host buffer, so the result is that
 * of the whole string (pageable buffers serialise the copies).
 *   host_in, host_out  [n] host; host_out == host_in is allowed.
 *   first_bad_host     one int64_t on the host, or NULL.
 */
int utf16_to_well_formed_host(const uint16_t *host_in, uint16_t *host_out, int64_t n, int64_t *first_bad_host);

/*
 * toWellFormed fused with the first-error index, allocating nothing.  The
 * paper has no counterpart: this exists for callers that cannot let a library
 * call cudaMalloc -- processes whose device memory is fully reserved by a
 * host framework or a fixed budget, pipelines that forbid allocation after
 * start-up, code that must not change the device's memory footprint.  Its
 * only scratch is a 256-byte array compiled into the library (one 32-byte
 * first-error slot), which every GPU that loads the library holds until the
 * process exits.
 *   in, out, n, first_bad, stream  as utf16_to_well_formed_first_bad (the
 *                                  output is identical).
 *   n must not exceed 2^40 units; longer inputs return UTF16_ETOOBIG.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before capturing a
 * stream into a CUDA graph.  Under CUDA's lazy module loading (the default)
 * that first call is also when the library's kernels and the array are loaded
 * onto the device, so the device footprint grows once, at that call, and never
 * again: a caller with a fixed footprint makes it at start-up (n == 1 will do).
 * The chunk width and data path follow the regular entry point's defaults
 * (2-vector chunks below 40,960 units per SM).  Every call shares the one array and keeps the
 * last call's contents, clearing what must start cleared in stream order:
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it and may return wrong first-error indices.
 */
int utf16_to_well_formed_first_bad_noalloc(const uint16_t *in, uint16_t *out, int64_t n, int64_t *first_bad,
                                           utf16_stream_t stream);

/*
 * Launch configuration of the current device.  The kernels are the same in
 * every configuration (results are identical); only speed changes.
 */
typedef struct {
    int single_variant;          /* 0: 128-bit loads; 1: 128-bit loads, next chunk requested before the
                                    current one is processed; 2: TMA bulk copies into a 4-stage
                                    shared-memory ring (16 KiB tiles); repair forms only */
    int single_units_per_thread; /* 16-byte vectors per thread per warp chunk: 2 or 4 (TMA uses 4); 0
                                    (default): 2 below 40,960 units per SM (about 6.2M units on 152
                                    SMs), 4 from there on */
    int single_blocks_per_sm;    /* persistent grid = SMs x this; 0 = as many as fit */
    int batch_units_per_thread;  /* batch chunk: 2 = 1,024 units, 4 = 2,048 units; 0 (default) = by form:
                                    1,024 out of place, 2,048 in place and for the per-string check */
    int batch_prefetch;          /* batch repair: 1 = next chunk requested before the current one is
                                    processed; 0 (default) */
    int batch_blocks_per_sm;     /* 0 = as many as fit */
    int check_variant;           /* read-only check (utf16_is_well_formed): 0, 1 or 2 as single_variant */
    int inplace_unit_stores;     /* in-place repair of single strings: 0 = store each 16-byte block that
                                    holds a replaced unit, 1 = store only the replaced units (2 bytes) */
    int inplace_variant;         /* in-place repair of single strings: 0, 1 or 2 as single_variant */
    int check_blocks_per_sm;     /* read-only check: persistent grid = SMs x this; 0 = as many as fit */
    int inplace_blocks_per_sm;   /* in-place repair of single strings: the same */
    int batch_check_prefetch;    /* per-string check of batches (utf16_is_well_formed_batch): 0 or 1 */
    int block_threads;           /* threads per block: 128, 256 or 512; 0 (default) = 256 for single strings,
                                    512 for batches.  The TMA data path always uses 256 */
    int vector_bytes;            /* bytes each lane loads at once in the batch kernels: 8, 16 or 32 (256-bit
                                    loads); 0 (default) = 32 for in-place batch repair, 16 for the other batch
                                    forms.  Single strings use 16 */
    int repair_variant;          /* out-of-place repair without the first-error index (utf16_to_well_formed,
                                    single strings): 0, 1 or 2 as single_variant; -1 (default) = single_variant.
                                    Its kernel keeps no first-error state, so its best data path can differ */
    int repair_units_per_thread; /* the same repair: 2 or 4; 0 (default) = single_units_per_thread */
    int repair_blocks_per_sm;    /* the same repair: persistent grid = SMs x this, 0 = as many as fit;
                                    -1 (default) = single_blocks_per_sm */
    int repair_block_threads;    /* threads per block of single strings, by form: the repair without the */
    int check_block_threads;     /* first-error index, the read-only check, in-place repair; 128, 256 or */
    int inplace_block_threads;   /* 512; 0 (default) = block_threads.  The TMA data path always uses 256 */
} utf16_config;

/* Default configuration of the current device (used where nothing is tuned). */
int utf16_get_config(utf16_config *cfg);
/* Replace the default configuration; clears all tuned entries.  Values out
 * of range return UTF16_EINVAL. */
int utf16_set_config(const utf16_config *cfg);

/*
 * Autotuner.  Times every candidate configuration (variant x units per thread
 * x blocks per SM) on the caller's own device buffers with CUDA events, on a
 * library stream: after one warm-up launch, three trials of `reps` launches
 * each, the fastest trial counting; synchronous.
 * The fastest is stored for the size bucket floor(log2(n)) of single strings
 * (utf16_autotune_single: out-of-place repair with first-error index; then
 * the data path, chunk width and grid of the out-of-place repair without it;
 * then the data path and grid of the read-only check, timed on the repaired
 * (well-formed) string in `out`, and of in-place repair, timed on copies of
 * `in`) or for
 * the bucket floor(log2(num_strings)) of batches (utf16_autotune_batch, the
 * out-of-place batch repair), and used by later calls in that bucket.
 *   out   scratch output of the same size as in (written).
 *   best  (optional, host) receives the chosen configuration.
 */
int utf16_autotune_single(const uint16_t *in, uint16_t *out, int64_t n, int reps, utf16_config *best);
int utf16_autotune_batch(const uint16_t *in, uint16_t *out, const int64_t *offsets, int64_t num_strings, int reps,
                         utf16_config *best);

/*
 * Autotuner without caller data, from a length histogram: the library makes
 * synthetic mixed text (mostly ASCII and other BMP text, about 8 % of cells
 * surrogate pairs and 1 % lone surrogates) and tunes on it.
 *   op 0  single strings: length_histogram[b] > 0 tunes bucket b on one
 *         string of 2^b units (at most 2^29; larger buckets take that result)
 *   op 1  batches: length_histogram[b] strings with lengths in [2^b, 2^(b+1))
 *         (bucket 0: 0 or 1 unit), shuffled into one batch of at most 2^29
 *         units (counts scaled down in proportion), tuned for that batch's
 *         string-count bucket and the histogram's own total
 *   buckets  1..64 entries, none negative.
 * Allocates and frees its own device buffers; synchronous.
 */
int utf16_autotune(int op, const int64_t *length_histogram, int buckets);

/*
 * Tuned entries (what the autotuner stored), for saving and restoring a
 * tuning cache.  op: 0 = single strings (bucket = floor(log2(n))), 1 =
 * batches (bucket = floor(log2(num_strings))); bucket 0..63.
 * utf16_get_tuned returns UTF16_EAGAIN when nothing is tuned for the bucket.
 */
int utf16_get_tuned(int op, int bucket, utf16_config *cfg);
int utf16_set_tuned(int op, int bucket, const utf16_config *cfg);

/*
 * UTF16_ETIMEOUT if a kernel of this device gave up a bounded wait (a TMA
 * copy that did not complete within one second) since the last call, which
 * means its outputs are not valid; UTF16_OK otherwise.  Synchronises the
 * device.
 */
int utf16_check_device_errors(void);

/*
 * Self-test of the kernels' bounded waits: one GPU thread waits on a barrier
 * that nothing completes, with the TMA kernel's wait routine and a limit of
 * `limit_ns` (1 .. 2e9).  Returns UTF16_ETIMEOUT when the wait gave up as it
 * must (and the device-error flag is then set, as after a real timeout);
 * synchronous.  Nothing faults and nothing hangs: the wait is bounded.
 */
int utf16_selftest_bounded_wait(int64_t limit_ns);

/* ===================================================================== *
 * Serving: continuous batching of repair requests (host strings).
 *
 * Not in the paper; the paper's function repairs one string at a time.
 * Requests arrive through utf16_server_submit at any time.  A scheduler
 * thread admits them in arrival order against a device arena of
 * `hbm_budget_bytes` (a FIFO ring) and launches whatever has arrived as one
 * ragged batch as soon as one of `max_inflight_batches` batch slots is free
 * -- it never waits for a batch to fill.  Each batch is copied in, repaired
 * in place with the per-string first-error index, and copied out on its
 * slot's stream; batches of different slots overlap, so transfers of one
 * batch overlap the kernels of others.  Small requests (< small_request_bytes)
 * are packed through a pinned staging buffer per slot.  A larger request
 * whose buffers kernels can reach (pinned host memory, or pageable memory on a
 * device that accesses it coherently; one buffer, or two that do not
 * overlap) is repaired where it is, by one fused pass of the single-string
 * kernel over the host link on a few SMs (8 by default; environment
 * UTF16WF_SERVE_HOST_PASS_SMS, 0 = off); other large ones are copied straight
 * from and to the caller's buffers (pageable ones synchronously by the CUDA
 * runtime).  With direct_host_access, small
 * requests in pinned buffers are read and written by the GPU directly (one
 * gather and one scatter kernel per batch), which keeps the CPU out of the
 * data path.  Each string of a batch is repaired on
 * its own, so a request's result is the same alone and in any mix.
 * ===================================================================== */
typedef struct utf16_server utf16_server;

typedef struct {
    int64_t hbm_budget_bytes;     /* device arena for admitted batches (>= 1 MiB) */
    int64_t max_batch_strings;    /* strings per launched batch (requests count at most 2 each) */
    int64_t max_batch_bytes;      /* input bytes packed into one launched batch; a longer request is
                                     launched as a batch of its own */
    int max_inflight_batches;     /* batches between admission and completion (1..64) */
    int64_t staging_bytes;        /* pinned host staging per batch slot */
    int64_t small_request_bytes;  /* requests below this size are packed through staging */
    int64_t inject_fail_mod;      /* testing: 0 = off; k > 0 = the admission of every request whose
                                     ticket % k == k - 1 fails with UTF16_ENOMEM (host-side fault
                                     injection; other requests are unaffected) */
    int direct_host_access;       /* 1: a small request whose host buffers are pinned (page-locked, mapped) is
                                     copied in and out by the GPU itself, in 8 KiB pieces (no CPU copies; each
                                     submit then queries the buffers' attributes); 0 (default): staged */
    int64_t inject_copy_fail_mod; /* testing: 0 = off; k > 0 = a copy step of every k-th launched batch (launch
                                     number % k == k - 1) fails: the copies are not issued, the batch's later work
                                     neither, and its requests complete with UTF16_ECUDA (host-side fault injection,
                                     nothing faults on the GPU) */
    int inject_copy_fail_step;    /* the failing step: 0 = the host-to-device copies (no output is touched), 1 = the
                                     device-to-host copies (outputs the engine copies back stay untouched; requests
                                     the GPU writes itself -- host passes, direct access -- may hold their result) */
} utf16_server_options;

typedef struct {
    uint64_t ticket;
    int64_t first_bad;   /* first-error index of the request's string (n if well formed) */
    int64_t n;
    int64_t arrival_ns;  /* utf16_server_clock_ns() time the request counts from */
    int64_t done_ns;     /* time its result was in the caller's buffer */
    int status;          /* UTF16_OK, UTF16_ENOMEM (rejected), UTF16_ECANCELED, UTF16_ECLOSED, UTF16_ECUDA */
} utf16_completion;

typedef struct {
    int64_t batches, completed, rejected, units;
    int64_t max_batch_requests;
    int64_t pending, inflight_batches, arena_used_bytes;
} utf16_server_stats;

/* Defaults: 4 GiB budget, 65536 strings / 16 MiB packed per batch, 8 slots, 32 MiB staging per slot,
 * 256 KiB small limit. */
int utf16_server_default_options(utf16_server_options *opt);
/* Allocates the arena, staging and streams on the current device; starts two host threads. */
int utf16_server_create(const utf16_server_options *opt, utf16_server **server);
/* Monotonic clock (ns) the server's timestamps use. */
int64_t utf16_server_clock_ns(void);
/*
 * Queue one string.  host_in / host_out: [n] host buffers (may be the same),
 * valid until the request completes.  arrival_ns: the time latency counts
 * from (utf16_server_clock_ns(); 0 = now).  Non-blocking.  A request that
 * cannot fit an empty arena, batch or staging buffer returns UTF16_ENOMEM.
 */
int utf16_server_submit(utf16_server *server, const uint16_t *host_in, uint16_t *host_out, int64_t n,
                        int64_t arrival_ns, uint64_t *ticket);
/* Remove a request that has not been admitted yet (completes with UTF16_ECANCELED); UTF16_EAGAIN if it has. */
int utf16_server_cancel(utf16_server *server, uint64_t ticket);
/* Next completion (any order of tickets).  timeout_us: 0 = poll (UTF16_EAGAIN), < 0 = up to an hour,
 * else the bound (UTF16_ETIMEOUT). */
int utf16_server_next(utf16_server *server, utf16_completion *completion, int64_t timeout_us);
int utf16_server_stats_get(utf16_server *server, utf16_server_stats *stats);
/* Stops admission, completes pending requests with UTF16_ECLOSED, waits for in-flight batches, frees all. */
int utf16_server_destroy(utf16_server *server);

/*
 * Load replay (benchmarking): submit `count` requests with exponential
 * inter-arrival times at `rate_per_s` (xoshiro256** seeded with `seed`;
 * rate <= 0: all at once), each latency counted from its scheduled arrival,
 * and wait for all.  Outputs per request index: latency_s (done - arrival)
 * and first_bad (status < 0 stored as the status).  Blocking.
 *   utf16_server_replay  through a serving engine (continuous batching);
 *   utf16_plain_replay   one plain launch per request in arrival order:
 *                        H2D, fused repair + first-error kernel, D2H, wait.
 *   utf16_plain_replay_streams  the same plain launches pipelined: `streams`
 *                        (1..64) host threads, each with its own stream and
 *                        device buffer, take the requests in arrival order,
 *                        so up to `streams` requests are in flight at once
 *                        (what overlap alone gives, without batching).
 */
int utf16_server_replay(utf16_server *server, const uint16_t *const *inputs, uint16_t *const *outputs,
                        const int64_t *lengths, int64_t count, double rate_per_s, uint64_t seed, double *latency_s,
                        int64_t *first_bad);
int utf16_plain_replay(const uint16_t *const *inputs, uint16_t *const *outputs, const int64_t *lengths, int64_t count,
                       double rate_per_s, uint64_t seed, double *latency_s, int64_t *first_bad);
int utf16_plain_replay_streams(const uint16_t *const *inputs, uint16_t *const *outputs, const int64_t *lengths,
                               int64_t count, double rate_per_s, uint64_t seed, int streams, double *latency_s,
                               int64_t *first_bad);

/*
 * FIFO ring allocator used for serving admission, exposed for reuse and for
 * testing: offsets in [0, capacity); blocks are freed oldest first.
 */
typedef struct utf16_arena utf16_arena;
int utf16_arena_create(int64_t capacity, utf16_arena **arena);
int64_t utf16_arena_alloc(utf16_arena *arena, int64_t size); /* offset, or -1 if it does not fit */
int utf16_arena_free_oldest(utf16_arena *arena);
int64_t utf16_arena_used(const utf16_arena *arena);
int utf16_arena_destroy(utf16_arena *arena);

/*
 * Prepare the current device (SM count, occupancy, scratch pool, launch
 * tuning).  Called implicitly by the first entry point that needs it; call it
 * explicitly before capturing a stream into a CUDA graph, since it allocates.
 */
int utf16_init_device(void);

/* Free the current device's scratch and staging memory (after a device sync). */
int utf16_release_device(void);

#ifdef __cplusplus
}
#endif

#endif /* UTF16WF_H */
