/*
 * sinet.h - C ABI of the GB300 session discrimination + histogram library.
 *
 * The method (arXiv 2106.12863):
 *   - Algorithm 1 ("session ingoing/outgoing discrimination"): for a CIDR
 *     entry Y/Z and an address X, SB = bitmask(X, Z), CB = bitmask(Y, Z),
 *     and a zero SB - CB is a match. bitmask keeps the top Z bits of the
 *     32-bit address (Fig. 4). The input is a CIDR list; an address is inside
 *     when any entry matches.
 *   - Section 5 ("Pairwise Reduction Pattern with GPU", "Merge Scatter
 *     Pattern with CPU"): the discriminated sessions are histogrammed into
 *     <timestamp, count> and <timestamp, bytes> maps at millisecond
 *     granularity (86,400,000 bins per day), one per direction.
 *
 * Conventions shared by every entry point:
 *   - Addresses are uint32 with the first octet most significant
 *     (192.168.1.5 == 0xC0A80105).
 *   - Records are structure-of-arrays: ts_ms uint64[n], src uint32[n],
 *     dst uint32[n], bytes uint32[n] (Table 1 fields capture_time,
 *     source_ip, destination_ip, bytes). Record and output pointers are
 *     DEVICE pointers owned by the caller, each aligned to its element size;
 *     16-byte alignment lets the kernels use 128-bit loads.
 *   - class of a record = src_in | dst_in << 1: 0 neither, 1 source inside
 *     (outgoing), 2 destination inside (ingoing), 3 both.
 *   - Direction index d: 0 = outgoing (egress), 1 = ingoing (ingress).
 *   - Calls are asynchronous on `stream` (NULL = the legacy default stream).
 *     SINET_OK means validated and enqueued. Host-detectable errors return
 *     before anything is launched. Device-side failures (a bounded wait that
 *     ran out, a failed bounds check in a checked build) are latched in a
 *     per-device status word read by sinet_device_status().
 *   - Nothing aborts, prints or traps. Library-owned scratch comes from
 *     stream-ordered cudaMallocAsync and is released on the same stream.
 *   - Limits: n <= 2^40 records, 1 <= n_bins <= 2^31 - 1, bin width >= 1,
 *     t0 + n_bins * bin_width must fit in uint64, prefix length <= 32.
 */
#ifndef SINET_H
#define SINET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (the runtime's type is this same pointer). */
typedef struct CUstream_st *sinet_stream_t;

typedef enum {
    SINET_OK = 0,
    SINET_ERR_INVALID_ARG = 1,     /* bad pointer, size, length or parameter */
    SINET_ERR_CUDA = 2,            /* a CUDA runtime call failed; see sinet_last_cuda_error() */
    SINET_ERR_OOM = 3,             /* device allocation failed */
    SINET_ERR_BUDGET = 4,          /* a request does not fit the caller's memory budget */
    SINET_ERR_TIMEOUT = 5,         /* a bounded device-side wait ran out */
    SINET_ERR_TABLE_TOO_LARGE = 6, /* more prefixes than the table format holds */
    SINET_ERR_DEVICE_CHECK = 7,    /* a device-side bounds check failed (checked builds) */
    SINET_ERR_UNSUPPORTED = 8      /* option combination not available */
} sinet_status;

/* How the histogram update is carried out. All give identical results. */
typedef enum {
    SINET_STRAT_AUTO = 0,          /* autotuner / heuristics choose */
    SINET_STRAT_GLOBAL_ATOMIC = 1, /* warp match + reduce, then global atomics */
    SINET_STRAT_PRIV_TILE = 2,     /* shared-memory bin tile per chunk (time-sorted input) */
    SINET_STRAT_SORT_REDUCE = 3,   /* plain path: discriminate, radix sort, reduce by key */
    SINET_STRAT_SMEM_FULL = 4,     /* whole histogram privatised in shared memory (small n_bins) */
    SINET_STRAT_ATOMIC_NOAGG = 5,  /* global atomics without warp aggregation */
    SINET_STRAT_ATOMIC_CELL = 6,   /* GLOBAL_ATOMIC into a library scratch of one 32-byte cell per
                                      bin (both directions' count and byte sum in one DRAM sector),
                                      then expanded into the output arrays: for unsorted input over
                                      histograms far larger than L2 */
    SINET_STRAT_OWNER = 7,         /* owner computes, for time-sorted input: each CTA owns a block
                                      of bin ranges, takes the run of records that falls into each
                                      range (binary search on ts) through a circular shared-memory
                                      tile that also spans half a range on either side, and stores
                                      every bin once with plain stores, so the outputs need no
                                      zeroing and see no read-modify-write. Exact for any input:
                                      records out of order by more than the halo, and runs longer
                                      than 32,767 records, are added by a second kernel with global
                                      reductions. tile_bins sets the tile (rounded down to a power
                                      of two, at least 16; ranges are half of it). Scratch, stream-
                                      ordered: 8 bytes per range, 4 per CTA, 32 per queued item
                                      (at most one per range plus one per 32,767 records). At most
                                      512 threads per block. */
    SINET_STRAT_PARTITION = 8      /* hot/cold partition, for unsorted input over histograms far
                                      larger than L2 (Section 5's map-reduce with the reduction
                                      kept on chip): a strided sample of about n / 4,096 records
                                      ranks the bins; the most sampled ones (up to 16,384 slots,
                                      as shared memory allows) are summed in shared memory by
                                      every CTA; every other routed update is appended as an
                                      8-byte (bin, direction, bytes) entry to a page of its
                                      bin range, and a cooperative second kernel sorts the pages
                                      by owner CTA in place and has each CTA sum its own bins in
                                      shared memory and store each of them once. The outputs
                                      need no zeroing and see no read-modify-write. tile_bins, a
                                      power of two, sets the bins per range (default 2^19; raised
                                      until there are at most 256 ranges; at most 2^20).
                                      sinet_discriminate_histogram only, no watch list; at most
                                      2^32 - 4,096 routed updates and 2^28 bins. Scratch, stream-
                                      ordered: 16 KB pages of 2,048 entries, namely a region
                                      per CTA and range (pages for an even share of 30 % of the
                                      routed updates, plus one, at most 16) and a shared pool for
                                      every routed update (8 bytes each) plus two pages per CTA
                                      and range; about 320 bytes of bookkeeping per page, and
                                      64 MB at most for the sample. The second kernel is a
                                      cooperative launch (one CTA per SM, all resident). */
} sinet_strategy;

/* How membership is looked up. Both are exact. */
typedef enum {
    SINET_LOOKUP_AUTO = 0,
    SINET_LOOKUP_INTERVAL = 1, /* merged disjoint intervals + top-k-bit direct index */
    SINET_LOOKUP_PML = 2       /* per-mask-length binary search over canonical networks */
} sinet_lookup;

/* Direction bits used in sinet_hist_params.policy. */
#define SINET_DIR_OUT 1u
#define SINET_DIR_IN 2u

/* Input hints (sinet_hist_params.hints). */
#define SINET_HINT_TIME_SORTED 1u  /* records are (nearly) sorted by ts */
#define SINET_HINT_TUNE 2u         /* strategy AUTO, not accumulating: the first call of an input class
                                      (lookup form, sortedness, log2 of n_bins and of n, unit width,
                                      two-direction policy) times every candidate strategy on its own
                                      input, synchronising the stream, and the fastest is cached for
                                      the process; later AUTO calls of the class run it directly */

typedef struct sinet_prefix_table sinet_prefix_table;

typedef struct {
    uint64_t t0_ms;        /* window start */
    uint64_t bin_width_ms; /* >= 1 */
    uint64_t n_bins;       /* window = [t0, t0 + n_bins * bin_width) */
    uint8_t policy[4];     /* class -> direction bits; exclusive default {0, OUT, IN, 0} */
    int32_t accumulate;    /* 0: outputs and stats are overwritten; 1: added to */
    int32_t strategy;      /* sinet_strategy */
    int32_t lookup;        /* sinet_lookup */
    uint32_t hints;        /* SINET_HINT_* */
    uint32_t tile_bins;    /* PRIV_TILE / OWNER bins per direction per tile (0 = default) */
    uint32_t block_threads;/* threads per CTA (0 = default) */
    const struct sinet_prefix_table *watch; /* optional watch list (the blocklist views of Section 6):
                              only records whose src or dst is in it are classified and binned,
                              every other record counts in stats[6]. Runs with GLOBAL_ATOMIC,
                              ATOMIC_NOAGG and ATOMIC_CELL (AUTO picks among them);
                              sinet_discriminate_histogram only. NULL = no filter. */
} sinet_hist_params;

/*
 * Histogram outputs, caller-owned device arrays:
 *   count[d]: uint32[n_bins]  (sessions per bin; wraps modulo 2^32 when accumulating)
 *   bytes[d]: uint64[n_bins]  (sum of the records' bytes field)
 *   stats:    uint64[8]       (records per class [0..3], out-of-window records per
 *                              routed direction [4..5], records left out by the watch
 *                              list [6]; [7]: its low 32 bits carry the device-side
 *                              status of sinet_discriminate_histogram_noalloc, which
 *                              clears them at every call; otherwise reserved)
 * A record routed to direction d whose ts lies outside the window is not
 * binned; it is counted in stats[4 + d].
 */
typedef struct {
    uint32_t *count[2];
    uint64_t *bytes[2];
    uint64_t *stats;
} sinet_hist_out;

/* sinet_prefix_table (declared above): opaque, library-owned, device-resident compiled CIDR list. */

/* Library version, e.g. 0x000100 for 0.1.0. */
uint32_t sinet_version(void);

/* Human-readable name of a status code (static string). */
const char *sinet_status_string(sinet_status s);

/* The last CUDA error code seen by this thread (0 if none). */
int sinet_last_cuda_error(void);

/*
 * Parse "a.b.c.d/z" (or "a.b.c.d", meaning /32) into net and len. Host only.
 * The CIDR notation Y.Y.Y.Y/Z of Algorithm 1. Host bits are kept as written.
 * Returns SINET_ERR_INVALID_ARG on malformed text or z > 32.
 */
sinet_status sinet_parse_cidr(const char *text, uint32_t *net, uint8_t *len);

/*
 * Compile a CIDR list on the host (no CUDA call) and report the derived
 * structures. Entries are canonicalised (net &= bitmask(len), the CB of
 * Algorithm 1), deduplicated and grouped by mask length; the union of all
 * entries is also emitted as sorted, disjoint, non-adjacent closed intervals
 * [lo, hi], with a direct index over the top `index_bits` address bits:
 * index[b] = first interval whose hi >= b << (32 - index_bits); the interval
 * that can hold an address of bucket b is among index[b] .. index[b + 1].
 *
 *   h_net, h_len  host arrays of n entries (len <= 32)
 *   index_bits    0..20 (0 = choose: the fewest bits, >= 6, whose buckets hold
 *                 at most four candidate intervals, within a shared-memory budget)
 *   nets_by_len   out, capacity n: canonical unique networks, ascending length,
 *                 sorted within each length (may be NULL)
 *   len_offset    out, uint32[34]: length L occupies [len_offset[L], len_offset[L+1])
 *   iv_lo, iv_hi  out, capacity n: the intervals (may be NULL)
 *   index         out, capacity 2^index_bits + 1 (may be NULL)
 *   counts        out, uint32[4]: unique entries, intervals, index bits used,
 *                 largest candidate range of a bucket
 * Returns SINET_ERR_INVALID_ARG for a length > 32, a NULL required pointer,
 * or index_bits > 20; SINET_ERR_TABLE_TOO_LARGE for n > 2^24.
 */
sinet_status sinet_compile_prefix_table(const uint32_t *h_net, const uint8_t *h_len, uint32_t n,
                                        uint32_t index_bits, uint32_t *nets_by_len,
                                        uint32_t *len_offset, uint32_t *iv_lo, uint32_t *iv_hi,
                                        uint32_t *index, uint32_t *counts);

/*
 * The device image of a compiled CIDR list, serialised on the host (no CUDA
 * call), for inspection and tests. layout (uint32[16]) receives: toggle
 * blocks offset, bucket descriptor offset, descriptor bits, bytes staged for
 * the toggle form, per-length networks offset, group table offset, groups,
 * bytes staged for the per-length form, global lo/hi/index offsets, index
 * bits, intervals, most toggle blocks of one bucket, and whether each form
 * fits shared memory. *bytes receives the image size; image (capacity bytes,
 * may be NULL to query the size) receives the image.
 */
sinet_status sinet_prefix_table_image(const uint32_t *h_net, const uint8_t *h_len, uint32_t n,
                                      uint8_t *image, size_t capacity, uint32_t *layout,
                                      size_t *bytes);

/*
 * Compile a CIDR list (as sinet_compile_prefix_table) and upload it to the
 * current device on `stream`. The table is owned by the library until
 * sinet_destroy_prefix_table. An empty list (n == 0) is valid: nothing is
 * inside. h_net/h_len are host arrays and are not retained.
 */
sinet_status sinet_build_prefix_table(const uint32_t *h_net, const uint8_t *h_len, uint32_t n,
                                      sinet_stream_t stream, sinet_prefix_table **out);

/* Free a table (synchronises the device it lives on). NULL is a no-op. */
sinet_status sinet_destroy_prefix_table(sinet_prefix_table *t);

/*
 * Algorithm 1 per record: class[i] = in(src[i]) | in(dst[i]) << 1.
 *   d_class         device uint8[n], may be NULL (counts only)
 *   d_class_counts  device uint64[4], overwritten with records per class
 *   lookup          sinet_lookup
 * n == 0 writes zero counts.
 */
sinet_status sinet_discriminate(const sinet_prefix_table *t, const uint32_t *d_src,
                                const uint32_t *d_dst, uint64_t n, uint8_t *d_class,
                                uint64_t *d_class_counts, int32_t lookup, sinet_stream_t stream);

/*
 * Histogram of already-classified records (Section 5's map-reduce step):
 * every record routed by p->policy[class] to direction d lands in bin
 * (ts - t0) / w of count[d] / bytes[d], or in stats[4 + d] when outside the
 * window. stats[0..3] count the classes seen. Classes must be 0..3
 * (values above 3 use their low two bits).
 */
sinet_status sinet_histogram(const uint64_t *d_ts, const uint32_t *d_bytes, const uint8_t *d_class,
                             uint64_t n, const sinet_hist_params *p, const sinet_hist_out *o,
                             sinet_stream_t stream);

/*
 * The binning step of Section 5 alone: d_bin[i] = (ts[i] - t0) / w for a
 * record inside the window [t0, t0 + n_bins * w), else 0xFFFFFFFF. The same
 * device division (an invariant-divisor multiply) as every histogram kernel.
 *   d_ts   device uint64[n]; d_bin device uint32[n] (caller-owned)
 * Parameters are checked as for the histogram (w >= 1, 1 <= n_bins < 2^31,
 * t0 + n_bins * w within uint64); SINET_ERR_INVALID_ARG otherwise.
 */
sinet_status sinet_bin(const uint64_t *d_ts, uint64_t n, uint64_t t0_ms, uint64_t bin_width_ms,
                       uint64_t n_bins, uint32_t *d_bin, sinet_stream_t stream);

/*
 * Fused Algorithm 1 + histogram in one pass over the records (the hot path).
 * p->strategy selects the update scheme (SINET_STRAT_SORT_REDUCE runs the
 * plain discriminate -> radix sort -> reduce-by-key path). Output as in
 * sinet_histogram.
 */
sinet_status sinet_discriminate_histogram(const sinet_prefix_table *t, const uint64_t *d_ts,
                                          const uint32_t *d_src, const uint32_t *d_dst,
                                          const uint32_t *d_bytes, uint64_t n,
                                          const sinet_hist_params *p, const sinet_hist_out *o,
                                          sinet_stream_t stream);

/*
 * Allocation-free form of sinet_discriminate_histogram. The paper has no
 * counterpart: it exists for callers that cannot allocate device memory on
 * the call path (a host application whose own memory manager owns every
 * device allocation, or a latency-bound loop where an allocator call could
 * synchronise the device or fail under fragmentation).
 *
 * It always runs the plain path (discriminate, radix sort, reduce by key;
 * p->strategy is ignored) with its scratch in a fixed 32 MiB device array
 * that is part of the library image: about 16.5 bytes per routed record,
 * so a little over 2 M records when every class routes to at most one
 * direction, about half that when a class routes to both. Larger inputs
 * return SINET_ERR_BUDGET before anything is launched. The call itself makes
 * no cudaMalloc/cudaFree or other allocating call; the prefix table is an
 * input and must have been built beforehand (sinet_build_prefix_table does
 * allocate).
 *
 * The first call on a device looks up that device's copy of the array (once,
 * with the device current); make that first call before any stream capture.
 * Every call on a device shares the one array, and calls that overlap on the
 * GPU (different streams, no ordering between them) race on it: order them.
 * The array keeps the previous call's contents; the call clears what must
 * start at zero itself. A device-side failure (a bounded wait that ran out)
 * is latched into the low 32 bits of stats[7] as a sinet_status code; every
 * call clears those 32 bits first (also when accumulating), so they report
 * this call only.
 * Other arguments, outputs and errors as in sinet_discriminate_histogram.
 */
sinet_status sinet_discriminate_histogram_noalloc(const sinet_prefix_table *t, const uint64_t *d_ts,
                                                  const uint32_t *d_src, const uint32_t *d_dst,
                                                  const uint32_t *d_bytes, uint64_t n,
                                                  const sinet_hist_params *p,
                                                  const sinet_hist_out *o, sinet_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched persistent launch (Section 4's coordinated batches: many chunks,
 * each discriminated and reduced, their outputs kept apart).
 *
 * A batch is a fixed set of independent slices, each with its own records,
 * prefix table, window, bin width, class policy and outputs. One launch of
 * one persistent kernel processes all of them: its CTAs pull (slice, chunk)
 * work items from a device counter, restage a slice's table into shared
 * memory when it differs from the one they hold, and update the slice's
 * histogram with the strategy chosen for it. The launch (a zeroing kernel
 * for non-accumulating slices, then the batch kernel) is captured once as a
 * CUDA graph at creation; sinet_batch_run replays it.
 */
typedef struct {
    const uint64_t *ts;               /* device records, as in sinet_discriminate_histogram */
    const uint32_t *src;
    const uint32_t *dst;
    const uint32_t *bytes;
    uint64_t n;
    const sinet_prefix_table *table;  /* must outlive the batch */
    sinet_hist_params params;         /* strategy: AUTO, GLOBAL_ATOMIC, ATOMIC_NOAGG, SMEM_FULL or
                                         SORT_REDUCE (the plain path, run as its own chain of
                                         kernels after the persistent kernel in the same graph,
                                         with scratch allocated at creation); lookup: AUTO or
                                         INTERVAL; hints, tile_bins and block_threads are ignored */
    sinet_hist_out out;               /* device outputs; must outlive the batch */
    const uint32_t *ready;            /* optional device word: when non-NULL the slice's work
                                         items wait until it equals ready_value, so its records
                                         can still be landing (a copy on another stream that ends
                                         by writing the word) when the launch starts. A wait is
                                         bounded (sinet_batch_set_wait); an item whose wait runs
                                         out is left out and SINET_ERR_TIMEOUT is latched in the
                                         device status word. */
    uint32_t ready_value;
} sinet_batch_slice;

/* Flags of sinet_batch_create. */
#define SINET_BATCH_AUTOTUNE 1u /* time the candidate strategies of AUTO slices (see below) */

typedef struct sinet_batch sinet_batch;

/*
 * Validate and plan n_slices slices (1 <= n_slices <= 65,536), upload their
 * descriptors and capture the launch. Slices with strategy AUTO get one from
 * the autotuner: slices are grouped into classes (lookup form, whether the
 * histogram fits a shared-memory tile, log2 of n_bins and of n, unit bin
 * width, both-direction policy); with SINET_BATCH_AUTOTUNE, each class not
 * yet in the process-wide cache is tuned by timing every candidate strategy
 * on its largest slice (its first 8 M records at most, into scratch outputs:
 * the slice's own outputs are not touched). The candidates are the batch
 * kernel's schemes (warp combining, plain atomics, the whole-histogram tile
 * when it fits), each run as enough copies to keep every CTA busy, and the
 * plain path (sort + reduce by key), run as its own chain; the fastest per record is cached and, if the environment
 * variable SINET_AUTOTUNE_CACHE names a file, appended to it as a line
 * "class strategy ns_per_record" (the file is read on first use). Without the flag a class absent from the
 * cache takes a fixed rule. Tuning runs on `stream` and synchronises it.
 * The records, tables and outputs are referenced, not copied: they must
 * stay valid, and the records unchanged between runs only if the caller
 * wants the same result. Returns SINET_ERR_INVALID_ARG for a NULL slice
 * array, table or output, misaligned pointers or bad params (as
 * sinet_discriminate_histogram), SINET_ERR_UNSUPPORTED for a strategy or
 * lookup the batch kernel does not run, or SMEM_FULL for a histogram that
 * does not fit a tile.
 */
sinet_status sinet_batch_create(const sinet_batch_slice *slices, uint32_t n_slices, uint32_t flags,
                                sinet_stream_t stream, sinet_batch **out);

/* Enqueue one run of the batch on `stream` (a graph launch). Non-accumulating
 * slices' outputs are zeroed first; accumulating slices are added to. */
sinet_status sinet_batch_run(sinet_batch *b, sinet_stream_t stream);

/* Bound, in nanoseconds of the GPU's global timer, of a work item's wait on
 * its slice's ready word (default 2 s). Synchronous. */
sinet_status sinet_batch_set_wait(sinet_batch *b, uint64_t wait_ns);

/* The strategy (sinet_strategy) the batch runs for slice i, after tuning. */
sinet_status sinet_batch_strategy(const sinet_batch *b, uint32_t i, int32_t *strategy);

/* Work items and records of the batch (either pointer may be NULL). */
sinet_status sinet_batch_info(const sinet_batch *b, uint64_t *work_items, uint64_t *records);

/* Synchronise the device, then free the batch (NULL is a no-op). */
sinet_status sinet_batch_destroy(sinet_batch *b);

/* ------------------------------------------------------------------------
 * Serving loop with continuous batching (Section 4's bounded work queue:
 * chunks are queued by a producer and each is to be processed within a
 * bounded time).
 *
 * A server owns, for each tenant, a prefix table reference, histogram
 * parameters and a RESIDENT histogram in device memory that every request of
 * the tenant accumulates into. Requests carry host records. A worker thread
 * admits queued requests in arrival order while the in-flight budget (a
 * device arena holding the admitted requests' records) has room, copies their
 * records to the device on a copy stream while the previous launch runs, and
 * then starts one batched launch (the kernel of sinet_batch_run) over every
 * admitted request whose copy has been issued, up to max_requests_per_launch.
 * A request is done when its launch has completed; its arena space is then
 * reused.
 */
typedef struct {
    const sinet_prefix_table *table; /* must outlive the server */
    sinet_hist_params params;        /* window, width, bins, policy; strategy AUTO, GLOBAL_ATOMIC,
                                        ATOMIC_NOAGG or SMEM_FULL (SORT_REDUCE is refused:
                                        requests share launches of the batch kernel);
                                        accumulate is implied */
} sinet_tenant;

typedef struct {
    uint64_t inflight_budget_bytes;   /* device arena for admitted requests' records (>= 1 MiB) */
    uint32_t max_requests_per_launch; /* requests one launch takes, 1..4096 */
    uint32_t max_queued;              /* submitted, not yet done requests; beyond it submit
                                         returns SINET_ERR_BUDGET */
} sinet_server_config;

typedef struct {
    uint64_t n;          /* records */
    uint64_t launch;     /* sequence number of the launch that processed it */
    uint64_t latency_ns; /* from submit to the host seeing its launch complete */
} sinet_request_info;

typedef struct {
    uint64_t requests_done;
    uint64_t records_done;
    uint64_t launches;
    uint64_t p50_latency_ns; /* over requests done since the last reset */
    uint64_t p99_latency_ns;
    uint64_t max_latency_ns;
    uint64_t busy_ns;        /* host-observed time with a launch in flight */
} sinet_server_counters;

typedef struct sinet_server sinet_server;

/* Create a server on the current device: allocates the tenants' resident
 * histograms (zeroed; 24 bytes per bin) and the arena, captures the launch,
 * and starts the worker. SINET_ERR_INVALID_ARG for bad tenants or config
 * (checked as in sinet_batch_create), SINET_ERR_OOM if device memory runs out. */
sinet_status sinet_server_create(const sinet_server_config *cfg, const sinet_tenant *tenants,
                                 uint32_t n_tenants, sinet_server **out);

/* Queue a request of n records (host pointers, each aligned to its element
 * size; pinned memory lets the copy overlap). The buffers must stay valid and
 * unchanged until the request is done. Returns SINET_ERR_BUDGET, queueing
 * nothing, if 20 n bytes (plus alignment) exceed the whole arena or
 * max_queued requests are outstanding; *ticket identifies the request. */
sinet_status sinet_server_submit(sinet_server *s, uint32_t tenant, const uint64_t *h_ts,
                                 const uint32_t *h_src, const uint32_t *h_dst, const uint32_t *h_bytes,
                                 uint64_t n, uint64_t *ticket);

/* Block until the request is done (info may be NULL), or return
 * SINET_ERR_TIMEOUT after timeout_ms. A done request's info can be read once;
 * SINET_ERR_INVALID_ARG for an unknown or already collected ticket. */
sinet_status sinet_server_wait(sinet_server *s, uint64_t ticket, uint32_t timeout_ms,
                               sinet_request_info *info);

/* Block until every submitted request is done, or SINET_ERR_TIMEOUT. */
sinet_status sinet_server_drain(sinet_server *s, uint32_t timeout_ms);

/* Device pointers of a tenant's resident histogram (read them after a drain). */
sinet_status sinet_server_tenant_output(sinet_server *s, uint32_t tenant, sinet_hist_out *out);

/* Copy a tenant's resident histogram to host memory (count: uint32[2 * n_bins],
 * direction 0 first; bytes: uint64[2 * n_bins]; stats: uint64[8]). Waits for
 * the launch in flight, if any, and for nothing else: drain first for a
 * result that includes every submitted request. */
sinet_status sinet_server_export(sinet_server *s, uint32_t tenant, uint32_t *h_count, uint64_t *h_bytes,
                                 uint64_t *h_stats);

/* The reverse of sinet_server_export: replace a tenant's resident histogram
 * with host arrays in the same layout (a checkpoint taken earlier, on this
 * or another server). Waits for the launch in flight, if any; requests
 * admitted later accumulate onto the imported state. */
sinet_status sinet_server_import(sinet_server *s, uint32_t tenant, const uint32_t *h_count, const uint64_t *h_bytes,
                                 const uint64_t *h_stats);

/* Counters and latency percentiles; reset = 1 clears them afterwards. */
sinet_status sinet_server_stats(sinet_server *s, int reset, sinet_server_counters *st);

/* Stop the worker (requests not yet done are dropped), free everything. */
sinet_status sinet_server_destroy(sinet_server *s);

/* ------------------------------------------------------------------------
 * Post-processing of a histogram on the device (the coarser views of
 * Section 6: hourly and ten-minute series; the present-keys output of the
 * reduce-by-key of Section 5).
 */

/* Roll a histogram of n_bins bins up into ceil(n_bins / factor) coarser bins:
 * out bin j = the sum of in bins [j * factor, (j + 1) * factor) in both
 * directions (counts modulo 2^32, byte sums modulo 2^64), which equals the
 * histogram taken directly with bin width factor * w at the same t0. out's
 * arrays hold ceil(n_bins / factor) entries and must not overlap in's; with
 * accumulate = 0 they are overwritten, else added to. in->stats is copied to
 * out->stats when both are given. Device pointers; asynchronous on stream. */
sinet_status sinet_histogram_rollup(const sinet_hist_out *in, uint64_t n_bins, uint64_t factor, int accumulate,
                                    const sinet_hist_out *out, sinet_stream_t stream);

/* Sparse form: the bins with a non-zero count or byte sum in either
 * direction, in increasing bin order, as parallel device arrays (bin index,
 * count per direction, byte sum per direction) of capacity cap. The number
 * of such bins is written to the device word *d_n_out; when it exceeds cap,
 * only the first cap are written. Asynchronous on stream (one small
 * stream-ordered scratch allocation). */
sinet_status sinet_histogram_sparse(const sinet_hist_out *in, uint64_t n_bins, uint32_t *d_bin, uint32_t *d_count0,
                                    uint32_t *d_count1, uint64_t *d_bytes0, uint64_t *d_bytes1, uint64_t cap,
                                    uint64_t *d_n_out, sinet_stream_t stream);

/*
 * The strategy (sinet_strategy) that a call of sinet_discriminate_histogram
 * with these parameters over n records would run: p->strategy unless it is
 * AUTO; for AUTO, the measured choice cached for the call's input class
 * (SINET_HINT_TUNE) or else the fixed rule (the whole-histogram tile for
 * small histograms, the chunk tile for time-sorted input, the hot/cold
 * partition for unsorted input over a histogram of 256 MB or more with at
 * least one record per four bins (the 32-byte cells where the partition's
 * limits are exceeded, or where its scratch does not fit the free device
 * memory at the call), warp combining otherwise). No kernel runs.
 */
sinet_status sinet_auto_strategy(const sinet_prefix_table *t, uint64_t n, const sinet_hist_params *p,
                                 int32_t *strategy);

/*
 * Read and clear the device status word of the current device, after
 * synchronising `stream`. *device_code receives the latched sinet_status
 * (SINET_OK if nothing failed).
 */
sinet_status sinet_device_status(sinet_stream_t stream, uint32_t *device_code);

/* Fill a params struct with defaults: exclusive policy, AUTO strategy/lookup. */
void sinet_default_params(sinet_hist_params *p, uint64_t t0_ms, uint64_t bin_width_ms,
                          uint64_t n_bins);

#ifdef __cplusplus
}
#endif

#endif /* SINET_H */
