// Hot/cold partitioned histogram update (SINET_STRAT_PARTITION): host-side
// plan of the launch sequence and its scratch layout.
//
// The scheme, for unsorted records over a histogram far larger than L2 (the
// heavy day's Zipf-skewed bins):
//   1. sample: classify and bin a strided sample of the records and count
//      sample hits per bin in an L2-resident hash table;
//   2. select: the bins with the most sample hits form a static hot table
//      (4-way sets, hottest first), the same in every CTA;
//   3. main pass (one read of the records, staged into shared memory by TMA
//      bulk copies): hot bins are accumulated in each CTA's shared-memory copy
//      of the hot table; every other routed update becomes an 8-byte entry
//      (bin << 1 | direction, bytes) appended to a CTA-private page of its
//      coarse bin range (a bucket);
//   4. pages are grouped by bucket;
//   5. cold pass (one cooperative launch): the CTAs' page-sorting groups take
//      each bucket's pages one at a time and sort each by owner CTA in place
//      (the pages stay in L2); behind them, each CTA's reducing warps sum its
//      own slice of the bucket's bins in a shared-memory tile and store every
//      bin of the slice once;
//   6. the hot table's totals are added to their bins.
// Every update is counted exactly once: in a hot slot or as a cold entry.
#pragma once
#include "launch.h"

namespace sinet {

// Main pass: 31 consumer warps and one producer warp, 1,024 threads (64
// registers each fit the register file), two adjacent records per consumer
// per stage (read with one 16-byte and three 8-byte shared-memory loads), two
// stages of 39 KB in flight.
constexpr int kPartConsumers = 992;                 // consumer threads of the main pass
constexpr int kPartThreads = kPartConsumers + 32;   // plus one producer warp (TMA)
constexpr int kPartRPT = 2;                         // records per consumer per stage
constexpr uint32_t kPartStageRecords = kPartRPT * kPartConsumers;  // records per TMA stage
static_assert((4 * kPartStageRecords) % 16 == 0, "every stage starts 16-byte aligned in every stream");
constexpr uint32_t kPartStages = 2;
constexpr uint32_t kPartStageBytes = 20 * kPartStageRecords;
constexpr uint32_t kPartPageBits = 11;              // 2,048 entries (16 KB) per page
constexpr uint32_t kPartPage = 1u << kPartPageBits;
constexpr uint32_t kPartMaxBuckets = 256;
constexpr uint32_t kPartMaxCand = 16384;            // hot candidates taken from the sample
constexpr uint32_t kPartSampleChunk = 512;          // records per sampled chunk
constexpr uint32_t kPartSampleSetBits = 9;          // sample pass: per-CTA pre-aggregation cache

// Device view of the scheme's scratch (all device pointers).
struct PartDev {
    // sample counts: open-addressing hash table over bins
    uint32_t *hash_keys;  // kNoKey when empty
    uint32_t *hash_cnt;
    uint32_t hash_mask;   // slots - 1
    uint32_t hash_shift;  // 32 - log2(slots): slot = top bits of the hash
    uint32_t *levels;     // [32] hash slots per log2 of their count; [32] sample hits in all
    uint32_t *cand_n;     // candidates collected
    uint2 *cand;          // [kPartMaxCand] (bin, sample count)
    // hot table (slot = 4 * set + way), the same in every CTA
    uint32_t *hot_keys;   // [slots] bin or kNoKey
    uint32_t *hot_cnt;    // [2][slots]
    uint64_t *hot_bytes;  // [2][slots]
    uint32_t set_bits;
    // cold entries: pages of kPartPage u64 entries, one bucket each. Pages
    // [0, dyn_base) are the CTAs' regions (CTA c's page k of bucket b is
    // (c * n_buckets + b) * creg + k); later pages are handed out on demand.
    uint32_t creg;          // region pages per CTA and bucket (at least 1)
    uint32_t dyn_base;      // first page handed out on demand
    uint32_t *page_alloc;   // pages handed out on demand
    uint32_t *page_bucket;  // [pages_cap]
    uint32_t *page_fill;    // [pages_cap] entries in the page
    uint64_t *pages;        // [pages_cap][kPartPage]
    uint32_t pages_cap;
    uint32_t cb_shift;      // bucket of a bin = bin >> cb_shift
    uint32_t n_buckets;
    // pages grouped by bucket
    uint32_t *bucket_cnt;   // [n_buckets] non-empty pages per bucket, then a cursor
    uint32_t *bucket_pg;    // [n_buckets + 1] first position of each bucket in page_list
    uint32_t *page_list;    // [pages_cap] page ids, grouped by bucket
    uint16_t *idx;          // [pages_cap][g_cold + 1] owner run offsets of each sorted page
    uint32_t *p1_done;      // [n_buckets] page-sorting groups done with the bucket
    uint32_t *pg_next;      // [n_buckets] pages of the bucket handed out for sorting
    // cold pass geometry
    uint32_t g_cold;        // CTAs of the cold pass (= owners per bucket)
    uint32_t own_bins;      // bins per owner
    Divider own_div;        // division by own_bins
    // main pass geometry: full TMA stages [i_lo, i_lo + n_full * R); the
    // other records (head, tail, or all when the streams cannot be staged)
    // are loaded one by one
    uint64_t i_lo, n_full;
    uint64_t n_head;        // records before i_lo
    // sample geometry: chunk k * sample_stride for k < sample_chunks
    uint64_t sample_chunks, sample_stride;
};

struct PartPlan {
    PartDev d;                 // pointers filled once the scratch exists
    uint32_t slots;            // 4 << set_bits
    int grid_main, grid_sample, grid_cold;
    int cold_groups;           // page-sorting groups of 256 threads in a 1,024-thread cold-pass CTA (1 or 2)
    size_t smem_main, smem_sample, smem_cold;
    size_t scratch_bytes;
    // scratch layout (byte offsets)
    size_t off_ff, bytes_ff;   // region set to 0xFF (hash keys, hot keys)
    size_t off_zero, bytes_zero;  // region set to zero
    size_t off_hash_keys, off_hot_keys, off_levels, off_cand_n, off_page_alloc, off_hot_cnt,
        off_hot_bytes, off_bucket_cnt, off_p1_done, off_pg_next, off_hash_cnt, off_cand, off_page_bucket,
        off_page_fill, off_bucket_pg, off_page_list, off_idx, off_pages;
};

// Plan for n records into h.n_bins bins with table lookup `lk`; returns
// cudaErrorNotSupported when the histogram or the input is beyond the
// scheme's limits (more than 256 buckets of 2^20 bins, 2^32 routed updates).
cudaError_t plan_partition(int lk, uint32_t table_smem, const RecArgs &r, const HistArgs &h,
                           uint32_t bucket_bits, int sm_count, size_t smem_optin, PartPlan *out);

// Enqueue the whole sequence; `scratch` holds plan.scratch_bytes.
cudaError_t run_partition(int lk, const RecArgs &r, const TableArgs &t, const HistArgs &h,
                          PartPlan plan, void *scratch, bool accumulate, const LaunchCfg &c);

}  // namespace sinet
