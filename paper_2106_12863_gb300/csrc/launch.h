// Host-side launchers of the kernels (one definition per .cu file).
#pragma once
#include <cuda_runtime.h>

#include "records.cuh"

namespace sinet {

struct LaunchCfg {
    int grid = 0;       // 0: persistent, SM count x resident CTAs per SM
    int block = 256;
    cudaStream_t stream = nullptr;
    uint32_t *status = nullptr;
    int sm_count = 0;
};

struct TileArgs {
    uint32_t tile_bins;   // bins per direction in the tile (FULL: n_bins)
    uint32_t iters;       // quads per thread per chunk
    uint32_t margin;      // bins kept below a chunk's first record
    uint32_t full;        // 1: the tile is the whole histogram (base 0)
};

// The bin of each record ((ts - t0) / w) or 0xFFFFFFFF outside the window.
cudaError_t run_bin(const uint64_t *ts, uint64_t n, const HistArgs &h, uint32_t *bin, const LaunchCfg &c);

// Algorithm 1 only: class bytes (optional) and class counts.
cudaError_t run_discriminate(int lk, const RecArgs &r, const TableArgs &t, uint64_t *counts,
                             const LaunchCfg &c);

// Fused discriminate + histogram with global atomics (warp-aggregated or not).
// `cache_set_bits`: log2 of the sets of the per-CTA hot-key cache (4 ways each).
// `watch` (optional): only records with src or dst in this list are counted
// and binned; the others count in stats[6].
cudaError_t run_fused_atomic(int lk, bool agg, const RecArgs &r, const TableArgs &t,
                             const HistArgs &h, uint32_t cache_set_bits, const LaunchCfg &c,
                             const TableArgs *watch = nullptr);

// Fused discriminate + histogram with shared-memory bin tiles.
cudaError_t run_fused_tile(int lk, const RecArgs &r, const TableArgs &t, const HistArgs &h,
                           const TileArgs &ta, const LaunchCfg &c);

// Expand per-bin cells (see HistArgs::cells) into the output arrays of h,
// adding to them when accumulate is set.
cudaError_t run_cells_expand(const HistArgs &h, bool accumulate, const LaunchCfg &c);

// Largest dynamic shared memory a CTA may use on this device.
size_t smem_optin_limit();

// ---------------------------------------------------------------------------
// Batched persistent launch: many slices, each with its own records, table,
// window, bin width and outputs, in one launch whose CTAs pull (slice, chunk)
// work items from a device counter.

// Histogram update of one slice inside the batch kernel.
enum : uint32_t {
    BS_AGG = 0,    // warp run-combining + per-CTA hot-key cache, then global atomics
    BS_NOAGG = 1,  // global atomics per run of equal keys
    BS_TILE = 2,   // the slice's whole histogram as a shared-memory tile per work item
};

struct BatchSlice {
    RecArgs r;
    TableArgs t;
    HistArgs h;
    uint32_t lk;         // LK_TOGGLE1, LK_TOGGLE2, LK_INTERVAL or LK_INTERVAL_GLOBAL
    uint32_t strat;      // BS_*
    uint32_t tile_bins;  // BS_TILE: bins per direction of the tile (>= n_bins, multiple of 4)
    uint32_t zero;       // 1: the outputs are zeroed by the launch (not accumulated into)
    uint32_t item_quads; // quads per work item of this slice
    uint32_t ready_value;       // with `ready`: the value that means the records are in place
    const uint32_t *ready;      // optional device word; items wait (bounded) until it equals ready_value
};

// Device-resident header read by both batch kernels at every launch, so one
// captured graph serves any slice set up to its capacity.
struct BatchHeader {
    uint32_t n_slices;
    uint32_t reserved;
    uint32_t total_items;  // work items of all slices
    uint32_t total_zero;   // zeroing items of all slices
    uint32_t counter;      // work-item counter, reset by the zeroing kernel
    uint32_t pad;
    uint64_t wait_ns;      // bound of a wait on a slice's ready word (global timer, ns)
};

// Device arrays of a batch (all device pointers).
struct BatchArgs {
    BatchHeader *hdr;
    const BatchSlice *slices;
    const uint32_t *item_start;  // [n_slices + 1] first work item of each slice
    const uint32_t *zero_start;  // [n_slices + 1] first zeroing item of each slice
};

// Bins per zeroing item of the batch zeroing kernel.
constexpr uint32_t kZeroBins = 1u << 16;
// Hot-key cache of the batch kernel: 2^9 sets x 4 ways, 16 bytes a slot.
constexpr uint32_t kBatchCacheSetBits = 9;
constexpr uint32_t kBatchCacheBytes = 16u << (kBatchCacheSetBits + 2);
// Threads of a batch CTA.
constexpr int kBatchBlock = 384;
// Batches of at most this many slices keep their work-item starts in shared memory.
constexpr uint32_t kBatchSmemStarts = 1024;

// Zero the outputs of the slices marked `zero` and reset the work counter.
cudaError_t run_batch_zero(const BatchArgs &b, int grid, cudaStream_t s);
// The persistent batch kernel with `smem` bytes of dynamic shared memory per
// CTA (table region + work region of any slice must fit).
cudaError_t run_batch(const BatchArgs &b, uint32_t smem, int grid, cudaStream_t s, uint32_t *status);
// Set the batch kernel's dynamic shared memory limit; returns CTAs per SM.
cudaError_t batch_occupancy(uint32_t smem, int *per_sm);

// Plain path: discriminate -> emit keys -> radix sort -> reduce by key.
struct SortPlan {
    uint64_t n_emit_max;   // upper bound of emitted (key, bytes) pairs
    uint32_t key_bits;     // bits of key = d * n_bins + bin
    uint32_t passes;       // 8-bit digit passes
    uint64_t emit_tiles;   // tiles of the emit kernel
    uint64_t sort_tiles;   // tiles of a radix pass (upper bound)
    size_t scratch_bytes;  // total scratch needed
    // offsets into scratch
    size_t off_keys0, off_vals0, off_keys1, off_vals1, off_hist, off_emit_status, off_sort_status,
        off_counters;
};
SortPlan plan_sort_reduce(uint64_t n, uint32_t n_bins, bool two_dir);
cudaError_t run_sort_reduce(int lk, const RecArgs &r, const TableArgs &t, const HistArgs &h,
                            const SortPlan &plan, void *scratch, bool accumulate,
                            const LaunchCfg &c);

}  // namespace sinet
