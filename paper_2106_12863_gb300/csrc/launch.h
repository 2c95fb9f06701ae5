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

// Algorithm 1 only: class bytes (optional) and class counts.
cudaError_t run_discriminate(int lk, const RecArgs &r, const TableArgs &t, uint64_t *counts,
                             const LaunchCfg &c);

// Fused discriminate + histogram with global atomics (warp-aggregated or not).
// `cache_set_bits`: log2 of the sets of the per-CTA hot-key cache (4 ways each).
cudaError_t run_fused_atomic(int lk, bool agg, const RecArgs &r, const TableArgs &t,
                             const HistArgs &h, uint32_t cache_set_bits, const LaunchCfg &c);

// Fused discriminate + histogram with shared-memory bin tiles.
cudaError_t run_fused_tile(int lk, const RecArgs &r, const TableArgs &t, const HistArgs &h,
                           const TileArgs &ta, const LaunchCfg &c);

// Largest dynamic shared memory a CTA may use on this device.
size_t smem_optin_limit();

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
