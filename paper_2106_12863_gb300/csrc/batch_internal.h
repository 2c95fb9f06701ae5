// Host side of the batched launch, shared by the batch API and the serving
// loop: slice planning, strategy resolution (the autotuner), and the device
// engine that owns the descriptors and the captured graph.
#pragma once
#include <string>
#include <vector>

#include "api_internal.h"

namespace sinet {

// Quads per work item: at most 64,000 records (below the 65,536 a tile entry
// counts). Slices updated with global atomics get items small enough that the
// whole grid works on one slice at a time (at least kMinItemQuads), so the
// histograms under random read-modify-write stay few enough to share L2.
constexpr uint32_t kItemQuads = 16000;
constexpr uint32_t kMinItemQuads = 4096;
// Records of the representative slice a tuning run uses at most, and the most
// copies of it one tuning launch runs.
constexpr uint64_t kTuneRecords = 8ull << 20;
constexpr uint32_t kTuneCopies = 64;

struct PlannedSlice {
    BatchSlice d;
    uint32_t items = 0;       // work items (0 for a slice run by the plain path)
    uint32_t zero_items = 0;  // zeroing items (0 when accumulating)
    int32_t strategy = 0;     // sinet_strategy; AUTO until resolved
    bool tile_fits = false;   // the whole histogram fits a tile next to the table
    uint32_t user_index = 0;  // position in the caller's slice array
};

// Dynamic shared memory of a batch CTA on this device (two CTAs per SM).
uint32_t batch_smem(const DeviceState *ds);
// CTAs of the persistent batch grid (two per SM).
uint32_t batch_grid(const DeviceState *ds);

// Host-only checks of one slice (no CUDA call).
sinet_status check_slice(const sinet_batch_slice &u);
// Quads per work item of a slice run with scheme `scheme` by `grid` CTAs.
uint32_t item_quads_for(uint64_t quads, uint32_t scheme, uint32_t grid);
// Set the strategy of a planned slice (scheme, item size, item count).
void set_strategy(PlannedSlice &ps, int32_t strategy, uint32_t grid);
// Plan a checked slice for a batch kernel with `smem` bytes of shared memory.
sinet_status plan_slice(const sinet_batch_slice &u, const DeviceState *ds, uint32_t smem, PlannedSlice &ps);
// Give every AUTO slice a strategy: from the autotune cache, by timing the
// candidates (tune), or by the fixed rule.
sinet_status resolve_strategies(std::vector<PlannedSlice> &v, bool tune, const DeviceState *ds,
                                uint32_t smem, cudaStream_t s);
// Map a public strategy to the batch kernel's update scheme.
uint32_t batch_scheme(int32_t strategy);

// A slice run by the plain path (discriminate, radix sort, reduce by key) as
// its own chain of kernels in the batch's graph, after the persistent kernel.
struct SortJob {
    RecArgs r;
    TableArgs t;
    HistArgs h;
    int lk = 0;
    SortPlan plan{};
    void *scratch = nullptr;  // plan.scratch_bytes, owned by the engine
};

// Whether the plain path can run a slice (its emitted pairs are counted in 32 bits).
bool sort_feasible(const PlannedSlice &ps);

// Device-resident descriptors + the captured launch.
struct BatchEngine {
    int device = 0;
    uint32_t cap = 0;  // slices
    uint32_t smem = 0;
    int grid = 0, zgrid = 0;
    int sm_count = 0;
    void *d_mem = nullptr;
    size_t bytes = 0;
    size_t off_item = 0, off_zero = 0, off_slices = 0;
    BatchArgs args{};
    uint64_t wait_ns = 2000000000ull;  // bound of a ready-word wait
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<SortJob> sorts;  // slices run by the plain path, after the batch kernel

    sinet_status init(uint32_t capacity, const DeviceState *ds, uint32_t smem_bytes);
    // host image (header, starts, descriptors) of `v` in descriptor order
    void image(const std::vector<PlannedSlice> &v, std::vector<uint8_t> &buf) const;
    // scratch for the slices of v run by the plain path (before capture)
    sinet_status plan_sorts(const std::vector<PlannedSlice> &v, const DeviceState *ds);
    sinet_status capture(uint32_t *status);  // capture zero + batch kernels (+ plain chains) as a graph
    sinet_status launch(cudaStream_t s) const;
    void release();
};

}  // namespace sinet
