// Owner-computes histogram update for time-sorted records (SINET_STRAT_OWNER).
//
// The bins are cut into ranges of T bins. Because the records are sorted by
// timestamp (up to a bounded disorder), the records of range k are one
// contiguous run, found by binary search on ts. Each CTA owns a contiguous
// block of ranges, balanced by records plus bins, and walks it in order:
// the run of each range goes into a circular shared-memory tile of S = 2T
// slots (slot = bin mod S) that also holds H = T/2 bins on either side of the
// range, and the bins that no later run of the block can reach are stored
// with plain stores, every bin exactly once. The histogram needs no zeroing
// pass and sees no read-modify-write; records out of order by fewer than H
// bins cost nothing extra.
//
// Exact for any input: the searched run boundaries are made a partition of
// [0, n) (prefix maximum); a record whose bin falls outside its tile window
// (disorder beyond H, or across a block boundary) is a stray, and a run
// longer than an owner takes (tile entries count in 16 bits) spills into
// overflow items. Both are added with global reductions by a second kernel,
// after every owner has stored its bins.
#pragma once
#include "launch.h"

namespace sinet {

// A work item of the remainder kernel: records [x, y) of range k.
// OWN_STRAYS: add the records whose bin is outside [wlo, wlo + wlen) (the
// owner tiled the rest). OWN_FULL: count, bin and add all of them; the
// range's bins [wlo, wlo + wlen) go through a tile first.
struct OwnerItem {
    uint64_t x, y;
    uint32_t k;
    uint32_t mode;
    uint32_t wlo, wlen;
};

enum : uint32_t { OWN_STRAYS = 0, OWN_FULL = 1 };

// Records an owner CTA takes from one run. A tile entry counts in 16 bits,
// and a bin's entry collects records of at most two runs before it is
// stored (its own range's and the one before or after), so 2 * 32,767 fit.
constexpr uint32_t kOwnerCap = 32767;

// Shapes and scratch layout of one owner-computes call (one stream-ordered
// allocation).
struct OwnerPlan {
    uint32_t slots;       // S: tile slots per direction (power of two, >= 16)
    uint32_t range_bins;  // T = S / 2
    uint32_t halo_bins;   // H = S / 4
    uint32_t n_ranges;    // ceil(n_bins / T)
    uint32_t grid;        // owner CTAs (one block of ranges each)
    uint64_t cap_items;   // capacity of the item list (never exceeded, see plan_owner)
    size_t off_bounds;    // u64[n_ranges + 1] run boundaries
    size_t off_part;      // u32[grid + 1] first range of each CTA's block
    size_t off_items;     // OwnerItem[cap_items]
    size_t off_count;     // u32 item count
    size_t scratch_bytes;
};

// `slots`: tile slots per direction (rounded down to a power of two).
OwnerPlan plan_owner(uint64_t n, uint32_t n_bins, uint32_t slots, uint32_t grid);

// Resident CTAs of the owner kernel for this lookup form, block size and
// tile (the grid plan_owner wants).
cudaError_t owner_grid(int lk, bool w1, const TableArgs &t, uint32_t slots, const LaunchCfg &c, int *grid);

// The four launches of the strategy on c.stream: run boundaries, their prefix
// maximum and the block partition, the owner kernel, the remainder kernel.
// `vec_ok`: the four output arrays are 16-byte aligned (the owner then stores
// 4 bins per thread).
cudaError_t run_fused_owner(int lk, const RecArgs &r, const TableArgs &t, const HistArgs &h,
                            uint64_t bin_width, const OwnerPlan &plan, void *scratch,
                            bool accumulate, bool vec_ok, const LaunchCfg &c);

}  // namespace sinet
