// Host-side compiled CIDR list and its device image layout.
#pragma once
#include <cstdint>
#include <vector>

namespace sinet {

// Shared-memory budget for a staged table image (intervals + direct index or
// per-length groups). Tables larger than this are looked up from global memory.
constexpr uint32_t kSmemTableBudget = 96 * 1024;

struct TableHost {
    // canonical unique networks, ascending mask length, sorted within a length
    std::vector<uint32_t> nets;
    uint32_t len_offset[34] = {0};
    // union of all entries as sorted, disjoint, non-adjacent closed intervals
    std::vector<uint32_t> lo, hi;
    uint32_t index_bits = 0;
    std::vector<uint32_t> index;  // 2^index_bits + 1 entries
    uint32_t max_range = 0;       // largest candidate range of an index bucket
    // toggle form for shared memory. A toggle is the offset t >= 1 from a
    // bucket's start (bucket = the top desc_bits address bits) at which
    // membership flips, stored as t - 1 in blocks of four (padded with the
    // never-reached 0x7FFFFFFF); membership of an address is the state at the
    // bucket start XOR the parity of the toggles at or below its offset. Block 0
    // is all padding and serves pure buckets. Per-bucket descriptor, bit 31 =
    // state at the bucket start, and:
    //   form 1: bits 0-14 = the bucket's only block (at most 4 toggles)
    //   form 2: bits 0-14 and 15-29 = its two blocks (at most 8 toggles; the
    //           second is block 0 when four suffice)
    //   form 0: bits 0-23 = first of consecutive blocks, bits 24-27 = count
    uint32_t desc_bits = 0;
    std::vector<uint32_t> desc;
    std::vector<uint32_t> blocks;  // 4 u32 per block
    uint32_t max_blocks = 0;       // most blocks one bucket needs
    uint32_t toggle_form = 0;  // 1, 2 or 0 as described above
    // per-length groups in probe order (most covered addresses first)
    struct Group { uint32_t len, off, cnt; };
    std::vector<Group> groups;
};

// Compile (canonicalise, dedup, group, merge, index). index_bits 0 = choose.
// Returns 0 or a sinet_status code.
int compile_table(const uint32_t *net, const uint8_t *len, uint32_t n, uint32_t index_bits,
                  TableHost &out);

// Layout of the single contiguous device image (all offsets 16-byte aligned).
struct TableImage {
    uint32_t off_blocks = 0, off_desc = 0;   // shared-memory toggle form
    uint32_t off_nets = 0, off_groups = 0;   // per-length form
    uint32_t off_lo = 0, off_hi = 0, off_idx32 = 0;  // global-memory interval form
    uint32_t iv_bytes = 0;    // bytes of [blocks | desc] staged for INTERVAL
    uint32_t pml_bytes = 0;   // bytes of [nets | groups] staged for PML
    uint32_t total = 0;
    bool iv_fits_smem = false, pml_fits_smem = false;
};

// Serialise into one buffer laid out as `img` describes.
std::vector<uint8_t> serialise(const TableHost &t, TableImage &img);

}  // namespace sinet
