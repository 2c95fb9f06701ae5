// Host compilation of a CIDR list (step a-1 of the hot path; runs once per table).
//
// Algorithm 1 compares bitmask(X, Z) with bitmask(Y, Z) for each entry Y/Z of
// the CIDR list. Everything the kernels need is derived here, exactly:
//   * canonical entries: net &= bitmask(len) (the CB of Algorithm 1), deduped,
//     grouped by length and sorted -> per-mask-length binary search;
//   * the union of the entries as disjoint intervals [lo, hi] (nested and
//     duplicate entries merged, adjacent ranges coalesced) with a direct index
//     over the top k address bits -> one index probe plus a short search.
// Membership in the list is membership in the union, so both forms answer
// the same question as the per-entry loop of Algorithm 1.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sinet.h"
#include "table_host.h"

namespace sinet {

static inline uint32_t prefix_mask(uint32_t len) { return len == 0 ? 0u : (0xFFFFFFFFu << (32 - len)); }

static uint32_t pad16(uint32_t b) { return (b + 15u) & ~15u; }

static uint32_t iv_image_bytes(uint32_t n_iv, uint32_t k) {
    return pad16(4 * n_iv) * 2 + pad16(2 * ((1u << k) + 1));
}

int compile_table(const uint32_t *net, const uint8_t *len, uint32_t n, uint32_t index_bits,
                  TableHost &t) {
    if (n > (1u << 24)) return SINET_ERR_TABLE_TOO_LARGE;
    if (n && (!net || !len)) return SINET_ERR_INVALID_ARG;
    if (index_bits > 20) return SINET_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < n; i++)
        if (len[i] > 32) return SINET_ERR_INVALID_ARG;

    // canonicalise, then sort by (len, net) and dedup
    std::vector<uint64_t> keyed(n);
    for (uint32_t i = 0; i < n; i++)
        keyed[i] = (uint64_t)len[i] << 32 | (net[i] & prefix_mask(len[i]));
    std::sort(keyed.begin(), keyed.end());
    keyed.erase(std::unique(keyed.begin(), keyed.end()), keyed.end());
    t.nets.resize(keyed.size());
    std::memset(t.len_offset, 0, sizeof t.len_offset);
    for (size_t i = 0; i < keyed.size(); i++) {
        t.nets[i] = (uint32_t)keyed[i];
        t.len_offset[(keyed[i] >> 32) + 1]++;
    }
    for (int L = 1; L < 34; L++) t.len_offset[L] += t.len_offset[L - 1];

    t.groups.clear();
    for (uint32_t L = 0; L <= 32; L++) {
        uint32_t c = t.len_offset[L + 1] - t.len_offset[L];
        if (c) t.groups.push_back({L, t.len_offset[L], c});
    }
    // probe the lengths that cover the most addresses first (early exit on a hit)
    std::stable_sort(t.groups.begin(), t.groups.end(), [](const TableHost::Group &a, const TableHost::Group &b) {
        long double ca = (long double)a.cnt * std::ldexp(1.0L, 32 - (int)a.len);
        long double cb = (long double)b.cnt * std::ldexp(1.0L, 32 - (int)b.len);
        return ca > cb;
    });

    // union as intervals: sort by start, merge overlapping or adjacent ranges
    std::vector<std::pair<uint32_t, uint32_t>> r(keyed.size());
    for (size_t i = 0; i < keyed.size(); i++) {
        uint32_t L = (uint32_t)(keyed[i] >> 32), s = (uint32_t)keyed[i];
        r[i] = {s, s | ~prefix_mask(L)};
    }
    std::sort(r.begin(), r.end());
    t.lo.clear();
    t.hi.clear();
    for (auto &iv : r) {
        if (!t.lo.empty() && (uint64_t)iv.first <= (uint64_t)t.hi.back() + 1) {
            t.hi.back() = std::max(t.hi.back(), iv.second);
        } else {
            t.lo.push_back(iv.first);
            t.hi.push_back(iv.second);
        }
    }
    const uint32_t n_iv = (uint32_t)t.lo.size();

    // direct index bits: the fewest (>= 6) whose buckets hold at most four
    // candidate intervals (two halving steps), else as many as fit the
    // shared-memory budget
    auto build_index = [&](uint32_t k) {
        const uint32_t nb = 1u << k;
        t.index.assign(nb + 1, n_iv);
        uint32_t j = 0;  // index[b] = first interval with hi >= bucket start
        for (uint32_t b = 0; b < nb; b++) {
            uint64_t start = (uint64_t)b << (32 - k);
            while (j < n_iv && (uint64_t)t.hi[j] < start) j++;
            t.index[b] = j;
        }
        t.index[nb] = n_iv;
        uint32_t mr = 0;
        for (uint32_t b = 0; b < nb && n_iv; b++) {
            uint32_t e = std::min(t.index[b + 1], n_iv - 1);
            uint32_t s0 = t.index[b];
            mr = std::max(mr, e >= s0 ? e - s0 + 1 : 0u);
        }
        return mr;
    };
    uint32_t k = index_bits;
    if (k == 0) {
        uint32_t best = 0;
        for (uint32_t c = 6; c <= 16; c++) {
            if (iv_image_bytes(n_iv, c) > kSmemTableBudget) break;
            best = c;
            if (build_index(c) <= 4) break;
        }
        k = best ? best : 16;  // nothing fits shared memory: global lookups
    }
    t.index_bits = k;
    t.max_range = build_index(k);

    // toggle form `form` (1, 2 or 0, see table_host.h) at kb bucket bits;
    // returns (most blocks one bucket needs, image bytes), or ~0 when the form
    // cannot hold this table
    auto build_toggles = [&](uint32_t kb, uint32_t form, bool keep) {
        const uint32_t nb = 1u << kb;
        const auto fail = std::pair<uint32_t, size_t>(~0u, ~size_t(0));
        std::vector<uint32_t> desc(nb, 0), blocks(4, 0x7FFFFFFFu);
        uint32_t maxb = 1, j = 0;
        std::vector<uint32_t> tog;
        for (uint32_t b = 0; b < nb; b++) {
            const uint64_t start = (uint64_t)b << (32 - kb);
            const uint64_t end = start + (1ull << (32 - kb)) - 1;
            while (j < n_iv && (uint64_t)t.hi[j] < start) j++;  // first with hi >= start
            const uint32_t s0 = (j < n_iv && (uint64_t)t.lo[j] <= start) ? 1u : 0u;
            tog.clear();
            for (uint32_t e = j; e < n_iv && (uint64_t)t.lo[e] <= end; e++) {
                if ((uint64_t)t.lo[e] > start) tog.push_back((uint32_t)((uint64_t)t.lo[e] - start));
                if ((uint64_t)t.hi[e] < end) tog.push_back((uint32_t)((uint64_t)t.hi[e] + 1 - start));
            }
            const uint32_t need = (uint32_t)(tog.size() + 3) / 4;
            maxb = std::max(maxb, need ? need : 1u);
            uint32_t first = 0;
            if (need) {
                first = (uint32_t)blocks.size() / 4;
                for (uint32_t i = 0; i < need * 4; i++) blocks.push_back(i < tog.size() ? tog[i] - 1 : 0x7FFFFFFFu);
            }
            if (form == 1) {
                if (need > 1 || first > 0x7FFFu) return fail;
                desc[b] = first | (s0 << 31);
            } else if (form == 2) {
                if (need > 2 || first + 1 > 0x7FFFu) return fail;
                desc[b] = first | ((need == 2 ? first + 1 : 0u) << 15) | (s0 << 31);
            } else {
                const uint32_t nblk = need ? need : 1u;
                if (nblk > 15 || first > 0xFFFFFFu) return fail;
                desc[b] = first | (nblk << 24) | (s0 << 31);
            }
        }
        const size_t bytes = 4 * blocks.size() + 4 * (size_t)nb;
        if (keep) {
            t.desc.swap(desc);
            t.blocks.swap(blocks);
            t.desc_bits = kb;
            t.max_blocks = maxb;
            t.toggle_form = form;
        }
        return std::pair<uint32_t, size_t>(maxb, bytes);
    };
    // one block per bucket if some bit count allows it, else two, else as
    // many as needed; within a form, the fewest bits that fit the budget
    uint32_t kb = 0, form = 0;
    for (uint32_t f : {1u, 2u}) {
        for (uint32_t c = 8; c <= 14 && !kb; c++) {
            auto r = build_toggles(c, f, false);
            if (r.first != ~0u && r.second <= kSmemTableBudget) {
                kb = c;
                form = f;
            }
        }
        if (kb) break;
    }
    if (!kb) {
        size_t best = ~size_t(0);
        for (uint32_t c = 8; c <= 14; c++) {
            auto r = build_toggles(c, 0, false);
            if (r.first != ~0u && r.second < best) {
                best = r.second;
                kb = c;
            }
        }
        if (!kb) kb = 14;
        form = 0;
    }
    build_toggles(kb, form, true);
    return SINET_OK;
}

std::vector<uint8_t> serialise(const TableHost &t, TableImage &img) {
    const uint32_t n_iv = (uint32_t)t.lo.size();
    const uint32_t n_pairs = n_iv ? n_iv : 1;  // an empty table keeps one empty interval
    const uint32_t nb1 = (1u << t.index_bits) + 1;
    img = TableImage{};
    uint32_t off = 0;
    img.off_blocks = off;
    off += pad16(4 * (uint32_t)t.blocks.size());
    img.off_desc = off;
    off += pad16(4 * (uint32_t)t.desc.size());
    img.iv_bytes = off;
    img.iv_fits_smem = !t.desc.empty() && t.max_blocks <= 15 && img.iv_bytes <= kSmemTableBudget;
    img.off_nets = off;
    off += pad16(4 * (uint32_t)t.nets.size());
    img.off_groups = off;
    off += 16 * (uint32_t)t.groups.size();
    img.pml_bytes = off - img.off_nets;
    img.pml_fits_smem = img.pml_bytes <= kSmemTableBudget;
    img.off_lo = off;
    off += pad16(4 * n_pairs);
    img.off_hi = off;
    off += pad16(4 * n_pairs);
    img.off_idx32 = off;
    off += pad16(4 * nb1);
    img.total = off;

    std::vector<uint8_t> buf(img.total, 0);
    uint32_t *lo = reinterpret_cast<uint32_t *>(buf.data() + img.off_lo);
    uint32_t *hi = reinterpret_cast<uint32_t *>(buf.data() + img.off_hi);
    if (n_iv) {
        std::memcpy(lo, t.lo.data(), 4 * n_iv);
        std::memcpy(hi, t.hi.data(), 4 * n_iv);
    } else {
        lo[0] = 1;  // lo > hi: contains nothing
        hi[0] = 0;
    }
    if (!t.blocks.empty()) std::memcpy(buf.data() + img.off_blocks, t.blocks.data(), 4 * t.blocks.size());
    if (!t.desc.empty()) std::memcpy(buf.data() + img.off_desc, t.desc.data(), 4 * t.desc.size());
    if (!t.nets.empty()) std::memcpy(buf.data() + img.off_nets, t.nets.data(), 4 * t.nets.size());
    uint32_t *g = reinterpret_cast<uint32_t *>(buf.data() + img.off_groups);
    for (size_t i = 0; i < t.groups.size(); i++) {
        g[4 * i + 0] = t.groups[i].len;
        g[4 * i + 1] = t.groups[i].off;
        g[4 * i + 2] = t.groups[i].cnt;
        g[4 * i + 3] = 0;
    }
    std::memcpy(buf.data() + img.off_idx32, t.index.data(), 4 * nb1);
    return buf;
}

}  // namespace sinet

extern "C" sinet_status sinet_compile_prefix_table(const uint32_t *h_net, const uint8_t *h_len,
                                                   uint32_t n, uint32_t index_bits,
                                                   uint32_t *nets_by_len, uint32_t *len_offset,
                                                   uint32_t *iv_lo, uint32_t *iv_hi,
                                                   uint32_t *index, uint32_t *counts) {
    if (!len_offset || !counts) return SINET_ERR_INVALID_ARG;
    sinet::TableHost t;
    int rc = sinet::compile_table(h_net, h_len, n, index_bits, t);
    if (rc != SINET_OK) return (sinet_status)rc;
    if (nets_by_len && !t.nets.empty()) std::memcpy(nets_by_len, t.nets.data(), 4 * t.nets.size());
    std::memcpy(len_offset, t.len_offset, sizeof t.len_offset);
    if (iv_lo && !t.lo.empty()) std::memcpy(iv_lo, t.lo.data(), 4 * t.lo.size());
    if (iv_hi && !t.hi.empty()) std::memcpy(iv_hi, t.hi.data(), 4 * t.hi.size());
    if (index) std::memcpy(index, t.index.data(), 4 * t.index.size());
    counts[0] = (uint32_t)t.nets.size();
    counts[1] = (uint32_t)t.lo.size();
    counts[2] = t.index_bits;
    counts[3] = t.max_range;
    return SINET_OK;
}

extern "C" sinet_status sinet_prefix_table_image(const uint32_t *h_net, const uint8_t *h_len,
                                                 uint32_t n, uint8_t *image, size_t capacity,
                                                 uint32_t *layout, size_t *bytes) {
    if (!layout || !bytes) return SINET_ERR_INVALID_ARG;
    sinet::TableHost t;
    int rc = sinet::compile_table(h_net, h_len, n, 0, t);
    if (rc != SINET_OK) return (sinet_status)rc;
    sinet::TableImage img;
    std::vector<uint8_t> buf = sinet::serialise(t, img);
    *bytes = buf.size();
    const uint32_t v[16] = {img.off_blocks, img.off_desc, t.desc_bits, img.iv_bytes,
                            img.off_nets, img.off_groups, (uint32_t)t.groups.size(), img.pml_bytes,
                            img.off_lo, img.off_hi, img.off_idx32, t.index_bits,
                            (uint32_t)t.lo.size(), t.max_blocks | (t.toggle_form << 8),
                            img.iv_fits_smem ? 1u : 0u, img.pml_fits_smem ? 1u : 0u};
    std::memcpy(layout, v, sizeof v);
    if (image) {
        if (capacity < buf.size()) return SINET_ERR_INVALID_ARG;
        std::memcpy(image, buf.data(), buf.size());
    }
    return SINET_OK;
}
