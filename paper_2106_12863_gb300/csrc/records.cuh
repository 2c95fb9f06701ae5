// Per-record pieces of the hot path shared by every kernel: loading a quad of
// SoA records, classifying (Algorithm 1 against the staged table), routing a
// class to directions, and binning (Section 5's millisecond histogram).
#pragma once
#include "common.cuh"

namespace sinet {

// Lookup kinds: LK_INTERVAL / LK_TOGGLE1 / LK_TOGGLE2 are the shared-memory
// toggle form with a variable / one / two blocks per bucket.
enum : int { LK_INTERVAL = 0, LK_PML = 1, LK_INTERVAL_GLOBAL = 2, LK_CLASS_IN = 3, LK_TOGGLE1 = 4,
             LK_TOGGLE2 = 5 };

struct RecArgs {
    const uint64_t *ts;
    const uint32_t *src;
    const uint32_t *dst;
    const uint32_t *bytes;
    const uint8_t *cls_in;  // classified input (sinet_histogram)
    uint8_t *cls_out;       // class output (sinet_discriminate), may be null
    QuadGeom g;
};

struct HistArgs {
    uint32_t *cnt[2];
    uint64_t *byt[2];
    uint64_t *stats;  // [0..3] per class, [4..5] out of window per direction
    uint64_t t0;
    uint64_t span;    // n_bins * w
    Divider div;
    uint32_t w_is_one;
    uint32_t policy;  // byte c = direction bits of class c
    uint32_t two_dir; // some class routes to both directions
    uint32_t n_bins;
    uint32_t *status;  // device status word
    // When set, updates go to one 32-byte cell per bin instead of the four
    // output arrays: u64 byte sums of directions 0 and 1, then their u32
    // counts (one DRAM sector per update where the arrays would touch two).
    uint64_t *cells;
};

// ---------------------------------------------------------------------------
// Classifier: stages the table image into shared memory (interval or
// per-length form) or reads it from global memory, and answers in(a).
template <int LK>
struct Classifier;

template <int NB>
struct ToggleClassifier {
    ToggleView<NB> v;
    // false (in every thread of the CTA) when the table did not land
    __device__ __forceinline__ bool init(const TableArgs &t, uint8_t *smem, uint64_t *bar,
                                         uint32_t *status) {
        const bool ok = stage_to_smem(smem, t.image, t.iv_bytes, bar, status);
        attach(t, smem);
        return ok;
    }
    // views over an image already staged at `smem`
    __device__ __forceinline__ void attach(const TableArgs &t, const uint8_t *smem) {
        v.blocks = reinterpret_cast<const uint4 *>(smem + t.off_blocks);
        v.desc = reinterpret_cast<const uint32_t *>(smem + t.off_desc);
        v.shift = 32 - t.desc_bits;
        v.off_mask = (1u << v.shift) - 1u;
    }
    static __host__ __device__ uint32_t smem_bytes(const TableArgs &t) { return t.iv_bytes; }
    template <int N>
    __device__ __forceinline__ void in_n(const uint32_t (&a)[N], uint32_t (&r)[N]) const {
        v.template contains_n<N>(a, r);
    }
    // in_n for a whole converged warp: when no lane's address falls in a
    // bucket with blocks (the common case: most buckets are pure), the
    // descriptors' parity bits are the answers and one vote replaces the
    // per-lookup block branches.
    template <int N>
    __device__ __forceinline__ void in_n_warp(const uint32_t (&a)[N], uint32_t (&r)[N]) const {
        if (NB == 0) {  // every bucket has a block
            v.template contains_n<N>(a, r);
            return;
        }
        constexpr uint32_t kBlocks = NB == 2 ? 0x3FFFFFFFu : 0x7FFFu;
        uint32_t d[N], any = 0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            d[i] = v.desc[a[i] >> v.shift];
            any |= d[i] & kBlocks;
        }
        if (__any_sync(kFull, any)) {
            v.template contains_n<N>(a, r);
            return;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) r[i] = d[i] >> 31;
    }
};
template <>
struct Classifier<LK_INTERVAL> : ToggleClassifier<0> {};
template <>
struct Classifier<LK_TOGGLE1> : ToggleClassifier<1> {};
template <>
struct Classifier<LK_TOGGLE2> : ToggleClassifier<2> {};

template <>
struct Classifier<LK_PML> {
    PmlView v;
    __device__ __forceinline__ bool init(const TableArgs &t, uint8_t *smem, uint64_t *bar,
                                         uint32_t *status) {
        const bool ok = stage_to_smem(smem, t.image + t.off_nets, t.pml_bytes, bar, status);
        v.nets = reinterpret_cast<const uint32_t *>(smem);
        v.groups = reinterpret_cast<const uint4 *>(smem + (t.off_groups - t.off_nets));
        v.n_groups = t.n_groups;
        return ok;
    }
    static __host__ __device__ uint32_t smem_bytes(const TableArgs &t) { return t.pml_bytes; }
    template <int N>
    __device__ __forceinline__ void in_n(const uint32_t (&a)[N], uint32_t (&r)[N]) const {
#pragma unroll
        for (int i = 0; i < N; ++i) r[i] = v.contains(a[i]);
    }
    template <int N>
    __device__ __forceinline__ void in_n_warp(const uint32_t (&a)[N], uint32_t (&r)[N]) const {
        in_n<N>(a, r);
    }
};

template <>
struct Classifier<LK_INTERVAL_GLOBAL> {
    IntervalView<uint32_t> v;
    __device__ __forceinline__ bool init(const TableArgs &t, uint8_t *, uint64_t *, uint32_t *) {
        attach(t, nullptr);
        return true;
    }
    __device__ __forceinline__ void attach(const TableArgs &t, const uint8_t *) {
        v.lo = reinterpret_cast<const uint32_t *>(t.image + t.off_lo);
        v.hi = reinterpret_cast<const uint32_t *>(t.image + t.off_hi);
        v.idx = reinterpret_cast<const uint32_t *>(t.image + t.off_idx32);
        v.shift = 32 - t.index_bits;
        v.n_iv = t.n_iv;
    }
    static __host__ __device__ uint32_t smem_bytes(const TableArgs &) { return 0; }
    template <int N>
    __device__ __forceinline__ void in_n(const uint32_t (&a)[N], uint32_t (&r)[N]) const {
#pragma unroll
        for (int i = 0; i < N; ++i) r[i] = v.contains(a[i]);
    }
    template <int N>
    __device__ __forceinline__ void in_n_warp(const uint32_t (&a)[N], uint32_t (&r)[N]) const {
        in_n<N>(a, r);
    }
};

template <>
struct Classifier<LK_CLASS_IN> {
    __device__ __forceinline__ bool init(const TableArgs &, uint8_t *, uint64_t *, uint32_t *) { return true; }
    static __host__ __device__ uint32_t smem_bytes(const TableArgs &) { return 0; }
    template <int N>
    __device__ __forceinline__ void in_n(const uint32_t (&)[N], uint32_t (&r)[N]) const {
#pragma unroll
        for (int i = 0; i < N; ++i) r[i] = 0;
    }
};

// ---------------------------------------------------------------------------
// A quad of records. `valid` has bit j set when record j exists.
struct Quad {
    uint64_t ts[4];
    uint32_t src[4], dst[4], by[4], cls[4];
    uint32_t valid;
};

// Load quad q with the fields the caller needs.
template <bool TS, bool ADDR, bool BY, bool CIN>
__device__ __forceinline__ void load_quad(const RecArgs &r, uint64_t q, uint64_t pol, Quad &Q) {
    const int64_t base = quad_base(r.g, q);
    if (q < r.g.quads && quad_full(r.g, base)) {
        if (TS) {
            ulonglong2 a = ld_stream_v2u64(r.ts + base, pol);
            ulonglong2 b = ld_stream_v2u64(r.ts + base + 2, pol);
            Q.ts[0] = a.x; Q.ts[1] = a.y; Q.ts[2] = b.x; Q.ts[3] = b.y;
        }
        if (ADDR) {
            uint4 s = ld_stream_v4(r.src + base, pol);
            uint4 d = ld_stream_v4(r.dst + base, pol);
            Q.src[0] = s.x; Q.src[1] = s.y; Q.src[2] = s.z; Q.src[3] = s.w;
            Q.dst[0] = d.x; Q.dst[1] = d.y; Q.dst[2] = d.z; Q.dst[3] = d.w;
        }
        if (BY) {
            uint4 b = ld_stream_v4(r.bytes + base, pol);
            Q.by[0] = b.x; Q.by[1] = b.y; Q.by[2] = b.z; Q.by[3] = b.w;
        }
        if (CIN) {
            uint32_t w = ld_stream_u32(reinterpret_cast<const uint32_t *>(r.cls_in + base), pol);
            Q.cls[0] = w & 3u; Q.cls[1] = (w >> 8) & 3u; Q.cls[2] = (w >> 16) & 3u; Q.cls[3] = (w >> 24) & 3u;
        }
        Q.valid = 0xFu;
        return;
    }
    // partial quad (head, tail, unaligned streams) or past the end: scalar
    // loads of the records that exist, zeros elsewhere
    Q.valid = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        Q.ts[j] = 0;
        Q.src[j] = Q.dst[j] = Q.by[j] = Q.cls[j] = 0;
        const int64_t i = base + j;
        if (q >= r.g.quads || i < 0 || (uint64_t)i >= r.g.n) continue;
        Q.valid |= 1u << j;
        if (TS) Q.ts[j] = ld_stream_u64(r.ts + i, pol);
        if (ADDR) {
            Q.src[j] = ld_stream_u32(r.src + i, pol);
            Q.dst[j] = ld_stream_u32(r.dst + i, pol);
        }
        if (BY) Q.by[j] = ld_stream_u32(r.bytes + i, pol);
        if (CIN) Q.cls[j] = ld_stream_u8(r.cls_in + i) & 3u;
    }
}

// class = in(src) | in(dst) << 1 for the valid records of a quad (Algorithm 1).
template <int LK>
__device__ __forceinline__ void classify_quad(const Classifier<LK> &C, Quad &Q) {
    if (LK == LK_CLASS_IN) return;
    uint32_t a[4], r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = Q.src[j];
    C.template in_n<4>(a, r);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        Q.cls[j] = r[j];
        a[j] = Q.dst[j];
    }
    C.template in_n<4>(a, r);
#pragma unroll
    for (int j = 0; j < 4; ++j) Q.cls[j] |= r[j] << 1;
}

// Route + bin one record: returns its direction bits with out-of-window
// directions removed (they are counted in oor[]), and the bin. W1: the bin
// width is 1 ms (no division); otherwise division by the invariant width.
template <bool W1>
__device__ __forceinline__ uint32_t route_w(const HistArgs &h, uint32_t cls, uint64_t ts,
                                            uint32_t &bin, uint32_t oor[2]) {
    uint32_t dirs = (h.policy >> (8 * cls)) & 3u;
    const uint64_t rel = ts - h.t0;  // wraps for ts < t0, and t0 + span fits in 64 bits
    if (rel >= h.span) {
        oor[0] += dirs & 1u;
        oor[1] += dirs >> 1;
        bin = 0;
        return 0u;
    }
    bin = W1 ? (uint32_t)rel : (uint32_t)divide(rel, h.div);
    return dirs;
}

__device__ __forceinline__ uint32_t route(const HistArgs &h, uint32_t cls, uint64_t ts,
                                          uint32_t &bin, uint32_t oor[2]) {
    return h.w_is_one ? route_w<true>(h, cls, ts, bin, oor) : route_w<false>(h, cls, ts, bin, oor);
}

// Bin the quad's timestamps first (so the 64-bit timestamps are dead before
// the table lookups): bin[j] and bit j of the returned mask for in-window
// records; out-of-window records keep bin 0.
template <bool W1>
__device__ __forceinline__ uint32_t bin_quad(const HistArgs &h, const Quad &Q, uint32_t bin[4]) {
    uint32_t inr = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint64_t rel = Q.ts[j] - h.t0;
        const bool in = rel < h.span;
        bin[j] = in ? (W1 ? (uint32_t)rel : (uint32_t)divide(rel, h.div)) : 0u;
        inr |= (uint32_t)in << j;
    }
    return inr;
}

// Direction bits of a record from its class; a routed record outside the
// window routes nowhere and is counted per direction in a packed word (16
// bits per direction).
__device__ __forceinline__ uint32_t dirs_of_packed(const HistArgs &h, uint32_t cls, bool in_window,
                                                   uint32_t &oorp) {
    const uint32_t dirs = (h.policy >> (8 * cls)) & 3u;
    if (!in_window) {
        oorp += (dirs & 1u) | ((dirs >> 1) << 16);
        return 0u;
    }
    return dirs;
}

// A 64-bit sum kept in shared memory as two 32-bit words and updated with
// native 32-bit atomics: the low word takes the low half of the addend, and
// the carry out of that add (seen in the returned old value) goes to the high
// word with the addend's high half. `hi_extra` is added to the high word too
// (callers pack a count into its upper bits).
__device__ __forceinline__ void smem_add_wide(uint32_t *lo, uint32_t *hi, uint64_t v, uint32_t hi_extra) {
    const uint32_t vl = (uint32_t)v;
    const uint32_t old = atomicAdd(lo, vl);
    const uint32_t carry = (uint32_t)(old + vl < old);
    const uint32_t add_hi = (uint32_t)(v >> 32) + carry + hi_extra;
    if (add_hi) atomicAdd(hi, add_hi);
}

// cc[c] += 1 without dynamic register-array indexing (which would spill to
// local memory).
__device__ __forceinline__ void bump_class(uint32_t cc[4], uint32_t c) {
#pragma unroll
    for (int k = 0; k < 4; ++k) cc[k] += (c == (uint32_t)k) ? 1u : 0u;
}

// Per-thread class and out-of-window counters packed in 16-bit fields of one
// 64-bit word (classes in bits 0-63, four fields) and one 32-bit word (two
// directions); callers drain them into wider counters before 65,536 records.
__device__ __forceinline__ void bump_class_packed(uint64_t &cc, uint32_t c) { cc += 1ull << (16 * c); }

// Warp totals of packed counters added into per-CTA shared counters
// (s_cnt[0..3] classes, s_cnt[4..5] out of window).
__device__ __forceinline__ void drain_packed(uint64_t &cc, uint32_t &oorp, unsigned long long *s_cnt) {
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t v = __reduce_add_sync(kFull, (uint32_t)(cc >> (16 * k)) & 0xFFFFu);
        if (lane == 0 && v) atomicAdd(s_cnt + k, (unsigned long long)v);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const uint32_t v = __reduce_add_sync(kFull, (oorp >> (16 * k)) & 0xFFFFu);
        if (lane == 0 && v) atomicAdd(s_cnt + 4 + k, (unsigned long long)v);
    }
    cc = 0;
    oorp = 0;
}

// Warp totals of the per-thread counters into stats (lane 0 of every warp).
__device__ __forceinline__ void flush_counters(uint64_t *stats, const uint32_t cc[4],
                                               const uint32_t oor[2], bool with_oor) {
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t v = __reduce_add_sync(kFull, cc[k]);
        if (lane == 0 && v) atomicAdd(reinterpret_cast<unsigned long long *>(stats + k), (unsigned long long)v);
    }
    if (with_oor) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            uint32_t v = __reduce_add_sync(kFull, oor[k]);
            if (lane == 0 && v)
                atomicAdd(reinterpret_cast<unsigned long long *>(stats + 4 + k), (unsigned long long)v);
        }
    }
}

__device__ __forceinline__ void gadd(const HistArgs &h, uint32_t d, uint32_t bin, uint32_t c, uint64_t s) {
    if (h.cells) {
        uint64_t *cell = h.cells + 4 * (uint64_t)bin;
        red_add_u64(cell + d, s);
        red_add_u32(reinterpret_cast<uint32_t *>(cell + 2) + d, c);
        return;
    }
    uint32_t *cp = d ? h.cnt[1] : h.cnt[0];
    uint64_t *bp = d ? h.byt[1] : h.byt[0];
    red_add_u32(cp + bin, c);
    red_add_u64(bp + bin, s);
}

}  // namespace sinet

