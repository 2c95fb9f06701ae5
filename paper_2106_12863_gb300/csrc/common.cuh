// Device-side building blocks shared by the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "sinet.h"

namespace sinet {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kNoKey = 0xFFFFFFFFu;  // sentinel update key (bins are < 2^31)
// Upper bound on polling iterations of any device-side wait (~1 s at a few
// hundred ns per poll); a wait that runs out latches SINET_ERR_TIMEOUT.
constexpr uint32_t kSpinLimit = 1u << 22;

// Device status word (one per device, owned by the runtime): the first
// failure wins.
__device__ __forceinline__ void latch_status(uint32_t *status, uint32_t code) {
    atomicCAS(status, 0u, code);
}

// ---------------------------------------------------------------------------
// Division by a run-time invariant divisor w (the bin width), after
// Granlund & Montgomery, "Division by invariant integers using
// multiplication" (PLDI 1994), unsigned N-bit case with N = 64:
//   l = ceil(log2 w), m' = floor(2^64 (2^l - w) / w) + 1,
//   sh1 = min(l, 1), sh2 = max(l - 1, 0),
//   q = (t1 + ((n - t1) >> sh1)) >> sh2 with t1 = mulhi(m', n).
// Exact for every 64-bit n; w = 1 gives m' = 1, sh1 = sh2 = 0.
struct Divider {
    uint64_t m;
    uint32_t sh1, sh2;
};

__device__ __forceinline__ uint64_t divide(uint64_t n, const Divider &d) {
    uint64_t t1 = __umul64hi(d.m, n);
    return (t1 + ((n - t1) >> d.sh1)) >> d.sh2;
}

// ---------------------------------------------------------------------------
// Cache-hinted loads: records are streamed once (evict-first in L2 so the
// histogram lines stay resident; no L1 allocation for the 32-bit streams).

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint4 ld_stream_v4(const void *ptr, uint64_t pol) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ ulonglong2 ld_stream_v2u64(const void *ptr, uint64_t pol) {
    ulonglong2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.u64 {%0,%1}, [%2], %3;"
                 : "=l"(v.x), "=l"(v.y)
                 : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t *ptr, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;"
                 : "=r"(v)
                 : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ uint64_t ld_stream_u64(const uint64_t *ptr, uint64_t pol) {
    uint64_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ uint32_t ld_stream_u8(const uint8_t *ptr) {
    uint16_t v;
    asm volatile("ld.global.nc.u8 %0, [%1];" : "=h"(v) : "l"(ptr));
    return v;
}

// Global-memory reductions (no return value). Written out so that they are
// always RED.global, also where the compiler cannot tell a pointer is global,
// and carry no memory clobber: nothing in a kernel reads the histogram back.
__device__ __forceinline__ void red_add_u32(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v));
}

__device__ __forceinline__ void red_add_u64(uint64_t *p, uint64_t v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v));
}

// ---------------------------------------------------------------------------
// Bulk (TMA engine, non-tensor) copy of a 16-byte-aligned global region into
// shared memory, completed on an mbarrier. Called by all threads of the CTA;
// returns false in every thread (and latches SINET_ERR_TIMEOUT) if the copy
// did not land within the polling bound: the caller must then not classify
// against the shared memory.

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ inline bool stage_to_smem(void *sdst, const void *gsrc, uint32_t bytes, uint64_t *bar,
                                     uint32_t *status) {
    if (bytes == 0) return true;
    const uint32_t b = smem_u32(bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes)
                     : "memory");
        const uint32_t kChunk = 32768;
        for (uint32_t off = 0; off < bytes; off += kChunk) {
            uint32_t sz = bytes - off < kChunk ? bytes - off : kChunk;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(static_cast<char *>(sdst) + off)),
                "l"(static_cast<const char *>(gsrc) + off), "r"(sz), "r"(b)
                : "memory");
        }
    }
    __syncthreads();  // barrier initialised before anyone polls it
    bool ok = false;
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        if (mbar_try_wait(b, 0)) { ok = true; break; }
    }
    if (!ok) {
        latch_status(status, SINET_ERR_TIMEOUT);
        // give the copy in flight a second bounded chance to land before the
        // CTA's shared memory can be reused
        for (uint32_t it = 0; it < kSpinLimit && !mbar_try_wait(b, 0); ++it) {
        }
    }
    // one answer for the whole CTA: a thread whose polls ran out makes every
    // thread treat the staged table as absent
    return __syncthreads_and(ok) != 0;
}

// ---------------------------------------------------------------------------
// Membership of an address in the compiled CIDR list.

// Interval form: sorted disjoint [lo, hi]; the bucket of the top k bits gives
// the candidate range [idx[b], idx[b+1]] (clipped to the last interval); the
// answer is the last candidate with lo <= a, if its hi >= a.
template <typename IdxT>
struct IntervalView {
    const uint32_t *lo;
    const uint32_t *hi;
    const IdxT *idx;
    uint32_t shift;  // 32 - index bits
    uint32_t n_iv;

    __device__ __forceinline__ uint32_t contains(uint32_t a) const {
        const uint32_t bkt = a >> shift;
        uint32_t j = idx[bkt];
        uint32_t e = idx[bkt + 1];
        if (j >= n_iv) return 0u;
        if (e >= n_iv) e = n_iv - 1;
        uint32_t len = e - j + 1;
        while (len > 1) {  // last position with lo <= a (lower-bound style halving)
            uint32_t half = len >> 1;
            if (lo[j + half] <= a) j += half;
            len -= half;
        }
        return (lo[j] <= a) & (a <= hi[j]);
    }
};

// Per-mask-length form: for each length group (most covered addresses
// first), mask the address to that length and binary-search the group's
// sorted canonical networks: the SB == CB comparison of Algorithm 1 against
// every entry of that length at once.
struct PmlView {
    const uint32_t *nets;
    const uint4 *groups;  // {len, offset, count, 0}
    uint32_t n_groups;

    __device__ __forceinline__ uint32_t contains(uint32_t a) const {
        for (uint32_t g = 0; g < n_groups; ++g) {
            const uint4 gr = groups[g];
            const uint32_t m = gr.x ? (0xFFFFFFFFu << (32 - gr.x)) : 0u;
            const uint32_t x = a & m;
            uint32_t j = gr.y, len = gr.z;
            while (len > 1) {
                uint32_t half = len >> 1;
                if (nets[j + half] <= x) j += half;
                len -= half;
            }
            if (nets[j] == x) return 1u;
        }
        return 0u;
    }
};

// Toggle form (shared memory). For the bucket of the top `bits` address bits,
// desc gives the membership of the bucket's first address (bit 31) and the
// blocks holding the ascending offsets t at which membership flips, stored as
// t - 1 (< 2^24; padded with 0x7FFFFFFF): NB = 1, one block (bits 0-14);
// NB = 2, two blocks (bits 0-14, 15-29; the second may be the all-padding
// block 0); NB = 0, consecutive blocks (bits 0-23 first, 24-27 count). A
// toggle lies at or below the address's offset `off` exactly when
// (t - 1) - off is negative as a 32-bit signed value, so the XOR of the four
// differences (and of desc, for the start state) carries the membership in
// bit 31. Pure buckets use block 0, so for NB = 1, 2 every lookup is the same
// branch-free sequence of loads and integer operations.
template <int NB>  // 1 or 2 blocks per bucket, loaded unconditionally; 0: as counted
struct ToggleView {
    const uint4 *blocks;
    const uint32_t *desc;
    uint32_t shift;     // 32 - bits
    uint32_t off_mask;  // (1 << shift) - 1

    static __device__ __forceinline__ uint32_t parity_bits(const uint4 &b, uint32_t off) {
        return (b.x - off) ^ (b.y - off) ^ (b.z - off) ^ (b.w - off);
    }

    template <int N>
    __device__ __forceinline__ void contains_n(const uint32_t (&a)[N], uint32_t (&in)[N]) const {
        uint32_t d[N];
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] = desc[a[i] >> shift];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const uint32_t off = a[i] & off_mask;
            uint32_t x;
            if (NB == 0) {
                const uint4 *bp = blocks + (d[i] & 0xFFFFFFu);
                x = parity_bits(bp[0], off) ^ d[i];
                if (d[i] & 0x0E000000u) {  // more than one block (rare)
                    const uint32_t nb = (d[i] >> 24) & 0xFu;
                    for (uint32_t k = 1; k < nb; ++k) x ^= parity_bits(bp[k], off);
                }
            } else {
                // block 0 is all padding, and four equal differences XOR to
                // zero, so a pure bucket (or an unused second index) needs no
                // load: skipping it saves the shared-memory wavefronts
                x = d[i];
                const uint32_t b1 = d[i] & 0x7FFFu;
                if (b1) x ^= parity_bits(blocks[b1], off);
                if (NB == 2) {
                    const uint32_t b2 = (d[i] >> 15) & 0x7FFFu;
                    if (b2) x ^= parity_bits(blocks[b2], off);
                }
            }
            in[i] = x >> 31;
        }
    }
};

// Device description of a staged table (byte offsets inside the image).
struct TableArgs {
    const uint8_t *image;     // device image base
    uint32_t iv_bytes;        // [blocks | desc] staged for the toggle form
    uint32_t off_blocks, off_desc, desc_bits, toggle_form;
    uint32_t off_lo, off_hi, off_idx32;  // global-memory interval form
    uint32_t n_iv, index_bits;
    uint32_t off_nets, off_groups, pml_bytes, n_groups;
};

// ---------------------------------------------------------------------------
// Record geometry: quads of 4 records start at index `shift + 4 q`
// (shift in {-3..0}) so that every full quad is 16-byte aligned in every
// stream; the first and last quads may be partial and use scalar loads.
struct QuadGeom {
    uint64_t n;      // records
    uint64_t quads;  // number of quads
    int32_t shift;   // index of quad 0's first record (<= 0)
    int32_t vec;     // 1 if full quads may use vector loads
};

__device__ __forceinline__ int64_t quad_base(const QuadGeom &g, uint64_t q) {
    return (int64_t)g.shift + 4 * (int64_t)q;
}

__device__ __forceinline__ bool quad_full(const QuadGeom &g, int64_t base) {
    return g.vec && base >= 0 && (uint64_t)base + 4 <= g.n;
}

}  // namespace sinet
