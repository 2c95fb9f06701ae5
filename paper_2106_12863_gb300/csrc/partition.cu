// Hot/cold partitioned histogram update (SINET_STRAT_PARTITION), for
// unsorted, skewed records over a histogram far larger than L2.
//
// The update step of Section 5 (per-direction <timestamp, count> and
// <timestamp, bytes> sums) split by how often a bin is hit. A bin hit often
// lives in shared memory for the whole pass; a bin hit rarely is handled by a
// bucketed two-level partition whose second level stays in L2, so every
// output bin is stored once with plain stores and no sector of the histogram
// is ever read-modified-written in DRAM. See partition.h for the sequence.
#include <algorithm>

#include "combine.cuh"
#include "partition.h"

namespace sinet {

namespace {

// Fibonacci hashing: the top bits of bin * 2^32 / phi spread any run of bins
__device__ __forceinline__ uint32_t fib_hash(uint32_t b) { return b * 0x9E3779B1u; }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait for the phase of `bar` with parity `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// TMA bulk copy (non-tensor) of `bytes` from global memory into this CTA's
// shared memory, completing on `bar`; 16-byte aligned ends, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t vload(const uint32_t *p) { return *reinterpret_cast<const volatile uint32_t *>(p); }

// Sample counts: linear probing over the open-addressing table. A key that
// finds no slot within the probe bound is dropped: the sample only ranks
// bins, it is not part of the result.
__device__ void hash_add(const PartDev &p, uint32_t key, uint32_t c) {
    uint32_t s = fib_hash(key) >> p.hash_shift;
    for (int probe = 0; probe < 64; ++probe) {
        uint32_t k = vload(p.hash_keys + s);
        if (k == kNoKey) {
            k = atomicCAS(p.hash_keys + s, kNoKey, key);
            if (k == kNoKey) k = key;
        }
        if (k == key) {
            atomicAdd(p.hash_cnt + s, c);
            return;
        }
        s = (s + 1) & p.hash_mask;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// 1. Sample: every sample_stride-th chunk of kPartSampleChunk records is
// classified and binned; hits per bin (both directions together) are
// pre-aggregated in a per-CTA shared-memory cache, then counted in the hash.
template <int LK>
__global__ void __launch_bounds__(256) k_part_sample(RecArgs r, TableArgs t, HistArgs h, PartDev p,
                                                     uint32_t *status) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t bar;
    Classifier<LK> C;
    if (!C.init(t, smem, &bar, status)) return;
    uint8_t *cm = smem + ((Classifier<LK>::smem_bytes(t) + 15u) & ~15u);
    const uint32_t slots = HotCache::kWays << kPartSampleSetBits;
    HotCache hc;
    hc.keys = reinterpret_cast<uint32_t *>(cm);
    hc.cnt = hc.keys + slots;
    hc.lo = hc.cnt + slots;
    hc.hi = hc.lo + slots;
    hc.set_bits = kPartSampleSetBits;
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
        hc.keys[i] = kNoKey;
        hc.cnt[i] = 0;
        hc.lo[i] = 0;
        hc.hi[i] = 0;
    }
    __syncthreads();
    const uint64_t pol = policy_evict_first();
    const uint64_t qpc = kPartSampleChunk / 4;
    const uint64_t total = p.sample_chunks * qpc;
    uint32_t oor[2] = {0, 0};
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total;
         w += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q = (w / qpc) * p.sample_stride * qpc + w % qpc;
        Quad Q;
        load_quad<true, true, true, false>(r, q, pol, Q);
        classify_quad<LK>(C, Q);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!(Q.valid >> j & 1u)) continue;
            uint32_t bin;
            const uint32_t dirs = route(h, Q.cls[j], Q.ts[j], bin, oor);
            if (!dirs) continue;
            const uint32_t c = __popc(dirs);
            if (!hc.add(bin, c, 0)) hash_add(p, bin, c);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x)
        if (hc.cnt[i]) hash_add(p, hc.keys[i], hc.cnt[i]);
}

// 2a. Hash slots per log2 of their sample count.
__global__ void __launch_bounds__(256) k_part_levels(PartDev p) {
    __shared__ uint32_t s[32];
    if (threadIdx.x < 32) s[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= p.hash_mask; i += gridDim.x * blockDim.x) {
        const uint32_t c = p.hash_cnt[i];
        if (c) atomicAdd(&s[31 - __clz(c)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32 && s[threadIdx.x]) atomicAdd(p.levels + threadIdx.x, s[threadIdx.x]);
}

// 2a'. Total sample hits (levels[32]), for the replication threshold.
__global__ void __launch_bounds__(256) k_part_total(PartDev p) {
    uint32_t t = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= p.hash_mask; i += gridDim.x * blockDim.x)
        t += p.hash_cnt[i];
    t = __reduce_add_sync(kFull, t);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(p.levels + 32, t);
}

// 2b. Candidates: the bins of the highest count levels that together hold at
// most kPartMaxCand bins.
__global__ void __launch_bounds__(256) k_part_collect(PartDev p) {
    __shared__ uint32_t s_min;
    if (threadIdx.x == 0) {
        uint32_t cum = 0, lowest = 32;
        for (int l = 31; l >= 0; --l) {
            cum += p.levels[l];
            if (cum > kPartMaxCand) break;
            lowest = (uint32_t)l;
        }
        s_min = lowest < 32 ? (1u << lowest) : 0xFFFFFFFFu;
    }
    __syncthreads();
    const uint32_t thr = s_min;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n_slots = p.hash_mask + 1;
    // warp-uniform trip count for the ballot
    for (uint32_t i0 = (blockIdx.x * blockDim.x + threadIdx.x) - lane; i0 < n_slots;
         i0 += gridDim.x * blockDim.x) {
        const uint32_t i = i0 + lane;
        const uint32_t c = i < n_slots ? p.hash_cnt[i] : 0u;
        const bool take = c != 0 && c >= thr;
        const uint32_t m = __ballot_sync(kFull, take);
        if (!m) continue;
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(p.cand_n, (uint32_t)__popc(m));
        base = __shfl_sync(kFull, base, 0);
        if (take) {
            const uint32_t pos = base + __popc(m & ((1u << lane) - 1u));
            if (pos < kPartMaxCand) p.cand[pos] = make_uint2(p.hash_keys[i], c);
        }
    }
}

// 2c. The hot table (one CTA): candidates are inserted level by level, the
// highest sample counts first, each into the first free way of its set; a
// candidate whose set is full stays cold.
__global__ void __launch_bounds__(1024) k_part_build(PartDev p, uint32_t slots) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *keys = reinterpret_cast<uint32_t *>(smem);
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) keys[i] = kNoKey;
    const uint32_t n = min(*p.cand_n, kPartMaxCand);
    constexpr int K = kPartMaxCand / 1024;
    uint32_t key[K], lev[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint32_t i = threadIdx.x + 1024u * k;
        const uint2 c = i < n ? p.cand[i] : make_uint2(kNoKey, 0u);
        key[k] = c.x;
        lev[k] = c.y ? 31 - __clz(c.y) : 0u;
    }
    __syncthreads();
    const uint32_t shift = 32 - p.set_bits;
    // bins with at least 1/64 of the sampled updates take all four ways of
    // their set (when it is free): the main pass spreads lanes over them
    const uint32_t total = p.levels[32];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (key[k] == kNoKey) continue;
        const uint32_t i = threadIdx.x + 1024u * k;
        if ((uint64_t)p.cand[i].y * 64 < (uint64_t)total || total == 0) continue;
        uint32_t *set = keys + 4 * (fib_hash(key[k]) >> shift);
        if (atomicCAS(set, kNoKey, key[k]) != kNoKey) continue;
        set[1] = set[2] = set[3] = key[k];  // the first way claimed the set; nobody else writes here yet
        key[k] = kNoKey;                    // placed
    }
    __syncthreads();
    for (int l = 31; l >= 0; --l) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (key[k] == kNoKey || lev[k] != (uint32_t)l) continue;
            uint32_t *set = keys + 4 * (fib_hash(key[k]) >> shift);
            bool placed = false;
            for (int w = 0; w < 4 && !placed; ++w) placed = atomicCAS(set + w, kNoKey, key[k]) == kNoKey;
            // a full set whose later ways repeat way 0 (a replicated bin)
            // gives one of the copies up: a hot bin that shares its set with
            // a replicated one must not fall to the cold path (way 0 keeps the
            // replicated bin, whose probe then finds it there)
            const uint32_t k0 = set[0];
            for (int w = 3; w >= 1 && !placed && k0 != kNoKey; --w) placed = atomicCAS(set + w, k0, key[k]) == k0;
        }
        __syncthreads();
    }
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) p.hot_keys[i] = keys[i];
}

// ---------------------------------------------------------------------------
// 3. Main pass.

namespace {

// Per-CTA state of the main pass, all in shared memory.
struct MainSmem {
    const uint32_t *hkeys;  // [slots]
    uint32_t *hcnt;         // [2][slots]
    uint32_t *hlo;          // [2][slots] byte sums, low words
    uint32_t *hhi;          // [2][slots] byte sums, high words
    uint64_t *slot;         // [n_buckets][4] page index << 32 | page id of the last four overflow pages
    uint32_t *cur;          // [n_buckets] cold entries appended so far
    uint32_t slots;
    uint32_t shift;         // 32 - set_bits
    uint32_t rbase;         // first page of this CTA's region: blockIdx.x * n_buckets * creg
    uint32_t quiet;         // positions below this need no overflow page: creg * kPartPage - kPartPage / 2
};

// Page k of bucket bk's overflow, taken from the pool's shared part (page
// ids from dyn_base on), into its slot.
__device__ __forceinline__ void alloc_overflow(const PartDev &p, const MainSmem &m, uint32_t bk, uint32_t k,
                                            uint32_t *status) {
    const uint32_t nxt = p.dyn_base + atomicAdd(p.page_alloc, 1u);
    if (nxt < p.pages_cap) {
        p.page_bucket[nxt] = bk;
        p.page_fill[nxt] = kPartPage;
    } else {
        latch_status(status, SINET_ERR_BUDGET);
    }
    reinterpret_cast<volatile uint64_t *>(m.slot)[4 * bk + (k & 3)] = (uint64_t)k << 32 | nxt;
}

// Append one cold entry (key = bin << 1 | direction, the record's bytes) to
// the CTA's current page of the bin's bucket. Positions come from a
// shared-memory counter. Pages 0 .. creg - 1 of every bucket are the CTA's
// own region of the pool, their ids fixed by CTA, bucket and page index.
// Later pages (overflow) come from the pool's shared part: the thread that
// takes the middle position of page k - 1 allocates page k, so the page a
// position falls in is (almost) always ready. Four slots per bucket keep
// (page index, page id) of the current overflow pages in one 64-bit word
// each, written and read whole, so no fence is needed: a thread holds at most
// one claimed position at a time, so the claimed but unwritten positions (at
// most one per thread) stay within two pages and a slot is never reused while
// a thread still needs it.
__device__ __forceinline__ void cold_emit_entry(const PartDev &p, const MainSmem &m, uint64_t e, uint32_t *status) {
    const uint32_t bk = (uint32_t)(e >> 33) >> p.cb_shift;
    const uint32_t pos = atomicAdd(m.cur + bk, 1u);
    const uint32_t pg = pos >> kPartPageBits, off = pos & (kPartPage - 1);
    uint32_t id = m.rbase + bk * p.creg + pg;
    if (pos >= m.quiet) {  // from the middle of the region's last page on
        if (off == kPartPage / 2) alloc_overflow(p, m, bk, pg + 1, status);
        if (pg >= p.creg) {
            volatile uint64_t *sl = m.slot + 4 * bk;
            uint64_t v = sl[pg & 3];
            for (uint32_t k = 0; (uint32_t)(v >> 32) != pg; ++k) {
                if (k > kSpinLimit) {
                    latch_status(status, SINET_ERR_TIMEOUT);
                    return;
                }
                v = sl[pg & 3];
            }
            id = (uint32_t)v;
            if (id >= p.pages_cap) return;
        }
    }
    p.pages[(uint64_t)id * kPartPage + off] = e;
}

__device__ __forceinline__ void cold_emit(const PartDev &p, const MainSmem &m, uint32_t key, uint32_t by,
                                          uint32_t *status) {
    cold_emit_entry(p, m, (uint64_t)key << 32 | by, status);
}

// One routed, in-window record: both directions share the bin's hot slot.
__device__ __forceinline__ void part_update(const PartDev &p, const MainSmem &m, uint32_t bin, uint32_t dirs,
                                            uint32_t by, uint32_t *status) {
    const uint32_t set = fib_hash(bin) >> m.shift;
    const uint4 k4 = *reinterpret_cast<const uint4 *>(m.hkeys + 4 * set);
    // a bin holding all four ways of its set is one of the very hottest:
    // lanes spread over its four copies, which cuts same-address atomics
    const int way = (k4.x == bin && k4.w == bin) ? (int)(threadIdx.x & 3u)
                    : k4.x == bin ? 0 : k4.y == bin ? 1 : k4.z == bin ? 2 : k4.w == bin ? 3 : -1;
    if (way >= 0) {
        const uint32_t i = 4 * set + (uint32_t)way;
        if (dirs & 1u) {
            atomicAdd(m.hcnt + i, 1u);
            smem_add_wide(m.hlo + i, m.hhi + i, by, 0u);
        }
        if (dirs & 2u) {
            const uint32_t j = m.slots + i;
            atomicAdd(m.hcnt + j, 1u);
            smem_add_wide(m.hlo + j, m.hhi + j, by, 0u);
        }
        return;
    }
    if (dirs & 1u) cold_emit(p, m, bin << 1, by, status);
    if (dirs & 2u) cold_emit(p, m, bin << 1 | 1u, by, status);
}

template <bool W1>
__device__ __forceinline__ void part_record(const HistArgs &h, const PartDev &p, const MainSmem &m, uint64_t ts,
                                            uint32_t by, uint32_t cls, uint64_t &ccp, uint32_t &oorp,
                                            uint32_t *status) {
    bump_class_packed(ccp, cls);
    const uint64_t rel = ts - h.t0;
    const bool inw = rel < h.span;
    const uint32_t bin = inw ? (W1 ? (uint32_t)rel : (uint32_t)divide(rel, h.div)) : 0u;
    const uint32_t dirs = dirs_of_packed(h, cls, inw, oorp);
    if (dirs) part_update(p, m, bin, dirs, by, status);
}

// The staged path's pieces, for two records per thread and warp-wide steps.

// Hot-table slot of a bin, or kNoKey, without branches: w has bit i set
// when way i holds the bin; a replicated set (all four ways hold one of the
// very hottest bins) spreads its lanes over the four copies.
__device__ __forceinline__ uint32_t hot_slot(const MainSmem &m, uint32_t bin) {
    const uint32_t set = fib_hash(bin) >> m.shift;
    const uint4 k4 = *reinterpret_cast<const uint4 *>(m.hkeys + 4 * set);
    const uint32_t w = (uint32_t)(k4.x == bin) | (uint32_t)(k4.y == bin) << 1 | (uint32_t)(k4.z == bin) << 2 |
                       (uint32_t)(k4.w == bin) << 3;
    const uint32_t way = w == 15u ? (threadIdx.x & 3u) : (uint32_t)(__ffs(w) - 1);
    return w ? 4 * set + way : kNoKey;
}

__device__ __forceinline__ void hot_add(const MainSmem &m, uint32_t slot, uint32_t d, uint32_t by) {
    const uint32_t i = d * m.slots + slot;
    atomicAdd(m.hcnt + i, 1u);
    smem_add_wide(m.hlo + i, m.hhi + i, by, 0u);
}

// First direction of a routed record: outgoing when its class routes there.
__device__ __forceinline__ uint32_t first_dir(uint32_t dirs) { return (dirs & 1u) ? 0u : 1u; }

__device__ __forceinline__ uint64_t cold_entry(uint32_t bin, uint32_t d, uint32_t by) {
    return (uint64_t)(bin << 1 | d) << 32 | by;
}

// Warp totals of 8-bit class counters and 16-bit out-of-window counters
// into the CTA's counters.
__device__ __forceinline__ void drain8(uint32_t &cc8, uint32_t &oorp, unsigned long long *s_cnt) {
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t v = __reduce_add_sync(kFull, (cc8 >> (8 * k)) & 0xFFu);
        if (lane == 0 && v) atomicAdd(s_cnt + k, (unsigned long long)v);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const uint32_t v = __reduce_add_sync(kFull, (oorp >> (16 * k)) & 0xFFFFu);
        if (lane == 0 && v) atomicAdd(s_cnt + 4 + k, (unsigned long long)v);
    }
    cc8 = 0;
    oorp = 0;
}

}  // namespace

// One CTA per SM: warp 31 issues TMA bulk copies of stage after stage (a
// chunk of kPartStageRecords records of each stream: ts, src, dst, bytes);
// warps 0-30 take one record per thread from each of two stages, release
// them, and classify, bin and update. Chunks go to CTAs round-robin.
template <int LK, bool W1>
__global__ void __launch_bounds__(kPartThreads, 1) k_part_main(RecArgs r, TableArgs t, HistArgs h, PartDev p,
                                                               uint32_t *status) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ uint64_t tbar;
    __shared__ uint64_t full_bar[kPartStages], empty_bar[kPartStages];
    __shared__ unsigned long long s_cnt[6];
    __shared__ uint32_t s_abort;
    Classifier<LK> C;
    if (!C.init(t, smem, &tbar, status)) return;  // table not staged: the status word says so
    const uint32_t tsm = (Classifier<LK>::smem_bytes(t) + 127u) & ~127u;
    uint8_t *stage = smem + tsm;
    MainSmem m;
    m.slots = 4u << p.set_bits;
    m.shift = 32 - p.set_bits;
    m.rbase = blockIdx.x * p.n_buckets * p.creg;
    m.quiet = p.creg * kPartPage - kPartPage / 2;
    uint32_t *hk = reinterpret_cast<uint32_t *>(stage + kPartStages * kPartStageBytes);
    m.hkeys = hk;
    m.hcnt = hk + m.slots;
    m.hlo = m.hcnt + 2 * m.slots;
    m.hhi = m.hlo + 2 * m.slots;
    m.slot = reinterpret_cast<uint64_t *>(m.hhi + 2 * m.slots);  // 8-byte aligned: slots % 4 == 0
    m.cur = reinterpret_cast<uint32_t *>(m.slot + 4 * p.n_buckets);
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = tid; i < m.slots; i += blockDim.x) hk[i] = p.hot_keys[i];
    for (uint32_t i = tid; i < 2 * m.slots; i += blockDim.x) {
        m.hcnt[i] = 0;
        m.hlo[i] = 0;
        m.hhi[i] = 0;
    }
    for (uint32_t b = tid; b < p.n_buckets; b += blockDim.x) {
        m.cur[b] = 0;
        m.slot[4 * b] = m.slot[4 * b + 1] = m.slot[4 * b + 2] = m.slot[4 * b + 3] = ~0ull;
    }
    if (tid < 6) s_cnt[tid] = 0;
    if (tid == 0) {
        s_abort = 0;
        for (uint32_t s = 0; s < kPartStages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), kPartConsumers / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const uint32_t warp = tid >> 5, lane = tid & 31;
    constexpr uint32_t R = kPartStageRecords;
    if (warp == kPartConsumers / 32) {
        // producer
        if (lane == 0) {
            uint64_t it = 0;
            for (;; ++it) {
                const uint64_t ch = blockIdx.x + it * gridDim.x;
                if (ch >= p.n_full) break;
                const uint32_t s = (uint32_t)(it % kPartStages);
                if (it >= kPartStages &&
                    !mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)((it / kPartStages) - 1) & 1u)) {
                    latch_status(status, SINET_ERR_TIMEOUT);
                    *reinterpret_cast<volatile uint32_t *>(&s_abort) = 1;
                    break;
                }
                if (vload(&s_abort)) break;
                // the consumers' reads of this stage precede the copy's writes
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const uint64_t i0 = p.i_lo + ch * R;
                const uint32_t fb = smem_u32(&full_bar[s]);
                const uint32_t sb = smem_u32(stage + s * kPartStageBytes);
                mbar_expect_tx(fb, kPartStageBytes);
                bulk_g2s(sb, r.ts + i0, 8 * R, fb);
                bulk_g2s(sb + 8 * R, r.src + i0, 4 * R, fb);
                bulk_g2s(sb + 12 * R, r.dst + i0, 4 * R, fb);
                bulk_g2s(sb + 16 * R, r.bytes + i0, 4 * R, fb);
            }
            // every copy issued has landed before the CTA can exit
            for (uint64_t k = it > kPartStages ? it - kPartStages : 0; k < it; ++k)
                mbar_wait(smem_u32(&full_bar[k % kPartStages]), (uint32_t)(k / kPartStages) & 1u);
        }
    } else {
        uint32_t cc8 = 0;   // per-thread class counts, 8-bit fields
        uint32_t oorp = 0;  // per-thread out-of-window counts, 16-bit fields
        uint32_t since = 0;
        // one stage per iteration: records 2 * tid and 2 * tid + 1 of the chunk
        static_assert(kPartRPT == 2, "two records per consumer thread and stage");
        for (uint64_t q = 0;; ++q) {
            const uint64_t ch0 = blockIdx.x + q * gridDim.x;
            if (ch0 >= p.n_full) break;
            uint64_t ts[2] = {0, 0};
            uint32_t a[4] = {0, 0, 0, 0}, by[2] = {0, 0};  // a: src, dst of record 0, then of record 1
            const uint32_t s = (uint32_t)(q % kPartStages);
            const bool ok = __all_sync(kFull, mbar_wait(smem_u32(&full_bar[s]), (uint32_t)(q / kPartStages) & 1u));
            if (ok) {
                const uint8_t *sp = stage + s * kPartStageBytes;
                const uint4 t2 = *reinterpret_cast<const uint4 *>(sp + 16 * tid);
                const uint2 s2 = *reinterpret_cast<const uint2 *>(sp + 8 * R + 8 * tid);
                const uint2 d2 = *reinterpret_cast<const uint2 *>(sp + 12 * R + 8 * tid);
                const uint2 b2 = *reinterpret_cast<const uint2 *>(sp + 16 * R + 8 * tid);
                ts[0] = (uint64_t)t2.y << 32 | t2.x;
                ts[1] = (uint64_t)t2.w << 32 | t2.z;
                a[0] = s2.x;
                a[1] = d2.x;
                a[2] = s2.y;
                a[3] = d2.y;
                by[0] = b2.x;
                by[1] = b2.y;
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&empty_bar[s]));
            }
            if (!ok) {
                if (lane == 0) {
                    latch_status(status, SINET_ERR_TIMEOUT);
                    *reinterpret_cast<volatile uint32_t *>(&s_abort) = 1;
                }
                break;
            }
            uint32_t in[4];
            C.template in_n_warp<4>(a, in);  // the warp is converged here
            uint32_t bin[2], dirs[2], slot[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const uint32_t cls = in[2 * j] | in[2 * j + 1] << 1;
                cc8 += 1u << (8 * cls);
                const uint64_t rel = ts[j] - h.t0;
                const bool inw = rel < h.span;
                bin[j] = inw ? (W1 ? (uint32_t)rel : (uint32_t)divide(rel, h.div)) : 0u;
                uint32_t d = (h.policy >> (8 * cls)) & 3u;
                if (!inw) {
                    oorp += (d & 1u) | ((d >> 1) << 16);
                    d = 0;
                }
                dirs[j] = d;
                slot[j] = d ? hot_slot(m, bin[j]) : kNoKey;
            }
            // hot bins, first direction: one shared-memory add per record
#pragma unroll
            for (int j = 0; j < 2; ++j)
                if (slot[j] != kNoKey) hot_add(m, slot[j], first_dir(dirs[j]), by[j]);
            // classes routed to both directions: the second one
            if (h.two_dir && __any_sync(kFull, dirs[0] == 3u || dirs[1] == 3u)) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    if (dirs[j] != 3u) continue;
                    if (slot[j] != kNoKey) hot_add(m, slot[j], 1u, by[j]);
                    else cold_emit_entry(p, m, cold_entry(bin[j], 1u, by[j]), status);
                }
            }
            // cold bins, first direction: each lane appends its own entries (a
            // gather of the warp's entries onto its lanes first costs more
            // instructions than the second append it saves)
#pragma unroll
            for (int j = 0; j < 2; ++j)
                if (dirs[j] && slot[j] == kNoKey) cold_emit_entry(p, m, cold_entry(bin[j], first_dir(dirs[j]), by[j]), status);
            // at most two records per field per iteration: drain before 8 bits fill
            if (++since == 127) {
                drain8(cc8, oorp, s_cnt);
                since = 0;
            }
        }
        uint64_t ccp = 0;  // the records outside the staged chunks: 16-bit class fields
        // records outside the staged chunks, one by one
        const uint64_t tail_lo = p.i_lo + p.n_full * R;
        const uint64_t n_scalar = p.n_head + (r.g.n - tail_lo);
        for (uint64_t k = (uint64_t)blockIdx.x * kPartConsumers + tid; k < n_scalar;
             k += (uint64_t)gridDim.x * kPartConsumers) {
            const uint64_t i = k < p.n_head ? k : tail_lo + (k - p.n_head);
            uint32_t a[1] = {r.src[i]}, in_s[1], in_d[1];
            C.template in_n<1>(a, in_s);
            a[0] = r.dst[i];
            C.template in_n<1>(a, in_d);
            part_record<W1>(h, p, m, r.ts[i], r.bytes[i], in_s[0] | in_d[0] << 1, ccp, oorp, status);
        }
        __syncwarp();
        drain_packed(ccp, oorp, s_cnt);
        drain8(cc8, oorp, s_cnt);
    }
    __syncthreads();

    // class and out-of-window counters
    if (tid < 6 && s_cnt[tid]) atomicAdd(reinterpret_cast<unsigned long long *>(h.stats) + tid, s_cnt[tid]);
    // this CTA's share of the hot table
    for (uint32_t i = tid; i < m.slots; i += blockDim.x) {
        if (hk[i] == kNoKey) continue;
#pragma unroll
        for (uint32_t d = 0; d < 2; ++d) {
            const uint32_t j = d * m.slots + i;
            const uint32_t c = m.hcnt[j];
            if (c) {
                red_add_u32(p.hot_cnt + j, c);
                red_add_u64(p.hot_bytes + j, (uint64_t)m.hhi[j] << 32 | m.hlo[j]);
            }
        }
    }
    // fills: every page of the region, then each bucket's last two overflow
    // pages (every earlier overflow page is full)
    for (uint32_t i = tid; i < p.n_buckets * p.creg; i += blockDim.x) {
        const uint32_t b = i / p.creg, k = i - b * p.creg;
        const int64_t f = (int64_t)m.cur[b] - (int64_t)k * kPartPage;
        p.page_bucket[m.rbase + i] = b;
        p.page_fill[m.rbase + i] = (uint32_t)(f < 0 ? 0 : f > kPartPage ? kPartPage : f);
    }
    for (uint32_t b = tid; b < p.n_buckets; b += blockDim.x) {
        const uint32_t E = m.cur[b];
        const uint32_t ka = E > kPartPage / 2 ? ((E - kPartPage / 2 - 1) >> kPartPageBits) + 1 : 0u;
        for (uint32_t k = ka ? ka - 1 : 0; k <= ka; ++k) {
            if (k < p.creg) continue;
            const uint64_t v = m.slot[4 * b + (k & 3)];
            if ((uint32_t)(v >> 32) != k) continue;
            const uint32_t id = (uint32_t)v;
            const int64_t f = (int64_t)E - (int64_t)k * kPartPage;
            if (id < p.pages_cap) p.page_fill[id] = (uint32_t)(f < 0 ? 0 : f > kPartPage ? kPartPage : f);
        }
    }
}

// ---------------------------------------------------------------------------
// 4. Pages grouped by bucket: counts, their scan, the lists. A page is
// listed when it holds entries (a region page a CTA left unused has fill 0).
__device__ __forceinline__ bool page_listed(const PartDev &p, uint32_t id) {
    const uint32_t f = p.page_fill[id];
    return f != 0 && f <= kPartPage && p.page_bucket[id] < p.n_buckets;
}

__global__ void __launch_bounds__(256) k_part_count_pages(PartDev p) {
    __shared__ uint32_t s[kPartMaxBuckets];
    for (uint32_t i = threadIdx.x; i < p.n_buckets; i += blockDim.x) s[i] = 0;
    __syncthreads();
    const uint32_t n = (uint32_t)min((uint64_t)p.dyn_base + *p.page_alloc, (uint64_t)p.pages_cap);
    for (uint32_t id = blockIdx.x * blockDim.x + threadIdx.x; id < n; id += gridDim.x * blockDim.x)
        if (page_listed(p, id)) atomicAdd(&s[p.page_bucket[id]], 1u);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < p.n_buckets; i += blockDim.x)
        if (s[i]) atomicAdd(p.bucket_cnt + i, s[i]);
}

__global__ void __launch_bounds__(kPartMaxBuckets) k_part_scan_pages(PartDev p) {
    __shared__ uint32_t s[kPartMaxBuckets + 1];
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (uint32_t b = 0; b < p.n_buckets; ++b) {
            s[b] = acc;
            acc += p.bucket_cnt[b];
        }
        s[p.n_buckets] = acc;
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b <= p.n_buckets; b += blockDim.x) p.bucket_pg[b] = s[b];
    for (uint32_t b = threadIdx.x; b < p.n_buckets; b += blockDim.x) p.bucket_cnt[b] = 0;  // cursors
}

__global__ void __launch_bounds__(256) k_part_list_pages(PartDev p) {
    const uint32_t n = (uint32_t)min((uint64_t)p.dyn_base + *p.page_alloc, (uint64_t)p.pages_cap);
    for (uint32_t id = blockIdx.x * blockDim.x + threadIdx.x; id < n; id += gridDim.x * blockDim.x) {
        if (!page_listed(p, id)) continue;
        const uint32_t b = p.page_bucket[id];
        const uint32_t pos = atomicAdd(p.bucket_cnt + b, 1u);
        p.page_list[p.bucket_pg[b] + pos] = id;
    }
}

// ---------------------------------------------------------------------------
// 5. Cold pass (cooperative: every CTA resident). CTA o owns bins
// [o * own_bins, (o + 1) * own_bins) of every bucket. Its page-sorting groups
// sort the pages of bucket after bucket by owner, a bucket's pages handed out
// one at a time from a per-bucket cursor to whichever group asks next (so
// every group ends its share of a bucket at about the same time); its
// reducing warps follow, summing bucket b once every group of every CTA has
// sorted it (k_part_cold below).

namespace {

constexpr uint32_t kColdThreads = 1024;  // threads of a cold-pass CTA: SG sorting groups, then reducers
constexpr uint32_t kSortThreads = 256;   // threads of one page-sorting group
constexpr uint32_t kReduceBar = 15;      // named barrier of the reducing warps
constexpr uint32_t kSortAhead = 8;       // buckets the sorting groups may run ahead of the reducers

// One page-sorting group's shared state: two page buffers (the copy of the
// next page lands in one while the page in the other is sorted in place) and
// the owner counts of each.
struct GroupSmem {
    uint64_t *buf;      // [2][kPartPage] (addressed by offset, never by a runtime array index,
                        // which would put the struct in local memory)
    uint32_t *ocnt;     // [2][ow] owner counts, then run offsets
    uint32_t ow;        // words of one owner-count array
    uint64_t *bar;      // [2] page copies
    uint32_t *s_id;     // [2] page id of the copy in flight into buf[k]
    uint32_t *s_fill;   // [2] its entries
    uint32_t *s_next;   // list position of the group's next page
    uint32_t *s_flag;   // a wait that ran out
    uint32_t g;         // group index (named barrier 1 + g)
};

__device__ __forceinline__ void group_sync(uint32_t g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kSortThreads) : "memory");
}

template <uint32_t NR>
__device__ __forceinline__ void reduce_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(kReduceBar), "n"(NR) : "memory");
}

// Exclusive prefix sum of v across the (converged) warp.
__device__ __forceinline__ uint32_t warp_exclusive(uint32_t v, uint32_t lane) {
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, d);
        if (lane >= (uint32_t)d) incl += y;
    }
    return incl - v;
}

// One thread of the group: start the TMA copy of the page at list position j into buf[k].
__device__ __forceinline__ void issue_page(const PartDev &p, const GroupSmem &gs, uint32_t j, uint32_t k) {
    const uint32_t id = p.page_list[j];
    const uint32_t fill = p.page_fill[id];
    gs.s_id[k] = id;
    gs.s_fill[k] = fill;
    const uint32_t bytes = (fill * 8u + 15u) & ~15u;  // within the 16 KB page
    const uint32_t bar = smem_u32(gs.bar + k);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier accesses of buf[k] first
    mbar_expect_tx(bar, bytes);
    if (bytes) bulk_g2s(smem_u32(gs.buf + k * kPartPage), p.pages + (uint64_t)id * kPartPage, bytes, bar);
}

// One thread of the group: claim bucket b's next unsorted page and start its
// copy into buf[k]. Returns its list position (the bucket's end or beyond
// when every page is taken).
__device__ __forceinline__ uint32_t claim_page(const PartDev &p, const GroupSmem &gs, uint32_t b, uint32_t k) {
    const uint32_t j = p.bucket_pg[b] + atomicAdd(p.pg_next + b, 1u);
    if (j < p.bucket_pg[b + 1]) issue_page(p, gs, j, k);
    return j;
}

// This group's pages of bucket b, each sorted by owner in place with its
// owner run offsets recorded (its row of idx), then the group counts itself
// done with the bucket. Four group barriers per page: the copy has landed;
// owners counted; offsets scanned; entries scattered (the claim and copy of
// the next page, into the other buffer, run during the scan). `seq` counts
// the group's pages over all buckets (buffer and phase). Returns false when a
// page copy's wait ran out.
__device__ __forceinline__ bool sort_pages(const PartDev &p, const GroupSmem &gs, uint32_t b, uint32_t &seq,
                                           uint32_t *status) {
    constexpr uint32_t GT = kSortThreads;
    constexpr int U = kPartPage / GT;
    const uint32_t G = p.g_cold, tid = threadIdx.x % GT, lane = tid & 31;
    const uint32_t bmask = (1u << p.cb_shift) - 1u, end = p.bucket_pg[b + 1];
    volatile uint32_t *s_next = gs.s_next;
    if (tid == 0) *s_next = claim_page(p, gs, b, seq & 1u);
    group_sync(gs.g);
    for (uint32_t j = *s_next; j < end; ++seq) {
        const uint32_t k = seq & 1u;
        // bounded wait for this page's copy (phase = uses of buffer k so far)
        if (!mbar_wait(smem_u32(gs.bar + k), (seq >> 1) & 1u)) *reinterpret_cast<volatile uint32_t *>(gs.s_flag) = 1;
        group_sync(gs.g);
        if (*reinterpret_cast<volatile uint32_t *>(gs.s_flag)) {
            if (tid == 0) latch_status(status, SINET_ERR_TIMEOUT);
            return false;
        }
        const uint32_t id = gs.s_id[k], fill = gs.s_fill[k];
        uint64_t *pg = gs.buf + k * kPartPage;
        uint32_t *oc = gs.ocnt + k * gs.ow;
        uint64_t ent[U];
        uint32_t pos[U];  // owner << 16 | rank among the owner's entries
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t e = tid + (uint32_t)u * GT;
            ent[u] = 0;
            pos[u] = 0;
            if (e < fill) {
                ent[u] = pg[e];
                const uint32_t own = (uint32_t)divide((uint32_t)(ent[u] >> 33) & bmask, p.own_div);
                pos[u] = own << 16 | atomicAdd(oc + own, 1u);
            }
        }
        // the next page's counts start from zero (the last page that used
        // them wrote its row before the barrier above)
        uint32_t *on = gs.ocnt + (k ^ 1u) * gs.ow;
        for (uint32_t o = tid; o <= G; o += GT) on[o] = 0;
        group_sync(gs.g);
        // while the first warp scans: the next page's claim and copy (into
        // the other buffer, whose page was stored back before the first
        // barrier) by the second warp, off the group's barrier-to-barrier path
        if (tid == 32) *s_next = claim_page(p, gs, b, k ^ 1u);
        // exclusive scan of the G + 1 counts by the group's first warp (the
        // last count is always zero, so its offset is the page's fill)
        if (tid < 32) {
            const uint32_t per = (G + 1 + 31) / 32, o0 = lane * per;
            if (per <= 8) {  // up to 255 owners: each lane's counts stay in registers
                uint32_t c[8], sum = 0;
#pragma unroll
                for (uint32_t q = 0; q < 8; ++q) {
                    c[q] = (q < per && o0 + q <= G) ? oc[o0 + q] : 0u;
                    sum += c[q];
                }
                uint32_t ex = warp_exclusive(sum, lane);
#pragma unroll
                for (uint32_t q = 0; q < 8; ++q) {
                    if (q < per && o0 + q <= G) oc[o0 + q] = ex;
                    ex += c[q];
                }
            } else {
                uint32_t sum = 0;
                for (uint32_t q = 0; q < per; ++q)
                    if (o0 + q <= G) sum += oc[o0 + q];
                uint32_t ex = warp_exclusive(sum, lane);
                for (uint32_t q = 0; q < per; ++q) {
                    if (o0 + q > G) break;
                    const uint32_t c = oc[o0 + q];
                    oc[o0 + q] = ex;
                    ex += c;
                }
            }
        }
        group_sync(gs.g);
        // every entry is in registers: scatter them in place, owner by owner
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (tid + (uint32_t)u * GT < fill) pg[oc[pos[u] >> 16] + (pos[u] & 0xFFFFu)] = ent[u];
        uint16_t *row = p.idx + (uint64_t)j * (G + 1);
        for (uint32_t o = tid; o <= G; o += GT) row[o] = (uint16_t)oc[o];
        group_sync(gs.g);
        // back to the page, 16 bytes per store
        uint4 *dst = reinterpret_cast<uint4 *>(p.pages + (uint64_t)id * kPartPage);
        const uint4 *v = reinterpret_cast<const uint4 *>(pg);
        for (uint32_t e = tid; 2 * e < fill; e += GT) {
            if (2 * e + 1 < fill) {
                dst[e] = v[e];
            } else {
                p.pages[(uint64_t)id * kPartPage + 2 * e] = pg[2 * e];
            }
        }
        j = *s_next;
    }
    // the group's pages and rows are stored: count the group done with bucket b
    __threadfence();
    group_sync(gs.g);
    if (tid == 0) atomicAdd(p.p1_done + b, 1u);
    return true;
}

// Sum this CTA's bins of bucket b from every page's run, then store them.
// `tile` holds [6][own_bins] words: counts of directions 0 and 1, byte sums'
// low words of both, high words of both. Each warp takes a contiguous share
// of the bucket's pages, 32 at a time (one per lane): it reads their run
// bounds, scans the run lengths across the warp, and walks the concatenated
// runs 32 entries per step, eight steps of loads in flight; a lane finds the
// run of its entry by binary search over the warp's run starts (the last run
// starting at or before the entry holds it, empty runs included).
template <uint32_t NR>
__device__ __forceinline__ bool reduce_bucket(const HistArgs &h, const PartDev &p, uint32_t *tile, uint32_t b,
                                              uint32_t groups, uint32_t accumulate, uint32_t *s_ok,
                                              const uint32_t *s_fail, uint32_t tid, uint32_t *status) {
    const uint32_t G = p.g_cold, T = p.own_bins, o = blockIdx.x;
    if (tid == 0) {
        bool ok = false;
        for (uint32_t k = 0; k < kSpinLimit; ++k) {
            if (ld_acquire(p.p1_done + b) >= G * groups) {
                ok = true;
                break;
            }
            if (*reinterpret_cast<const volatile uint32_t *>(s_fail)) break;
        }
        if (!ok) latch_status(status, SINET_ERR_TIMEOUT);
        *s_ok = ok ? 1u : 0u;
    }
    reduce_sync<NR>();  // the tile was zeroed by the previous bucket's store (or at the start)
    if (!*s_ok) return false;
    const uint64_t lo_bin = ((uint64_t)b << p.cb_shift) + (uint64_t)o * T;
    const uint32_t warp = tid >> 5, lane = tid & 31, nw = NR >> 5;
    const uint32_t pb = p.bucket_pg[b], pn = p.bucket_pg[b + 1] - pb;
    const uint32_t w1 = pb + (uint32_t)((uint64_t)pn * (warp + 1) / nw);
    for (uint32_t j0 = pb + (uint32_t)((uint64_t)pn * warp / nw); j0 < w1; j0 += 32) {
        const uint32_t j = j0 + lane;
        uint32_t len = 0;
        uint64_t at = 0;  // position in `pages` of the run's first entry
        if (j < w1) {
            const uint16_t *row = p.idx + (uint64_t)j * (G + 1);
            const uint32_t e0 = row[o];
            len = row[o + 1] - e0;
            at = (uint64_t)p.page_list[j] * kPartPage + e0;
        }
        uint32_t incl = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, d);
            if (lane >= (uint32_t)d) incl += y;
        }
        const uint32_t start = incl - len, total = __shfl_sync(kFull, incl, 31);
        for (uint32_t k0 = 0; k0 < total; k0 += 8 * 32) {
            uint64_t e[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t k = k0 + (uint32_t)u * 32 + lane;
                uint32_t r = 0;
#pragma unroll
                for (uint32_t s = 16; s; s >>= 1)
                    if (__shfl_sync(kFull, start, (int)(r + s)) <= k) r += s;
                const uint64_t a = __shfl_sync(kFull, at, (int)r);
                const uint32_t sr = __shfl_sync(kFull, start, (int)r);
                e[u] = k < total ? p.pages[a + (k - sr)] : 0ull;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (k0 + (uint32_t)u * 32 + lane >= total) continue;
                const uint32_t key = (uint32_t)(e[u] >> 32);
                const uint32_t d = key & 1u;
                const uint32_t tb = (uint32_t)((key >> 1) - lo_bin);
                if (tb >= T) {  // not this owner's bin: cannot happen for a sorted page
                    latch_status(status, SINET_ERR_DEVICE_CHECK);
                    continue;
                }
                atomicAdd(tile + d * T + tb, 1u);
                smem_add_wide(tile + (2 + d) * T + tb, tile + (4 + d) * T + tb, (uint32_t)e[u], 0u);
            }
        }
    }
    reduce_sync<NR>();
    uint64_t hi_bin = lo_bin + T;
    const uint64_t b_end = (uint64_t)(b + 1) << p.cb_shift;
    if (hi_bin > b_end) hi_bin = b_end;
    if (hi_bin > h.n_bins) hi_bin = h.n_bins;
    if (lo_bin < hi_bin) {
        const uint32_t n = (uint32_t)(hi_bin - lo_bin);
        for (uint32_t i = tid; i < n; i += NR) {
            const uint64_t bin = lo_bin + i;
            uint32_t c0 = tile[i], c1 = tile[T + i];
            uint64_t s0 = (uint64_t)tile[4 * T + i] << 32 | tile[2 * T + i];
            uint64_t s1 = (uint64_t)tile[5 * T + i] << 32 | tile[3 * T + i];
#pragma unroll
            for (uint32_t k = 0; k < 6; ++k) tile[k * T + i] = 0;  // ready for the next bucket
            if (accumulate) {
                c0 += h.cnt[0][bin];
                c1 += h.cnt[1][bin];
                s0 += h.byt[0][bin];
                s1 += h.byt[1][bin];
            }
            h.cnt[0][bin] = c0;
            h.cnt[1][bin] = c1;
            h.byt[0][bin] = s0;
            h.byt[1][bin] = s1;
        }
    }
    reduce_sync<NR>();  // every bin stored and zeroed before the next bucket's adds
    return true;
}

}  // namespace

// Shared memory of the cold pass: SG page-sorting groups (two page buffers
// and two owner-count arrays each), then the tile.
__host__ __device__ constexpr uint32_t cold_ocnt_words(uint32_t g_cold) { return (g_cold + 1 + 3) & ~3u; }
__host__ __device__ constexpr size_t cold_group_bytes(uint32_t g_cold) {
    return 16ull * kPartPage + 8ull * cold_ocnt_words(g_cold);
}

// Threads [0, SG * 256) are SG page-sorting groups; they sort bucket after
// bucket, at most kSortAhead buckets ahead of this CTA's reducers. The other
// threads reduce: bucket after bucket, once every group of every CTA has
// sorted it. The two roles meet only at those two waits, so the sorting's
// barriers and the gathering's loads overlap. A role that fails (a bounded
// wait ran out) sets s_fail and the other stops at its next bucket.
template <int SG>
__global__ void __launch_bounds__(kColdThreads, 1) k_part_cold(HistArgs h, PartDev p, uint32_t accumulate,
                                                               uint32_t *status) {
    constexpr uint32_t NS = SG * kSortThreads, NR = kColdThreads - NS;
    static_assert(SG >= 1 && NR >= 64, "room for the reducing warps");
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ uint32_t s_ok, s_fail, s_reduced, s_go[SG], s_gflag[SG], s_id[SG][2], s_fill[SG][2], s_next[SG];
    __shared__ uint64_t s_bar[SG][2];
    const uint32_t ow = cold_ocnt_words(p.g_cold);
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem + SG * cold_group_bytes(p.g_cold));
    for (uint32_t i = threadIdx.x; i < 6 * p.own_bins; i += kColdThreads) tile[i] = 0;
    if (threadIdx.x < NS) {  // both owner-count arrays of every group start at zero
        uint32_t *oc = reinterpret_cast<uint32_t *>(smem + (threadIdx.x / kSortThreads) * cold_group_bytes(p.g_cold) +
                                                    16ull * kPartPage);
        for (uint32_t i = threadIdx.x % kSortThreads; i < 2 * ow; i += kSortThreads) oc[i] = 0;
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < SG; ++k) {
            mbar_init(smem_u32(&s_bar[k][0]), 1);
            mbar_init(smem_u32(&s_bar[k][1]), 1);
            s_gflag[k] = 0;
        }
        s_fail = 0;
        s_reduced = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile uint32_t *fail = &s_fail, *reduced = &s_reduced;
    if (threadIdx.x < NS) {
        const uint32_t g = threadIdx.x / kSortThreads, t = threadIdx.x % kSortThreads;
        GroupSmem gs;
        gs.buf = reinterpret_cast<uint64_t *>(smem + g * cold_group_bytes(p.g_cold));
        gs.ocnt = reinterpret_cast<uint32_t *>(gs.buf + 2 * kPartPage);
        gs.ow = ow;
        gs.bar = s_bar[g];
        gs.s_id = s_id[g];
        gs.s_fill = s_fill[g];
        gs.s_next = &s_next[g];
        gs.s_flag = &s_gflag[g];
        gs.g = g;
        uint32_t seq = 0;
        for (uint32_t b = 0; b < p.n_buckets; ++b) {
            if (t == 0) {  // the group goes on once the reducers are close enough behind
                uint32_t go = 0;
                for (uint32_t k = 0; k < kSpinLimit && !*fail; ++k)
                    if (*reduced + kSortAhead > b) {
                        go = 1;
                        break;
                    }
                if (!go && !*fail) {
                    latch_status(status, SINET_ERR_TIMEOUT);
                    *fail = 1;
                }
                s_go[g] = go && !*fail;
            }
            group_sync(g);
            if (!reinterpret_cast<volatile uint32_t *>(s_go)[g]) break;
            if (!sort_pages(p, gs, b, seq, status)) {
                *fail = 1;
                break;
            }
        }
    } else {
        const uint32_t t = threadIdx.x - NS;
        for (uint32_t b = 0; b < p.n_buckets; ++b) {
            if (!reduce_bucket<NR>(h, p, tile, b, SG, accumulate, &s_ok, &s_fail, t, status)) {
                *fail = 1;
                break;
            }
            if (t == 0) *reduced = b + 1;
        }
    }
    __syncthreads();
}

// 6. Hot totals into their bins (a replicated bin sits in four slots, so
// the adds are reductions).
__global__ void __launch_bounds__(256) k_part_hot_add(HistArgs h, PartDev p, uint32_t slots) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += gridDim.x * blockDim.x) {
        const uint32_t key = p.hot_keys[i];
        if (key == kNoKey || key >= h.n_bins) continue;
#pragma unroll
        for (uint32_t d = 0; d < 2; ++d) {
            const uint32_t c = p.hot_cnt[d * slots + i];
            if (!c) continue;
            red_add_u32(h.cnt[d] + key, c);
            red_add_u64(h.byt[d] + key, p.hot_bytes[d * slots + i]);
        }
    }
}

// ---------------------------------------------------------------------------
// Host side.

namespace {

uint32_t ceil_log2(uint64_t x) {
    uint32_t l = 0;
    while ((1ull << l) < x) ++l;
    return l;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

Divider make_divider(uint64_t w);  // api.cu

static size_t main_smem(uint32_t tsm, uint32_t slots, uint32_t n_buckets) {
    return ((size_t)(tsm + 127u) & ~(size_t)127u) + (size_t)kPartStages * kPartStageBytes + 28ull * slots +
           36ull * n_buckets;
}

cudaError_t plan_partition(int lk, uint32_t table_smem, const RecArgs &r, const HistArgs &h, uint32_t bucket_bits,
                           int sm_count, size_t smem_optin, PartPlan *out) {
    PartPlan P{};
    if (lk == LK_CLASS_IN || sm_count <= 0) return cudaErrorNotSupported;
    const uint64_t n = r.g.n;
    const uint64_t routed_max = n * (h.two_dir ? 2ull : 1ull);
    if (routed_max >= 0xFFFFF000ull) return cudaErrorNotSupported;  // u32 positions and fills
    const uint32_t G = (uint32_t)sm_count;
    if (G > 2048) return cudaErrorNotSupported;  // four owner counts per thread of a 512-thread group
    // buckets: 2^cb bins each, at most kPartMaxBuckets of them; owners of G bins slices
    uint32_t cb = bucket_bits ? bucket_bits : 19u;
    while (cb < 31 && (((uint64_t)h.n_bins + (1ull << cb) - 1) >> cb) > kPartMaxBuckets) ++cb;
    const uint32_t nb = (uint32_t)(((uint64_t)h.n_bins + (1ull << cb) - 1) >> cb);
    const uint32_t T = (uint32_t)(((1ull << cb) + G - 1) / G);
    // two page-sorting groups where the tile leaves room, else one
    // two page-sorting groups where the tile leaves room, else one (1 KB for
    // the kernel's static shared memory)
    const size_t group = cold_group_bytes(G);
    const size_t tail = 24ull * T;
    P.cold_groups = 2;
    while (P.cold_groups > 1 && P.cold_groups * group + tail + 1024 > smem_optin) P.cold_groups -= 1;
    P.smem_cold = P.cold_groups * group + tail;
    if (P.smem_cold + 1024 > smem_optin) return cudaErrorNotSupported;
    // hot table: as many sets as shared memory allows (at least 2^4)
    const uint32_t tsm = (table_smem + 127u) & ~127u;
    uint32_t sb = 12;
    while (sb > 4 && main_smem(tsm, 4u << sb, nb) + 1024 > smem_optin) --sb;
    if (main_smem(tsm, 4u << sb, nb) + 1024 > smem_optin) return cudaErrorNotSupported;
    P.slots = 4u << sb;
    P.smem_main = main_smem(tsm, P.slots, nb);
    // sample: about n / 4096 records (at least 2^19, at most all), in chunks;
    // bins holding 1 / 50,000 of the updates still get about ten hits
    const uint64_t chunks = (n + kPartSampleChunk - 1) / kPartSampleChunk;
    const uint64_t target = std::min<uint64_t>(n, std::max<uint64_t>(1ull << 19, n >> 12));
    uint64_t stride = target ? (chunks * kPartSampleChunk) / target : 1;
    if (stride < 1) stride = 1;
    const uint64_t s_chunks = (chunks + stride - 1) / stride;
    uint32_t hb = ceil_log2(2 * s_chunks * kPartSampleChunk);
    hb = std::min(23u, std::max(10u, hb));
    // records staged by TMA: from the first index at which all four streams
    // are 16-byte aligned, in whole stages
    PartDev &d = P.d;
    if (r.g.vec) {
        const uint64_t i_lo = r.g.shift < 0 ? (uint64_t)(r.g.shift + 4) : 0ull;
        d.i_lo = std::min<uint64_t>(i_lo, n);
        d.n_full = n > d.i_lo ? (n - d.i_lo) / kPartStageRecords : 0;
        d.n_head = d.i_lo;
    } else {
        d.i_lo = 0;
        d.n_full = 0;
        d.n_head = 0;
    }
    d.set_bits = sb;
    d.cb_shift = cb;
    d.n_buckets = nb;
    d.g_cold = G;
    d.own_bins = T;
    d.own_div = make_divider(T);
    d.hash_mask = (1u << hb) - 1u;
    d.hash_shift = 32 - hb;
    d.sample_chunks = s_chunks;
    d.sample_stride = stride;
    // pages: each CTA's region of creg pages per bucket (room for a cold
    // share of 30 % of the routed updates, spread evenly, plus one page),
    // then the shared part, which alone holds every routed update
    const uint64_t per_region = (3 * routed_max / 10 + (uint64_t)G * nb * kPartPage - 1) / ((uint64_t)G * nb * kPartPage);
    d.creg = (uint32_t)std::min<uint64_t>(16, per_region + 1);
    const uint64_t regions = (uint64_t)G * nb * d.creg;
    const uint64_t cap = regions + (routed_max + kPartPage - 1) / kPartPage + 2ull * G * nb + 1;
    if (cap >= 0xFFFFFFFFull) return cudaErrorNotSupported;
    d.dyn_base = (uint32_t)regions;
    d.pages_cap = (uint32_t)cap;
    P.grid_main = G;
    P.grid_sample = G;
    P.grid_cold = G;
    P.smem_sample = ((table_smem + 15u) & ~15u) + (size_t)HotCache::kSlotBytes * (HotCache::kWays << kPartSampleSetBits);
    // scratch layout
    size_t o = 0;
    P.off_ff = o;
    P.off_hash_keys = o;
    o = align256(o + (4ull << hb));
    P.off_hot_keys = o;
    o = align256(o + 4ull * P.slots);
    P.bytes_ff = o - P.off_ff;
    P.off_zero = o;
    P.off_levels = o;
    o = align256(o + 4ull * 32);
    P.off_cand_n = o;
    o = align256(o + 4);
    P.off_page_alloc = o;
    o = align256(o + 4);
    P.off_hot_cnt = o;
    o = align256(o + 8ull * P.slots);
    P.off_hot_bytes = o;
    o = align256(o + 16ull * P.slots);
    P.off_bucket_cnt = o;
    o = align256(o + 4ull * nb);
    P.off_p1_done = o;
    o = align256(o + 4ull * nb);
    P.off_pg_next = o;
    o = align256(o + 4ull * nb);
    P.off_hash_cnt = o;
    o = align256(o + (4ull << hb));
    P.bytes_zero = o - P.off_zero;
    P.off_cand = o;
    o = align256(o + 8ull * kPartMaxCand);
    P.off_page_bucket = o;
    o = align256(o + 4ull * cap);
    P.off_page_fill = o;
    o = align256(o + 4ull * cap);
    P.off_bucket_pg = o;
    o = align256(o + 4ull * (nb + 1));
    P.off_page_list = o;
    o = align256(o + 4ull * cap);
    P.off_idx = o;
    o = align256(o + 2ull * cap * (G + 1));
    P.off_pages = o;
    o = align256(o + 8ull * kPartPage * cap);
    P.scratch_bytes = o;
    *out = P;
    return cudaSuccess;
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int LK>
static cudaError_t launch_lk(const RecArgs &r, const TableArgs &t, const HistArgs &h, const PartPlan &P,
                             const LaunchCfg &c) {
    cudaError_t e;
    if ((e = set_smem(k_part_sample<LK>, P.smem_sample)) != cudaSuccess) return e;
    k_part_sample<LK><<<P.grid_sample, 256, P.smem_sample, c.stream>>>(r, t, h, P.d, c.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_part_levels<<<4 * P.grid_main, 256, 0, c.stream>>>(P.d);
    k_part_total<<<4 * P.grid_main, 256, 0, c.stream>>>(P.d);
    k_part_collect<<<4 * P.grid_main, 256, 0, c.stream>>>(P.d);
    if ((e = set_smem(k_part_build, 4ull * P.slots)) != cudaSuccess) return e;
    k_part_build<<<1, 1024, 4ull * P.slots, c.stream>>>(P.d, P.slots);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (h.w_is_one) {
        if ((e = set_smem(k_part_main<LK, true>, P.smem_main)) != cudaSuccess) return e;
        k_part_main<LK, true><<<P.grid_main, kPartThreads, P.smem_main, c.stream>>>(r, t, h, P.d, c.status);
    } else {
        if ((e = set_smem(k_part_main<LK, false>, P.smem_main)) != cudaSuccess) return e;
        k_part_main<LK, false><<<P.grid_main, kPartThreads, P.smem_main, c.stream>>>(r, t, h, P.d, c.status);
    }
    return cudaGetLastError();
}

cudaError_t run_partition(int lk, const RecArgs &r, const TableArgs &t, const HistArgs &h, PartPlan P,
                          void *scratch, bool accumulate, const LaunchCfg &c) {
    uint8_t *base = static_cast<uint8_t *>(scratch);
    PartDev &d = P.d;
    d.hash_keys = reinterpret_cast<uint32_t *>(base + P.off_hash_keys);
    d.hash_cnt = reinterpret_cast<uint32_t *>(base + P.off_hash_cnt);
    d.levels = reinterpret_cast<uint32_t *>(base + P.off_levels);
    d.cand_n = reinterpret_cast<uint32_t *>(base + P.off_cand_n);
    d.cand = reinterpret_cast<uint2 *>(base + P.off_cand);
    d.hot_keys = reinterpret_cast<uint32_t *>(base + P.off_hot_keys);
    d.hot_cnt = reinterpret_cast<uint32_t *>(base + P.off_hot_cnt);
    d.hot_bytes = reinterpret_cast<uint64_t *>(base + P.off_hot_bytes);
    d.page_alloc = reinterpret_cast<uint32_t *>(base + P.off_page_alloc);
    d.page_bucket = reinterpret_cast<uint32_t *>(base + P.off_page_bucket);
    d.page_fill = reinterpret_cast<uint32_t *>(base + P.off_page_fill);
    d.pages = reinterpret_cast<uint64_t *>(base + P.off_pages);
    d.bucket_cnt = reinterpret_cast<uint32_t *>(base + P.off_bucket_cnt);
    d.bucket_pg = reinterpret_cast<uint32_t *>(base + P.off_bucket_pg);
    d.page_list = reinterpret_cast<uint32_t *>(base + P.off_page_list);
    d.idx = reinterpret_cast<uint16_t *>(base + P.off_idx);
    d.p1_done = reinterpret_cast<uint32_t *>(base + P.off_p1_done);
    d.pg_next = reinterpret_cast<uint32_t *>(base + P.off_pg_next);
    cudaError_t e;
    if ((e = cudaMemsetAsync(base + P.off_ff, 0xFF, P.bytes_ff, c.stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(base + P.off_zero, 0, P.bytes_zero, c.stream)) != cudaSuccess) return e;
    // region pages count as empty unless their CTA records a fill
    if ((e = cudaMemsetAsync(d.page_fill, 0, 4ull * d.dyn_base, c.stream)) != cudaSuccess) return e;
    switch (lk) {
        case LK_INTERVAL: e = launch_lk<LK_INTERVAL>(r, t, h, P, c); break;
        case LK_TOGGLE1: e = launch_lk<LK_TOGGLE1>(r, t, h, P, c); break;
        case LK_TOGGLE2: e = launch_lk<LK_TOGGLE2>(r, t, h, P, c); break;
        case LK_PML: e = launch_lk<LK_PML>(r, t, h, P, c); break;
        case LK_INTERVAL_GLOBAL: e = launch_lk<LK_INTERVAL_GLOBAL>(r, t, h, P, c); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    k_part_count_pages<<<2 * P.grid_main, 256, 0, c.stream>>>(P.d);
    k_part_scan_pages<<<1, kPartMaxBuckets, 0, c.stream>>>(P.d);
    k_part_list_pages<<<2 * P.grid_main, 256, 0, c.stream>>>(P.d);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    uint32_t acc = accumulate ? 1u : 0u;
    HistArgs hh = h;
    uint32_t *status = c.status;
    void *args[] = {&hh, &d, &acc, &status};
    const void *cold = P.cold_groups == 2 ? (const void *)k_part_cold<2> : (const void *)k_part_cold<1>;
    if ((e = cudaFuncSetAttribute(cold, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem_cold)) !=
        cudaSuccess)
        return e;
    e = cudaLaunchCooperativeKernel(cold, dim3(P.grid_cold), dim3(kColdThreads), args, P.smem_cold, c.stream);
    if (e != cudaSuccess) return e;
    k_part_hot_add<<<std::max<uint32_t>(1, P.slots / 256), 256, 0, c.stream>>>(h, P.d, P.slots);
    return cudaGetLastError();
}

}  // namespace sinet
