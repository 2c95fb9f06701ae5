// Batched persistent discriminate + histogram: many independent slices (each
// with its own records, CIDR list, window, bin width and outputs) in one
// launch. The coordinated batches of Section 4 become work items (slice,
// chunk) that persistent CTAs pull from a device counter, so slices of very
// uneven size share the GPU without a launch per slice. A CTA restages the
// shared-memory table only when the slice's table changes.
#include "combine.cuh"
#include "launch.h"

namespace sinet {
namespace {

// Last s in [0, n) with start[s] <= item (start is non-decreasing, start[0] = 0):
// the slice that owns work item `item`, skipping slices with no items.
__device__ __forceinline__ uint32_t find_slice(const uint32_t *start, uint32_t n, uint32_t item) {
    uint32_t lo = 0, len = n;
    while (len > 1) {
        const uint32_t half = len >> 1;
        if (start[lo + half] <= item) lo += half;
        len -= half;
    }
    return lo;
}

// Zero n 32-bit words at a 4-byte-aligned address with 16-byte stores where aligned.
__device__ __forceinline__ void zero_words(uint32_t *p, uint32_t n) {
    uint32_t head = (uint32_t)((16u - ((uintptr_t)p & 15u)) & 15u) / 4u;
    if (head > n) head = n;
    if (threadIdx.x < head) p[threadIdx.x] = 0;
    uint4 *v = reinterpret_cast<uint4 *>(p + head);
    const uint32_t nv = (n - head) / 4;
    for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) v[i] = make_uint4(0, 0, 0, 0);
    for (uint32_t i = head + 4 * nv + threadIdx.x; i < n; i += blockDim.x) p[i] = 0;
}

__global__ void __launch_bounds__(256) k_batch_zero(BatchArgs b) {
    if (blockIdx.x == 0 && threadIdx.x == 0) b.hdr->counter = 0;
    const uint32_t total = b.hdr->total_zero, n = b.hdr->n_slices;
    for (uint32_t z = blockIdx.x; z < total; z += gridDim.x) {
        const uint32_t s = find_slice(b.zero_start, n, z);
        const HistArgs &h = b.slices[s].h;
        const uint32_t b0 = (z - b.zero_start[s]) * kZeroBins;
        const uint32_t nb = min(kZeroBins, h.n_bins - b0);
        zero_words(h.cnt[0] + b0, nb);
        zero_words(h.cnt[1] + b0, nb);
        zero_words(reinterpret_cast<uint32_t *>(h.byt[0] + b0), 2 * nb);
        zero_words(reinterpret_cast<uint32_t *>(h.byt[1] + b0), 2 * nb);
        if (b0 == 0 && threadIdx.x < 8) h.stats[threadIdx.x] = 0;
    }
}

// Bulk copy of a table image into shared memory on a barrier the CTA keeps for
// its lifetime (`phase` tracks its parity). Returns false, with
// SINET_ERR_TIMEOUT latched, if the copy did not land within the bound.
__device__ bool restage(uint8_t *sdst, const uint8_t *gsrc, uint32_t bytes, uint32_t bar,
                        uint32_t &phase, uint32_t *status) {
    if (threadIdx.x == 0) {
        // earlier generic-proxy reads of this shared memory precede the copy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                     : "memory");
        const uint32_t kChunk = 32768;
        for (uint32_t off = 0; off < bytes; off += kChunk) {
            const uint32_t sz = bytes - off < kChunk ? bytes - off : kChunk;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(sdst + off)),
                "l"(gsrc + off), "r"(sz), "r"(bar)
                : "memory");
        }
    }
    bool ok = false;
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        if (mbar_try_wait(bar, phase)) { ok = true; break; }
    }
    if (!ok) {
        latch_status(status, SINET_ERR_TIMEOUT);
        for (uint32_t it = 0; it < kSpinLimit && !mbar_try_wait(bar, phase); ++it) {
        }
    }
    phase ^= 1u;
    return ok;
}

// The current work item's slice descriptor, copied into shared memory once
// per item. The per-record code reads its fields with volatile loads at the
// point of use: kept in registers, the records' pointers, window, divider and
// output pointers would take about 40 registers for the whole loop and
// spill; a broadcast shared-memory load costs far less.
__shared__ __align__(16) BatchSlice g_desc;

template <typename T>
__device__ __forceinline__ T vld(const T &x) {
    return *reinterpret_cast<const volatile T *>(&x);
}

// Quad q (< q1) of the current slice; quads at or past q1 have no records.
__device__ __forceinline__ void bload(uint64_t q, uint64_t q1, uint64_t pol, Quad &Q) {
    const RecArgs &r = g_desc.r;
    const int64_t base = (int64_t)vld(r.g.shift) + 4 * (int64_t)q;
    const uint64_t n = vld(r.g.n);
    const uint64_t *ts = vld(r.ts);
    const uint32_t *src = vld(r.src), *dst = vld(r.dst), *by = vld(r.bytes);
    if (q < q1 && vld(r.g.vec) && base >= 0 && (uint64_t)base + 4 <= n) {
        const ulonglong2 a = ld_stream_v2u64(ts + base, pol);
        const ulonglong2 b = ld_stream_v2u64(ts + base + 2, pol);
        const uint4 s4 = ld_stream_v4(src + base, pol);
        const uint4 d4 = ld_stream_v4(dst + base, pol);
        const uint4 b4 = ld_stream_v4(by + base, pol);
        Q.ts[0] = a.x; Q.ts[1] = a.y; Q.ts[2] = b.x; Q.ts[3] = b.y;
        Q.src[0] = s4.x; Q.src[1] = s4.y; Q.src[2] = s4.z; Q.src[3] = s4.w;
        Q.dst[0] = d4.x; Q.dst[1] = d4.y; Q.dst[2] = d4.z; Q.dst[3] = d4.w;
        Q.by[0] = b4.x; Q.by[1] = b4.y; Q.by[2] = b4.z; Q.by[3] = b4.w;
        Q.valid = 0xFu;
        return;
    }
    Q.valid = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        Q.ts[j] = 0;
        Q.src[j] = Q.dst[j] = Q.by[j] = Q.cls[j] = 0;
        const int64_t i = base + j;
        if (q >= q1 || i < 0 || (uint64_t)i >= n) continue;
        Q.valid |= 1u << j;
        Q.ts[j] = ld_stream_u64(ts + i, pol);
        Q.src[j] = ld_stream_u32(src + i, pol);
        Q.dst[j] = ld_stream_u32(dst + i, pol);
        Q.by[j] = ld_stream_u32(by + i, pol);
    }
}

// Bins of the quad's records in the current slice's window (bit j of the
// result: record j is inside it).
__device__ __forceinline__ uint32_t bbin(const Quad &Q, uint32_t bins[4]) {
    const HistArgs &h = g_desc.h;
    const uint64_t t0 = vld(h.t0), span = vld(h.span);
    uint32_t inr = 0;
    if (vld(h.w_is_one)) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t rel = Q.ts[j] - t0;
            const bool in = rel < span;
            bins[j] = in ? (uint32_t)rel : 0u;
            inr |= (uint32_t)in << j;
        }
    } else {
        Divider dv;
        dv.m = vld(h.div.m);
        dv.sh1 = vld(h.div.sh1);
        dv.sh2 = vld(h.div.sh2);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t rel = Q.ts[j] - t0;
            const bool in = rel < span;
            bins[j] = in ? (uint32_t)divide(rel, dv) : 0u;
            inr |= (uint32_t)in << j;
        }
    }
    return inr;
}

// Direction bits of a record of class cls (out-of-window: counted, none).
__device__ __forceinline__ uint32_t bdirs(uint32_t policy, uint32_t cls, bool in_window, uint32_t &oorp) {
    const uint32_t dirs = (policy >> (8 * cls)) & 3u;
    if (!in_window) {
        oorp += (dirs & 1u) | ((dirs >> 1) << 16);
        return 0u;
    }
    return dirs;
}

// Add (c, s) to bin `bin` of direction d of the current slice's outputs.
__device__ __forceinline__ void bgadd(uint32_t d, uint32_t bin, uint32_t c, uint64_t s) {
    red_add_u32(vld(g_desc.h.cnt[d]) + bin, c);
    red_add_u64(vld(g_desc.h.byt[d]) + bin, s);
}

// Warp run-combining into the hot-key cache, else global reductions.
__device__ __forceinline__ void bupdate_agg(HotCache &hc, uint32_t key, uint32_t b) {
    const uint32_t peers = __match_any_sync(kFull, key);
    if (key == kNoKey) return;
    const uint32_t c = __popc(peers);
    uint64_t s = b;
    if (c > 1) {
        const uint32_t lo = __reduce_add_sync(peers, b & 0xFFFFu);
        const uint32_t hi = __reduce_add_sync(peers, b >> 16);
        s = (uint64_t)lo + ((uint64_t)hi << 16);
    }
    if ((threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1)) {
        if (!hc.add(key, c, s)) bgadd(key & 1u, key >> 1, c, s);
    }
}

// Quads [q0, q1) with warp run-combining and the hot-key cache (in `work`),
// flushed at the end of the item.
template <int LK>
__device__ __forceinline__ void item_agg(const Classifier<LK> &C, uint64_t q0, uint64_t q1, uint8_t *work,
                                         uint64_t pol, unsigned long long *s_cnt) {
    const uint32_t slots = HotCache::kWays << kBatchCacheSetBits;
    HotCache hc;
    hc.keys = reinterpret_cast<uint32_t *>(work);
    hc.cnt = hc.keys + slots;
    hc.lo = hc.cnt + slots;
    hc.hi = hc.lo + slots;
    hc.set_bits = kBatchCacheSetBits;
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
        hc.keys[i] = kNoKey;
        hc.cnt[i] = 0;
        hc.lo[i] = 0;
        hc.hi[i] = 0;
    }
    __syncthreads();
    uint64_t ccp = 0;
    uint32_t oorp = 0;
    const uint32_t lane = threadIdx.x & 31;
    // warp-uniform trip count: every lane reaches the warp-synchronous updates
    for (uint64_t qb = q0 + threadIdx.x - lane; qb < q1; qb += blockDim.x) {
        Quad Q;
        bload(qb + lane, q1, pol, Q);
        uint32_t bins[4];
        const uint32_t inr = bbin(Q, bins);
        classify_quad<LK>(C, Q);
        const uint32_t policy = vld(g_desc.h.policy);
        const bool two = vld(g_desc.h.two_dir) != 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t dirs = 0;
            if (Q.valid >> j & 1u) {
                bump_class_packed(ccp, Q.cls[j]);
                dirs = bdirs(policy, Q.cls[j], inr >> j & 1u, oorp);
            }
            const uint32_t key = dirs ? (bins[j] << 1 | (dirs & 1u ? 0u : 1u)) : kNoKey;
            bupdate_agg(hc, key, Q.by[j]);
            if (two) {
                const bool both = dirs == 3u;
                if (__any_sync(kFull, both)) bupdate_agg(hc, both ? (bins[j] << 1 | 1u) : kNoKey, Q.by[j]);
            }
        }
    }
    drain_packed(ccp, oorp, s_cnt);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
        const uint32_t c = hc.cnt[i];
        if (c) bgadd(hc.keys[i] & 1u, hc.keys[i] >> 1, c, (uint64_t)hc.hi[i] << 32 | hc.lo[i]);
    }
}

// Quads [q0, q1) with global reductions per run of equal keys inside a quad.
template <int LK>
__device__ __forceinline__ void item_noagg(const Classifier<LK> &C, uint64_t q0, uint64_t q1, uint64_t pol,
                                           unsigned long long *s_cnt) {
    uint64_t ccp = 0;
    uint32_t oorp = 0;
    for (uint64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        Quad Q;
        bload(q, q1, pol, Q);
        uint32_t bins[4];
        const uint32_t inr = bbin(Q, bins);
        classify_quad<LK>(C, Q);
        const uint32_t policy = vld(g_desc.h.policy);
        uint32_t pk = kNoKey, pc = 0;
        uint64_t ps = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!(Q.valid >> j & 1u)) continue;
            bump_class_packed(ccp, Q.cls[j]);
            const uint32_t dirs = bdirs(policy, Q.cls[j], inr >> j & 1u, oorp);
            if (!dirs) continue;
            const uint32_t key = bins[j] << 1 | (dirs & 1u ? 0u : 1u);
            if (key == pk) {
                pc++;
                ps += Q.by[j];
            } else {
                if (pk != kNoKey) bgadd(pk & 1u, pk >> 1, pc, ps);
                pk = key;
                pc = 1;
                ps = Q.by[j];
            }
            if (dirs == 3u) bgadd(1u, bins[j], 1u, Q.by[j]);
        }
        if (pk != kNoKey) bgadd(pk & 1u, pk >> 1, pc, ps);
    }
    drain_packed(ccp, oorp, s_cnt);
}

// Quads [q0, q1) into a shared-memory tile holding the slice's whole
// histogram (T >= n_bins bins per direction; entry layout as in the fused
// tile kernel: low word of the byte sum, and count << 16 | byte-sum bits
// 32-47; a work item holds at most 65,535 records). The touched range is
// flushed with global reductions.
template <int LK>
__device__ __forceinline__ void item_tile(const Classifier<LK> &C, uint64_t q0, uint64_t q1, uint8_t *work,
                                          uint32_t T, uint64_t pol, unsigned long long *s_cnt,
                                          uint32_t *s_lo, uint32_t *s_hi) {
    uint32_t *tlo = reinterpret_cast<uint32_t *>(work);
    uint32_t *thi = tlo + 2 * T;
    for (uint32_t i = threadIdx.x; i < T; i += blockDim.x)  // 4T words
        reinterpret_cast<uint4 *>(work)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    uint64_t ccp = 0;
    uint32_t oorp = 0;
    uint32_t omin = 0xFFFFFFFFu, omax = 0;
    for (uint64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        Quad Q;
        bload(q, q1, pol, Q);
        uint32_t bins[4];
        const uint32_t inr = bbin(Q, bins);
        classify_quad<LK>(C, Q);
        const uint32_t policy = vld(g_desc.h.policy);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!(Q.valid >> j & 1u)) continue;
            bump_class_packed(ccp, Q.cls[j]);
            const uint32_t dirs = bdirs(policy, Q.cls[j], inr >> j & 1u, oorp);
            if (!dirs) continue;
            const uint32_t off = bins[j];
            omin = min(omin, off);
            omax = max(omax, off);
            const uint32_t e = (dirs & 1u) ? off : T + off;
            smem_add_wide(tlo + e, thi + e, Q.by[j], 1u << 16);
            if (dirs == 3u) smem_add_wide(tlo + T + off, thi + T + off, Q.by[j], 1u << 16);
        }
    }
    drain_packed(ccp, oorp, s_cnt);
    omin = __reduce_min_sync(kFull, omin);
    omax = __reduce_max_sync(kFull, omax);
    if ((threadIdx.x & 31) == 0 && omin <= omax) {
        atomicMin(s_lo, omin);
        atomicMax(s_hi, omax);
    }
    __syncthreads();
    const uint32_t lo = *s_lo, hi = *s_hi;
    if (lo <= hi) {
        const uint32_t n = hi - lo + 1;
        for (uint32_t i = threadIdx.x; i < 2 * n; i += blockDim.x) {
            const uint32_t d = i >= n;
            const uint32_t off = lo + i - d * n;
            const uint32_t e = d * T + off;
            const uint32_t vh = thi[e];
            if (vh) bgadd(d, off, vh >> 16, (uint64_t)(vh & 0xFFFFu) << 32 | tlo[e]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *s_lo = 0xFFFFFFFFu;
        *s_hi = 0;
    }
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Poll a ready word until it holds `want` or `limit_ns` pass; the acquire
// fence orders the record loads after the observed value.
__device__ bool wait_ready(const uint32_t *word, uint32_t want, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(word) : "memory");
        if (v == want) return true;
        if (global_ns() - t0 > limit_ns) return false;
        __nanosleep(200);
    }
}

// Called (not inlined) once per work item, so each lookup form gets its own
// register allocation. Shared-memory addresses are rebuilt here from the
// dynamic shared array and a byte offset: a pointer passed in would be a
// generic address, and every table load and tile atomic through it would be
// a generic access instead of a shared-memory one.
template <int LK>
__device__ __noinline__ void run_item(uint32_t work_off, uint64_t q0, uint64_t q1, uint64_t pol,
                                      unsigned long long *s_cnt, uint32_t *s_lo, uint32_t *s_hi) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t *work = smem + work_off;
    Classifier<LK> C;
    C.attach(g_desc.t, smem);
    switch (g_desc.strat) {
        case BS_AGG:
            item_agg<LK>(C, q0, q1, work, pol, s_cnt);
            break;
        case BS_TILE:
            item_tile<LK>(C, q0, q1, work, g_desc.tile_bins, pol, s_cnt, s_lo, s_hi);
            break;
        default:
            item_noagg<LK>(C, q0, q1, pol, s_cnt);
            break;
    }
}

__global__ void __launch_bounds__(kBatchBlock, 2) k_batch(BatchArgs b, uint32_t *status) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t s_item, s_slice, s_lo, s_hi, s_ok;
    __shared__ unsigned long long s_cnt[6];
    // first work item of every slice, when the batch is small enough to keep it here
    __shared__ uint32_t s_starts[kBatchSmemStarts + 1];
    // per-CTA state lives in shared memory so the per-record loops keep the registers
    __shared__ const uint8_t *s_staged;  // image whose toggle form sits at smem[0]
    __shared__ uint32_t s_phase;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_lo = 0xFFFFFFFFu;
        s_hi = 0;
        s_staged = nullptr;
        s_phase = 0;
    }
    if (threadIdx.x < 6) s_cnt[threadIdx.x] = 0;
    const uint32_t n_sl = b.hdr->n_slices, total = b.hdr->total_items;
    const bool starts_here = n_sl <= kBatchSmemStarts;
    if (starts_here)
        for (uint32_t i = threadIdx.x; i <= n_sl; i += blockDim.x) s_starts[i] = b.item_start[i];
    // thread 0 keeps the next work item claimed ahead, so the counter's round
    // trip overlaps the current item
    uint32_t next = 0;
    if (threadIdx.x == 0) next = atomicAdd(&b.hdr->counter, 1u);
    for (;;) {
        __syncthreads();  // previous item done with shared memory; barrier initialised
        if (threadIdx.x == 0) {
            const uint32_t it = next;
            s_item = it;
            s_slice = it < total ? find_slice(starts_here ? s_starts : b.item_start, n_sl, it) : 0u;
            if (it < total) next = atomicAdd(&b.hdr->counter, 1u);
        }
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= total) break;
        const uint32_t si = s_slice;
        // the slice's descriptor, read by every thread, from shared memory
        static_assert(sizeof(BatchSlice) % 4 == 0, "descriptor copied in words");
        for (uint32_t i = threadIdx.x; i < sizeof(BatchSlice) / 4; i += blockDim.x)
            reinterpret_cast<uint32_t *>(&g_desc)[i] = reinterpret_cast<const uint32_t *>(b.slices + si)[i];
        __syncthreads();
        const BatchSlice &S = g_desc;
        if (S.ready) {
            // the slice's records are still being filled (by a copy on another
            // stream): wait, bounded, for its ready word
            if (threadIdx.x == 0) s_ok = wait_ready(S.ready, S.ready_value, b.hdr->wait_ns) ? 1u : 0u;
            __syncthreads();
            if (!s_ok) {
                if (threadIdx.x == 0) latch_status(status, SINET_ERR_TIMEOUT);
                continue;  // the item is left out; the status word says so
            }
        }
        const uint32_t lk = S.lk;
        uint32_t tbytes = 0;
        if (lk != LK_INTERVAL_GLOBAL) {
            tbytes = S.t.iv_bytes;
            if (S.t.image != s_staged) {
                uint32_t phase = s_phase;
                const bool ok = restage(smem, S.t.image, tbytes, smem_u32(&bar), phase, status);
                // everyone has read the old s_staged / s_phase; a copy that did
                // not land ends the whole CTA (the status word says why)
                if (!__syncthreads_and(ok)) return;
                if (threadIdx.x == 0) {
                    s_staged = S.t.image;
                    s_phase = phase;
                }
            }
        } else if (threadIdx.x == 0) {
            s_staged = nullptr;  // the work region overwrites the staged table
        }
        const uint32_t work_off = (tbytes + 15u) & ~15u;
        const uint64_t iq = S.item_quads;
        const uint64_t q0 = (uint64_t)(item - (starts_here ? s_starts[si] : b.item_start[si])) * iq;
        const uint64_t q1 = min(q0 + iq, S.r.g.quads);
        const uint64_t pol = policy_evict_first();
        switch (lk) {
            case LK_TOGGLE1:
                run_item<LK_TOGGLE1>(work_off, q0, q1, pol, s_cnt, &s_lo, &s_hi);
                break;
            case LK_TOGGLE2:
                run_item<LK_TOGGLE2>(work_off, q0, q1, pol, s_cnt, &s_lo, &s_hi);
                break;
            case LK_INTERVAL:
                run_item<LK_INTERVAL>(work_off, q0, q1, pol, s_cnt, &s_lo, &s_hi);
                break;
            default:
                run_item<LK_INTERVAL_GLOBAL>(work_off, q0, q1, pol, s_cnt, &s_lo, &s_hi);
                break;
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            const unsigned long long v = s_cnt[threadIdx.x];
            if (v) atomicAdd(reinterpret_cast<unsigned long long *>(S.h.stats) + threadIdx.x, v);
            s_cnt[threadIdx.x] = 0;
        }
    }
}

}  // namespace

cudaError_t run_batch_zero(const BatchArgs &b, int grid, cudaStream_t s) {
    k_batch_zero<<<grid, 256, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t batch_occupancy(uint32_t smem, int *per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch, kBatchBlock, smem);
}

cudaError_t run_batch(const BatchArgs &b, uint32_t smem, int grid, cudaStream_t s, uint32_t *status) {
    k_batch<<<grid, kBatchBlock, smem, s>>>(b, status);
    return cudaGetLastError();
}

}  // namespace sinet
