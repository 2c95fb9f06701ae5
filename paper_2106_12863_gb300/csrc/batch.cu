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

// Quads [q0, q1) of slice records with warp run-combining and the hot-key
// cache (in `work`), flushed at the end of the item.
template <int LK>
__device__ __forceinline__ void item_agg(const Classifier<LK> &C, const RecArgs &r, const HistArgs &h,
                                         uint64_t q0, uint64_t q1, uint8_t *work, uint64_t pol,
                                         unsigned long long *s_cnt) {
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
        const uint64_t q = qb + lane;
        Quad Q;
        load_quad<true, true, true, false>(r, q < q1 ? q : r.g.quads, pol, Q);
        uint32_t bins[4];
        const uint32_t inr = h.w_is_one ? bin_quad<true>(h, Q, bins) : bin_quad<false>(h, Q, bins);
        classify_quad<LK>(C, Q);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t dirs = 0;
            if (Q.valid >> j & 1u) {
                bump_class_packed(ccp, Q.cls[j]);
                dirs = dirs_of_packed(h, Q.cls[j], inr >> j & 1u, oorp);
            }
            const uint32_t key = dirs ? (bins[j] << 1 | (dirs & 1u ? 0u : 1u)) : kNoKey;
            update_agg(h, hc, key, Q.by[j]);
            if (h.two_dir) {
                const bool both = dirs == 3u;
                if (__any_sync(kFull, both)) update_agg(h, hc, both ? (bins[j] << 1 | 1u) : kNoKey, Q.by[j]);
            }
        }
    }
    drain_packed(ccp, oorp, s_cnt);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
        const uint32_t c = hc.cnt[i];
        if (c) gadd(h, hc.keys[i] & 1u, hc.keys[i] >> 1, c, (uint64_t)hc.hi[i] << 32 | hc.lo[i]);
    }
}

// Quads [q0, q1) with global atomics per run of equal keys inside a quad.
template <int LK>
__device__ __forceinline__ void item_noagg(const Classifier<LK> &C, const RecArgs &r, const HistArgs &h,
                                           uint64_t q0, uint64_t q1, uint64_t pol,
                                           unsigned long long *s_cnt) {
    uint64_t ccp = 0;
    uint32_t oorp = 0;
    for (uint64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        Quad Q;
        load_quad<true, true, true, false>(r, q, pol, Q);
        uint32_t bins[4];
        const uint32_t inr = h.w_is_one ? bin_quad<true>(h, Q, bins) : bin_quad<false>(h, Q, bins);
        classify_quad<LK>(C, Q);
        uint32_t pk = kNoKey, pc = 0;
        uint64_t ps = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!(Q.valid >> j & 1u)) continue;
            bump_class_packed(ccp, Q.cls[j]);
            const uint32_t dirs = dirs_of_packed(h, Q.cls[j], inr >> j & 1u, oorp);
            if (!dirs) continue;
            const uint32_t key = bins[j] << 1 | (dirs & 1u ? 0u : 1u);
            if (key == pk) {
                pc++;
                ps += Q.by[j];
            } else {
                if (pk != kNoKey) gadd(h, pk & 1u, pk >> 1, pc, ps);
                pk = key;
                pc = 1;
                ps = Q.by[j];
            }
            if (dirs == 3u) gadd(h, 1u, bins[j], 1u, Q.by[j]);
        }
        if (pk != kNoKey) gadd(h, pk & 1u, pk >> 1, pc, ps);
    }
    drain_packed(ccp, oorp, s_cnt);
}

// Quads [q0, q1) into a shared-memory tile holding the slice's whole
// histogram (T >= n_bins bins per direction; entry layout as in the fused
// tile kernel: low word of the byte sum, and count << 16 | byte-sum bits
// 32-47; a work item holds at most 65,535 records). The touched range is
// flushed with global atomics.
template <int LK>
__device__ __forceinline__ void item_tile(const Classifier<LK> &C, const RecArgs &r, const HistArgs &h,
                                          uint64_t q0, uint64_t q1, uint8_t *work, uint32_t T,
                                          uint64_t pol, unsigned long long *s_cnt, uint32_t *s_lo,
                                          uint32_t *s_hi) {
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
        load_quad<true, true, true, false>(r, q, pol, Q);
        uint32_t bins[4];
        const uint32_t inr = h.w_is_one ? bin_quad<true>(h, Q, bins) : bin_quad<false>(h, Q, bins);
        classify_quad<LK>(C, Q);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!(Q.valid >> j & 1u)) continue;
            bump_class_packed(ccp, Q.cls[j]);
            const uint32_t dirs = dirs_of_packed(h, Q.cls[j], inr >> j & 1u, oorp);
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
            if (vh) gadd(h, d, off, vh >> 16, (uint64_t)(vh & 0xFFFFu) << 32 | tlo[e]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *s_lo = 0xFFFFFFFFu;
        *s_hi = 0;
    }
}

template <int LK>
__device__ __noinline__ void run_item(const BatchSlice &S, const uint8_t *table, uint8_t *work,
                                         uint64_t q0, uint64_t q1, uint64_t pol,
                                         unsigned long long *s_cnt, uint32_t *s_lo, uint32_t *s_hi) {
    Classifier<LK> C;
    C.attach(S.t, table);
    const RecArgs &r = S.r;
    const HistArgs &h = S.h;
    switch (S.strat) {
        case BS_AGG:
            item_agg<LK>(C, r, h, q0, q1, work, pol, s_cnt);
            break;
        case BS_TILE:
            item_tile<LK>(C, r, h, q0, q1, work, S.tile_bins, pol, s_cnt, s_lo, s_hi);
            break;
        default:
            item_noagg<LK>(C, r, h, q0, q1, pol, s_cnt);
            break;
    }
}

__global__ void __launch_bounds__(kBatchBlock, 2) k_batch(BatchArgs b, uint32_t *status) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t s_item, s_slice, s_lo, s_hi;
    __shared__ unsigned long long s_cnt[6];
    __shared__ __align__(16) BatchSlice s_desc;
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
    for (;;) {
        __syncthreads();  // previous item done with shared memory; barrier initialised
        if (threadIdx.x == 0) {
            const uint32_t it = atomicAdd(&b.hdr->counter, 1u);
            s_item = it;
            s_slice = it < b.hdr->total_items ? find_slice(b.item_start, b.hdr->n_slices, it) : 0u;
        }
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= b.hdr->total_items) break;
        const uint32_t si = s_slice;
        // the slice's descriptor, read by every thread, from shared memory
        static_assert(sizeof(BatchSlice) % 4 == 0, "descriptor copied in words");
        for (uint32_t i = threadIdx.x; i < sizeof(BatchSlice) / 4; i += blockDim.x)
            reinterpret_cast<uint32_t *>(&s_desc)[i] = reinterpret_cast<const uint32_t *>(b.slices + si)[i];
        __syncthreads();
        const BatchSlice &S = s_desc;
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
        uint8_t *work = smem + ((tbytes + 15u) & ~15u);
        const uint64_t iq = b.hdr->item_quads;
        const uint64_t q0 = (uint64_t)(item - b.item_start[si]) * iq;
        const uint64_t q1 = min(q0 + iq, S.r.g.quads);
        const uint64_t pol = policy_evict_first();
        switch (lk) {
            case LK_TOGGLE1:
                run_item<LK_TOGGLE1>(S, smem, work, q0, q1, pol, s_cnt, &s_lo, &s_hi);
                break;
            case LK_TOGGLE2:
                run_item<LK_TOGGLE2>(S, smem, work, q0, q1, pol, s_cnt, &s_lo, &s_hi);
                break;
            case LK_INTERVAL:
                run_item<LK_INTERVAL>(S, smem, work, q0, q1, pol, s_cnt, &s_lo, &s_hi);
                break;
            default:
                run_item<LK_INTERVAL_GLOBAL>(S, smem, work, q0, q1, pol, s_cnt, &s_lo, &s_hi);
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
