// Discriminate-only and fused discriminate + histogram kernels (sm_103a).
//
// One pass over the SoA records: 128-bit streaming loads of 4 records per
// thread, Algorithm 1 against the shared-memory-staged table, routing by the
// class policy, millisecond binning, and the histogram update of Section 5
// (a merge-scatter with the associative, commutative integer +).
#include "combine.cuh"
#include "launch.h"

namespace sinet {

// ---------------------------------------------------------------------------
// Algorithm 1 only.
template <int LK>
__global__ void __launch_bounds__(256) k_discriminate(RecArgs r, TableArgs t, uint64_t *counts,
                                                      uint32_t *status) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t bar;
    Classifier<LK> C;
    if (!C.init(t, smem, &bar, status)) return;  // table not staged: the status word says so
    const uint64_t pol = policy_evict_first();
    uint32_t cc[4] = {0, 0, 0, 0}, oor[2] = {0, 0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < r.g.quads; q += stride) {
        Quad Q;
        load_quad<false, true, false, false>(r, q, pol, Q);
        classify_quad<LK>(C, Q);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (Q.valid >> j & 1u) bump_class(cc, Q.cls[j]);
        if (r.cls_out) {
            const int64_t base = quad_base(r.g, q);
            if (Q.valid == 0xFu && quad_full(r.g, base)) {
                uint32_t w = Q.cls[0] | Q.cls[1] << 8 | Q.cls[2] << 16 | Q.cls[3] << 24;
                *reinterpret_cast<uint32_t *>(r.cls_out + base) = w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (Q.valid >> j & 1u) r.cls_out[base + j] = (uint8_t)Q.cls[j];
            }
        }
    }
    flush_counters(counts, cc, oor, false);
}

// Watch list (the blocklist views of Section 6, as a filter): a record whose
// src and dst are both outside the second list leaves the quad and counts in
// `flt` (stats[6]); the list is looked up in its global-memory interval form.
template <bool WATCH>
__device__ __forceinline__ void watch_filter(const Classifier<LK_INTERVAL_GLOBAL> &W, Quad &Q, uint32_t &flt) {
    if (!WATCH) return;
    uint32_t a[4], ws[4], wd[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = Q.src[j];
    W.template in_n<4>(a, ws);
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = Q.dst[j];
    W.template in_n<4>(a, wd);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if ((Q.valid >> j & 1u) && !(ws[j] | wd[j])) {
            Q.valid &= ~(1u << j);
            flt++;
        }
    }
}

__device__ __forceinline__ void flush_filtered(uint64_t *stats, uint32_t flt) {
    const uint32_t v = __reduce_add_sync(kFull, flt);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(reinterpret_cast<unsigned long long *>(stats + 6), (unsigned long long)v);
}

template <int LK, bool AGG, bool WATCH>
__global__ void __launch_bounds__(256, 3) k_fused_atomic(RecArgs r, TableArgs t, HistArgs h,
                                                         uint32_t cache_set_bits, TableArgs wt, uint32_t *status) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t bar;
    Classifier<LK> C;
    if (!C.init(t, smem, &bar, status)) return;  // table not staged: the status word says so
    Classifier<LK_INTERVAL_GLOBAL> W;
    if (WATCH) W.attach(wt, nullptr);
    const uint64_t pol = policy_evict_first();
    uint32_t cc[4] = {0, 0, 0, 0}, oor[2] = {0, 0}, flt = 0;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (!AGG) {
        for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < r.g.quads; q += stride) {
            Quad Q;
            load_quad<true, LK != LK_CLASS_IN, true, LK == LK_CLASS_IN>(r, q, pol, Q);
            watch_filter<WATCH>(W, Q, flt);
            classify_quad<LK>(C, Q);
            combine_quad(h, Q, cc, oor, [&](uint32_t key, uint32_t c, uint64_t s) {
                gadd(h, key & 1u, key >> 1, c, s);
            });
        }
        flush_counters(h.stats, cc, oor, true);
        if (WATCH) flush_filtered(h.stats, flt);
        return;
    }
    // hot-key cache after the staged table
    uint8_t *cm = smem + ((Classifier<LK>::smem_bytes(t) + 15u) & ~15u);
    const uint32_t slots = HotCache::kWays << cache_set_bits;
    HotCache hc;
    hc.keys = reinterpret_cast<uint32_t *>(cm);
    hc.cnt = hc.keys + slots;
    hc.lo = hc.cnt + slots;
    hc.hi = hc.lo + slots;
    hc.set_bits = cache_set_bits;
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
        hc.keys[i] = kNoKey;
        hc.cnt[i] = 0;
        hc.lo[i] = 0;
        hc.hi[i] = 0;
    }
    __syncthreads();
    // warp-uniform trip count: every lane reaches the warp-synchronous updates
    for (uint64_t q0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) - lane; q0 < r.g.quads;
         q0 += stride) {
        Quad Q;
        load_quad<true, LK != LK_CLASS_IN, true, LK == LK_CLASS_IN>(r, q0 + lane, pol, Q);
        watch_filter<WATCH>(W, Q, flt);
        classify_quad<LK>(C, Q);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool v = Q.valid >> j & 1u;
            uint32_t bin = 0, dirs = 0;
            if (v) {
                bump_class(cc, Q.cls[j]);
                dirs = route(h, Q.cls[j], Q.ts[j], bin, oor);
            }
            const uint32_t key = dirs ? (bin << 1 | (dirs & 1u ? 0u : 1u)) : kNoKey;
            update_agg(h, hc, key, Q.by[j]);
            if (h.two_dir) {
                const bool both = dirs == 3u;
                if (__any_sync(kFull, both)) update_agg(h, hc, both ? (bin << 1 | 1u) : kNoKey, Q.by[j]);
            }
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
        const uint32_t c = hc.cnt[i];
        if (c) gadd(h, hc.keys[i] & 1u, hc.keys[i] >> 1, c, (uint64_t)hc.hi[i] << 32 | hc.lo[i]);
    }
    flush_counters(h.stats, cc, oor, true);
    if (WATCH) flush_filtered(h.stats, flt);
}

// ---------------------------------------------------------------------------
// Shared-memory privatised bins. A CTA takes chunks of blockDim * iters quads
// (at most 65,535 records); for each chunk it places a tile of `tile_bins`
// bins per direction just below the chunk's first record (time-sorted input
// keeps the chunk inside it). A tile entry is two 32-bit words updated with
// native shared atomics: the low 32 bits of the byte sum, and a high word
// holding the record count in its upper 16 bits and the byte sum's bits
// 32-47 in its lower 16 (a bin of one chunk holds at most 65,535 records,
// whose bytes sum below 2^48). The touched part of the tile is flushed with
// global atomics after the chunk. Records outside the tile go straight to
// global atomics. With `full`, the tile is the whole histogram (base 0).
template <int LK, bool W1>
__global__ void __launch_bounds__(1024) k_fused_tile(RecArgs r, TableArgs t, HistArgs h, TileArgs ta,
                                                     uint32_t *status) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t s_base, s_lo, s_hi;
    __shared__ unsigned long long s_cnt[6];
    Classifier<LK> C;
    if (!C.init(t, smem, &bar, status)) return;  // table not staged: the status word says so
    const uint32_t T = ta.tile_bins;
    uint32_t *tlo = reinterpret_cast<uint32_t *>(smem + ((Classifier<LK>::smem_bytes(t) + 15u) & ~15u));
    uint32_t *thi = tlo + 2 * T;
    for (uint32_t i = threadIdx.x; i < 2 * T; i += blockDim.x) {
        tlo[i] = 0;
        thi[i] = 0;
    }
    if (threadIdx.x == 0) {
        s_lo = 0xFFFFFFFFu;
        s_hi = 0;
    }
    if (threadIdx.x < 6) s_cnt[threadIdx.x] = 0;
    const uint64_t pol = policy_evict_first();
    uint64_t ccp = 0;   // packed per-thread class counts, drained every chunk
    uint32_t oorp = 0;  // packed per-thread out-of-window counts
    const uint64_t qpc = (uint64_t)blockDim.x * ta.iters;
    const uint64_t n_chunks = (r.g.quads + qpc - 1) / qpc;
    const uint32_t lane = threadIdx.x & 31;
    // thread 0 places each chunk's tile from the chunk's first timestamp,
    // loaded one chunk ahead so the CTA does not wait on it at the barrier
    uint64_t ts_first = 0;
    if (!ta.full && threadIdx.x == 0 && blockIdx.x < n_chunks) {
        int64_t i0 = quad_base(r.g, (uint64_t)blockIdx.x * qpc);
        ts_first = r.ts[i0 < 0 ? 0 : i0];
    }
    __syncthreads();

    for (uint64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        uint32_t base = 0;
        if (!ta.full) {
            if (threadIdx.x == 0) {
                uint32_t b = 0;
                const uint64_t rel = ts_first - h.t0;
                if (rel < h.span) {
                    b = h.w_is_one ? (uint32_t)rel : (uint32_t)divide(rel, h.div);
                    b = b > ta.margin ? b - ta.margin : 0u;
                }
                s_base = b;
                if (ch + gridDim.x < n_chunks) {
                    const int64_t i1 = quad_base(r.g, (ch + gridDim.x) * qpc);
                    ts_first = r.ts[i1 < 0 ? 0 : i1];
                }
            }
            __syncthreads();
            base = s_base;
        }
        uint32_t omin = 0xFFFFFFFFu, omax = 0;
        for (uint32_t it = 0; it < ta.iters; ++it) {
            const uint64_t q = ch * qpc + (uint64_t)it * blockDim.x + threadIdx.x;
            Quad Q;
            load_quad<true, LK != LK_CLASS_IN, true, LK == LK_CLASS_IN>(r, q, pol, Q);
            uint32_t bins[4];
            const uint32_t inr = bin_quad<W1>(h, Q, bins);
            classify_quad<LK>(C, Q);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!(Q.valid >> j & 1u)) continue;
                bump_class_packed(ccp, Q.cls[j]);
                const uint32_t bin = bins[j];
                const uint32_t dirs = dirs_of_packed(h, Q.cls[j], inr >> j & 1u, oorp);
                if (!dirs) continue;
                const uint32_t off = bin - base;
                if (off < T) {
                    omin = min(omin, off);
                    omax = max(omax, off);
                    const uint32_t e = (dirs & 1u) ? off : T + off;
                    smem_add_wide(tlo + e, thi + e, Q.by[j], 1u << 16);
                    if (dirs == 3u) smem_add_wide(tlo + T + off, thi + T + off, Q.by[j], 1u << 16);
                } else {
                    gadd(h, (dirs & 1u) ? 0u : 1u, bin, 1u, Q.by[j]);
                    if (dirs == 3u) gadd(h, 1u, bin, 1u, Q.by[j]);
                }
            }
        }
        drain_packed(ccp, oorp, s_cnt);
        // touched range of the tile, then flush it
        omin = __reduce_min_sync(kFull, omin);
        omax = __reduce_max_sync(kFull, omax);
        if (lane == 0 && omin <= omax) {
            atomicMin(&s_lo, omin);
            atomicMax(&s_hi, omax);
        }
        __syncthreads();
        const uint32_t lo = s_lo, hi = s_hi;
        if (lo <= hi) {
            // consecutive lanes take consecutive bins, so each warp-wide global
            // atomic covers as few sectors as possible
            const uint32_t n = hi - lo + 1;
            for (uint32_t i = threadIdx.x; i < 2 * n; i += blockDim.x) {
                const uint32_t d = i >= n;
                const uint32_t off = lo + i - d * n;
                const uint32_t e = d * T + off;
                const uint32_t vh = thi[e];
                if (vh) {
                    gadd(h, d, base + off, vh >> 16, (uint64_t)(vh & 0xFFFFu) << 32 | tlo[e]);
                    tlo[e] = 0;
                    thi[e] = 0;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_lo = 0xFFFFFFFFu;
            s_hi = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x < 6 && s_cnt[threadIdx.x])
        atomicAdd(reinterpret_cast<unsigned long long *>(h.stats) + threadIdx.x, s_cnt[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// Binning alone: the bin of each record, or kNoKey outside the window.
__global__ void __launch_bounds__(256) k_bin(const uint64_t *ts, uint64_t n, HistArgs h, uint32_t *bin) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t rel = ts[i] - h.t0;
        bin[i] = rel < h.span ? (uint32_t)divide(rel, h.div) : kNoKey;
    }
}

cudaError_t run_bin(const uint64_t *ts, uint64_t n, const HistArgs &h, uint32_t *bin, const LaunchCfg &c) {
    k_bin<<<8 * c.sm_count, 256, 0, c.stream>>>(ts, n, h, bin);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cell expansion: one thread per bin reads its 32-byte cell and writes (or
// adds to) the four output arrays; consecutive threads write consecutive bins.
__global__ void __launch_bounds__(256) k_cells_expand(HistArgs h, uint32_t accumulate) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < h.n_bins; b += stride) {
        const ulonglong2 sums = __ldcs(reinterpret_cast<const ulonglong2 *>(h.cells + 4 * b));
        const ulonglong2 cnts = __ldcs(reinterpret_cast<const ulonglong2 *>(h.cells + 4 * b + 2));
        uint32_t c0 = (uint32_t)cnts.x, c1 = (uint32_t)(cnts.x >> 32);
        uint64_t s0 = sums.x, s1 = sums.y;
        if (accumulate) {
            c0 += h.cnt[0][b];
            c1 += h.cnt[1][b];
            s0 += h.byt[0][b];
            s1 += h.byt[1][b];
        }
        h.cnt[0][b] = c0;
        h.cnt[1][b] = c1;
        h.byt[0][b] = s0;
        h.byt[1][b] = s1;
    }
}

// ---------------------------------------------------------------------------
// Host launchers.

size_t smem_optin_limit() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)v;
}

template <typename K>
static cudaError_t launch(K kernel, size_t smem, const LaunchCfg &c, int &grid) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    grid = c.grid;
    if (grid <= 0) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, c.block, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid = per_sm * c.sm_count;
    }
    return cudaSuccess;
}

cudaError_t run_cells_expand(const HistArgs &h, bool accumulate, const LaunchCfg &c) {
    const int grid = 8 * c.sm_count;
    k_cells_expand<<<grid, 256, 0, c.stream>>>(h, accumulate ? 1u : 0u);
    return cudaGetLastError();
}

cudaError_t run_discriminate(int lk, const RecArgs &r, const TableArgs &t, uint64_t *counts,
                             const LaunchCfg &c) {
    int grid = 0;
    cudaError_t e;
    switch (lk) {
#define SINET_DISC(L)                                                                           \
    case L: {                                                                                   \
        size_t smem = Classifier<L>::smem_bytes(t);                                             \
        if ((e = launch(k_discriminate<L>, smem, c, grid)) != cudaSuccess) return e;            \
        k_discriminate<L><<<grid, c.block, smem, c.stream>>>(r, t, counts, c.status);           \
        break;                                                                                  \
    }
        SINET_DISC(LK_INTERVAL)
        SINET_DISC(LK_TOGGLE1)
        SINET_DISC(LK_TOGGLE2)
        SINET_DISC(LK_PML)
        SINET_DISC(LK_INTERVAL_GLOBAL)
#undef SINET_DISC
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t run_fused_atomic(int lk, bool agg, const RecArgs &r, const TableArgs &t,
                             const HistArgs &h, uint32_t cache_set_bits, const LaunchCfg &c,
                             const TableArgs *watch) {
    int grid = 0;
    cudaError_t e;
    const TableArgs none{};
#define SINET_ATOM(L, A, WA)                                                                    \
    if (lk == L && agg == A && (watch != nullptr) == WA) {                                      \
        size_t smem = ((Classifier<L>::smem_bytes(t) + 15u) & ~15u) +                           \
                      (A ? (size_t)HotCache::kSlotBytes * (HotCache::kWays << cache_set_bits) : 0ull);                 \
        if ((e = launch(k_fused_atomic<L, A, WA>, smem, c, grid)) != cudaSuccess) return e;     \
        k_fused_atomic<L, A, WA><<<grid, c.block, smem, c.stream>>>(r, t, h, cache_set_bits,     \
                                                                   WA ? *watch : none, c.status); \
        return cudaGetLastError();                                                              \
    }
#define SINET_ATOM2(L, WA) SINET_ATOM(L, true, WA) SINET_ATOM(L, false, WA)
    SINET_ATOM2(LK_INTERVAL, false)
    SINET_ATOM2(LK_TOGGLE1, false)
    SINET_ATOM2(LK_TOGGLE2, false)
    SINET_ATOM2(LK_PML, false)
    SINET_ATOM2(LK_INTERVAL_GLOBAL, false)
    SINET_ATOM2(LK_CLASS_IN, false)
    SINET_ATOM2(LK_INTERVAL, true)
    SINET_ATOM2(LK_TOGGLE1, true)
    SINET_ATOM2(LK_TOGGLE2, true)
    SINET_ATOM2(LK_INTERVAL_GLOBAL, true)
#undef SINET_ATOM2
#undef SINET_ATOM
    return cudaErrorInvalidValue;
}

cudaError_t run_fused_tile(int lk, const RecArgs &r, const TableArgs &t, const HistArgs &h,
                           const TileArgs &ta, const LaunchCfg &c) {
    int grid = 0;
    cudaError_t e;
    const bool w1 = h.w_is_one != 0;
#define SINET_TILE(L, W)                                                                        \
    if (lk == L && w1 == W) {                                                                   \
        size_t smem = ((Classifier<L>::smem_bytes(t) + 15u) & ~15u) + 16ull * ta.tile_bins;     \
        if ((e = launch(k_fused_tile<L, W>, smem, c, grid)) != cudaSuccess) return e;           \
        k_fused_tile<L, W><<<grid, c.block, smem, c.stream>>>(r, t, h, ta, c.status);           \
        return cudaGetLastError();                                                              \
    }
    SINET_TILE(LK_INTERVAL, true)
    SINET_TILE(LK_INTERVAL, false)
    SINET_TILE(LK_TOGGLE1, true)
    SINET_TILE(LK_TOGGLE1, false)
    SINET_TILE(LK_TOGGLE2, true)
    SINET_TILE(LK_TOGGLE2, false)
    SINET_TILE(LK_PML, true)
    SINET_TILE(LK_PML, false)
    SINET_TILE(LK_INTERVAL_GLOBAL, true)
    SINET_TILE(LK_INTERVAL_GLOBAL, false)
    SINET_TILE(LK_CLASS_IN, true)
    SINET_TILE(LK_CLASS_IN, false)
#undef SINET_TILE
    return cudaErrorInvalidValue;
}

}  // namespace sinet
