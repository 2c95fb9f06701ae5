// The plain path, after the paper's structure (Section 5, "Pairwise Reduction
// Pattern with GPU": Thrust sort then reduce-by-key into <timestamp, count>
// and <timestamp, bytes>), written out by hand:
//   1. emit:   Algorithm 1 + routing + binning; every routed in-window record
//              becomes a (key = d * n_bins + bin, bytes) pair, compacted with a
//              decoupled look-back scan; per-pass digit counts are taken here.
//   2. sort:   LSD radix sort of the pairs, 8-bit digits, one kernel per pass
//              (tile ranking with warp match, per-digit decoupled look-back).
//   3. reduce: reduce-by-key over the sorted pairs (segmented scan per tile);
//              each run's count and byte sum is scattered into the dense
//              histogram (runs that cross a tile edge are added atomically).
#include "launch.h"

namespace sinet {

namespace {

constexpr int kEmitThreads = 256;
constexpr int kEmitQuadsPerThread = 4;               // 16 records per thread
constexpr int kEmitRecords = kEmitThreads * kEmitQuadsPerThread * 4;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys
constexpr int kWarps = kSortThreads / 32;

constexpr uint64_t kFlagAgg = 1ull << 54;
constexpr uint64_t kFlagIncl = 2ull << 54;
constexpr uint64_t kValMask = (1ull << 54) - 1;

__device__ __forceinline__ uint64_t ld_acquire(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Status word: epoch (8 bits) | flags (2 bits) | value (54 bits). A word whose
// epoch differs from the reader's is "not ready yet".
__device__ __forceinline__ uint64_t status_word(uint32_t epoch, uint64_t flag, uint64_t v) {
    return (uint64_t)epoch << 56 | flag | (v & kValMask);
}

// Exclusive prefix of `own` over all predecessor tiles (decoupled look-back).
// Publishes the aggregate, walks back until an inclusive prefix, publishes the
// inclusive value. Bounded: a wait that runs out latches SINET_ERR_TIMEOUT.
__device__ uint64_t look_back(uint64_t *st, uint64_t stride, uint64_t tile, uint64_t own,
                              uint32_t epoch, uint32_t *status) {
    if (tile == 0) {
        st_release(st, status_word(epoch, kFlagIncl, own));
        return 0;
    }
    st_release(st + tile * stride, status_word(epoch, kFlagAgg, own));
    uint64_t excl = 0;
    for (int64_t p = (int64_t)tile - 1; p >= 0; --p) {
        uint64_t w = 0;
        uint32_t it = 0;
        for (; it < kSpinLimit; ++it) {
            w = ld_acquire(st + (uint64_t)p * stride);
            if ((uint32_t)(w >> 56) == epoch && (w & (kFlagAgg | kFlagIncl))) break;
        }
        if (it == kSpinLimit) {
            latch_status(status, SINET_ERR_TIMEOUT);
            break;
        }
        excl += w & kValMask;
        if (w & kFlagIncl) break;
    }
    st_release(st + tile * stride, status_word(epoch, kFlagIncl, excl + own));
    return excl;
}

struct SortArgs {
    uint32_t *keys0, *vals0, *keys1, *vals1;
    uint32_t *digit_hist;    // [passes][256]
    uint64_t *emit_status;   // [emit tiles]
    uint64_t *sort_status;   // [sort tiles][256]
    uint64_t *counters;      // [0] n_emit, [1] emit ticket, [2 + p] pass tickets, [8] reduce ticket
    uint32_t n_bins;
    uint32_t passes;
};

// ---------------------------------------------------------------------------
// 1. emit
template <int LK>
__global__ void __launch_bounds__(kEmitThreads) k_emit(RecArgs r, TableArgs t, HistArgs h,
                                                       SortArgs sa, uint64_t n_tiles,
                                                       uint32_t *status) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t s_hist[4][256];
    __shared__ uint32_t s_warp[kEmitThreads / 32];
    __shared__ uint64_t s_tile, s_goff;
    Classifier<LK> C;
    // a table that did not land leaves this tile's records out (the status
    // word says so), but the tile still takes part in the look-back chain
    const bool tab_ok = C.init(t, smem, &bar, status);
    const uint32_t tsm = (Classifier<LK>::smem_bytes(t) + 15u) & ~15u;
    uint32_t *skey = reinterpret_cast<uint32_t *>(smem + tsm);
    const uint32_t cap = kEmitRecords * (h.two_dir ? 2 : 1);
    uint32_t *sval = skey + cap;
    for (uint32_t i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&s_hist[0][0])[i] = 0;
    if (threadIdx.x == 0) s_tile = atomicAdd(reinterpret_cast<unsigned long long *>(sa.counters + 1), 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t pol = policy_evict_first();
    uint32_t cc[4] = {0, 0, 0, 0}, oor[2] = {0, 0};

    uint32_t key[kEmitQuadsPerThread * 4], val[kEmitQuadsPerThread * 4];
    uint32_t both = 0, n_mine = 0;
#pragma unroll
    for (int it = 0; it < kEmitQuadsPerThread; ++it) {
        const uint64_t q = tile * (kEmitThreads * kEmitQuadsPerThread) + (uint64_t)it * kEmitThreads + threadIdx.x;
        Quad Q;
        load_quad<true, LK != LK_CLASS_IN, true, LK == LK_CLASS_IN>(r, q, pol, Q);
        if (!tab_ok) Q.valid = 0;
        classify_quad<LK>(C, Q);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = it * 4 + j;
            key[k] = kNoKey;
            val[k] = Q.by[j];
            if (!(Q.valid >> j & 1u)) continue;
            bump_class(cc, Q.cls[j]);
            uint32_t bin;
            const uint32_t dirs = route(h, Q.cls[j], Q.ts[j], bin, oor);
            if (!dirs) continue;
            key[k] = (dirs & 1u) ? bin : h.n_bins + bin;
            n_mine++;
            if (dirs == 3u) {
                both |= 1u << k;
                n_mine++;
            }
        }
    }
    // block exclusive scan of the per-thread emit counts
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = n_mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t woff = 0, total = 0;
    for (uint32_t w = 0; w < kEmitThreads / 32; ++w) {
        if (w < warp) woff += s_warp[w];
        total += s_warp[w];
    }
    uint32_t pos = woff + incl - n_mine;
#pragma unroll
    for (int k = 0; k < kEmitQuadsPerThread * 4; ++k) {
        if (key[k] == kNoKey) continue;
        skey[pos] = key[k];
        sval[pos] = val[k];
        pos++;
        if (both >> k & 1u) {
            skey[pos] = h.n_bins + key[k];
            sval[pos] = val[k];
            pos++;
        }
    }
    __syncthreads();
    // digit counts for every radix pass
    for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
        const uint32_t k = skey[i];
        for (uint32_t p = 0; p < sa.passes; ++p) atomicAdd(&s_hist[p][(k >> (8 * p)) & 255u], 1u);
    }
    if (threadIdx.x == 0) {
        s_goff = look_back(sa.emit_status, 1, tile, total, 1, status);
        if (tile == n_tiles - 1) sa.counters[0] = s_goff + total;
    }
    __syncthreads();
    const uint64_t goff = s_goff;
    for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
        sa.keys0[goff + i] = skey[i];
        sa.vals0[goff + i] = sval[i];
    }
    for (uint32_t i = threadIdx.x; i < sa.passes * 256; i += blockDim.x) {
        const uint32_t v = (&s_hist[0][0])[i];
        if (v) atomicAdd(sa.digit_hist + i, v);
    }
    flush_counters(h.stats, cc, oor, true);
}

// Block-wide exclusive scan of one value per thread (256 threads).
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t *s_warp, uint32_t &total) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= (uint32_t)o) incl += y;
    }
    __syncthreads();
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t woff = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        if (w < (int)warp) woff += s_warp[w];
        total += s_warp[w];
    }
    return woff + incl - v;
}

// ---------------------------------------------------------------------------
// 2. one LSD radix pass on bits [8p, 8p + 8)
__global__ void __launch_bounds__(kSortThreads) k_radix_pass(SortArgs sa, uint32_t p,
                                                             const uint32_t *kin, const uint32_t *vin,
                                                             uint32_t *kout, uint32_t *vout,
                                                             uint32_t *status) {
    __shared__ uint32_t s_key[kSortTile];
    __shared__ uint32_t s_val[kSortTile];
    __shared__ uint32_t s_whist[kWarps][257];
    __shared__ uint32_t s_lstart[256];
    __shared__ uint64_t s_gpos[256];
    __shared__ uint32_t s_warp[kWarps];
    __shared__ uint64_t s_tile;
    const uint64_t n = sa.counters[0];
    if (threadIdx.x == 0) s_tile = atomicAdd(reinterpret_cast<unsigned long long *>(sa.counters + 2 + p), 1ull);
    for (uint32_t i = threadIdx.x; i < kWarps * 257; i += blockDim.x) (&s_whist[0][0])[i] = 0;
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t tbase = tile * kSortTile;
    if (tbase >= n) return;  // block-uniform
    const uint32_t shift = 8 * p;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;

    // warp-striped load: item j of lane l is tile position warp*512 + j*32 + l
    uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint64_t i = tbase + (uint64_t)warp * (32 * kSortItems) + j * 32 + lane;
        key[j] = i < n ? kin[i] : kNoKey;
        val[j] = i < n ? vin[i] : 0u;
    }
    // rank within the warp, in position order (stable)
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint64_t i = tbase + (uint64_t)warp * (32 * kSortItems) + j * 32 + lane;
        const uint32_t dg = i < n ? (key[j] >> shift) & 255u : 256u;
        const uint32_t peers = __match_any_sync(kFull, dg);
        const uint32_t leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader) {
            old = s_whist[warp][dg];
            s_whist[warp][dg] = old + __popc(peers);
        }
        old = __shfl_sync(kFull, old, leader);
        rank[j] = old + __popc(peers & lt_mask);
        __syncwarp();
    }
    __syncthreads();
    // per digit: warp offsets and the tile count
    const uint32_t d = threadIdx.x;  // 256 threads, one digit each
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = s_whist[w][d];
        s_whist[w][d] = cnt;
        cnt += c;
    }
    uint32_t tot;
    const uint32_t lstart = block_excl_scan_256(cnt, s_warp, tot);
    s_lstart[d] = lstart;
    // global position of this tile's run of digit d
    {
        // digit start = exclusive scan of the global digit counts of this pass
        uint32_t gt;
        const uint32_t gstart = block_excl_scan_256(sa.digit_hist[p * 256 + d], s_warp, gt);
        const uint64_t excl = look_back(sa.sort_status + d, 256, tile, cnt, p + 1, status);
        s_gpos[d] = (uint64_t)gstart + excl;
    }
    __syncthreads();
    // scatter into the tile in sorted order
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        if (key[j] == kNoKey && (tbase + (uint64_t)warp * (32 * kSortItems) + j * 32 + lane) >= n) continue;
        const uint32_t dg = (key[j] >> shift) & 255u;
        const uint32_t at = s_lstart[dg] + s_whist[warp][dg] + rank[j];
        s_key[at] = key[j];
        s_val[at] = val[j];
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < tot; k += blockDim.x) {
        const uint32_t kk = s_key[k];
        const uint32_t dg = (kk >> shift) & 255u;
        const uint64_t at = s_gpos[dg] + (k - s_lstart[dg]);
        kout[at] = kk;
        vout[at] = s_val[k];
    }
}

// ---------------------------------------------------------------------------
// 3. reduce by key + dense scatter
struct Run {
    uint32_t f;  // a run head lies inside
    uint32_t c;
    uint64_t s;
};
__device__ __forceinline__ Run seg_op(const Run &a, const Run &b) {
    Run r;
    r.f = a.f | b.f;
    r.c = b.f ? b.c : a.c + b.c;
    r.s = b.f ? b.s : a.s + b.s;
    return r;
}

__global__ void __launch_bounds__(kSortThreads) k_reduce(SortArgs sa, const uint32_t *keys,
                                                         const uint32_t *vals, HistArgs h,
                                                         int accumulate) {
    __shared__ Run s_warp[kWarps];
    __shared__ uint32_t s_last[kSortThreads];
    const uint64_t n = sa.counters[0];
    const uint64_t tbase = (uint64_t)blockIdx.x * kSortTile;
    if (tbase >= n) return;
    const uint64_t tend = tbase + kSortTile < n ? tbase + kSortTile : n;
    const uint32_t prev_key = tbase > 0 ? keys[tbase - 1] : kNoKey;
    const uint32_t next_key = tend < n ? keys[tend] : kNoKey;
    const uint64_t mine = tbase + (uint64_t)threadIdx.x * kSortItems;
    uint32_t k[kSortItems], v[kSortItems];
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const uint64_t at = mine + i;
        k[i] = at < tend ? keys[at] : kNoKey;
        v[i] = at < tend ? vals[at] : 0u;
    }
    // last valid key of each thread, for the next thread's first head test
    uint32_t last = kNoKey;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i)
        if (mine + i < tend) last = k[i];
    s_last[threadIdx.x] = last;
    __syncthreads();
    const uint32_t pred = threadIdx.x == 0 ? prev_key : s_last[threadIdx.x - 1];
    // thread summary: trailing partial run
    Run agg = {0u, 0u, 0ull};
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        if (mine + i >= tend) break;
        const uint32_t before = i == 0 ? pred : k[i - 1];
        if (k[i] != before) {
            agg.f = 1;
            agg.c = 0;
            agg.s = 0;
        }
        agg.c += 1;
        agg.s += v[i];
    }
    // block exclusive segmented scan of the summaries
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Run inc = agg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        Run y;
        y.f = __shfl_up_sync(kFull, inc.f, o);
        y.c = __shfl_up_sync(kFull, inc.c, o);
        y.s = __shfl_up_sync(kFull, inc.s, o);
        if (lane >= (uint32_t)o) inc = seg_op(y, inc);
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    Run wpre = {0u, 0u, 0ull};
    for (uint32_t w = 0; w < warp; ++w) wpre = seg_op(wpre, s_warp[w]);
    Run ex;
    ex.f = __shfl_up_sync(kFull, inc.f, 1);
    ex.c = __shfl_up_sync(kFull, inc.c, 1);
    ex.s = __shfl_up_sync(kFull, inc.s, 1);
    if (lane == 0) ex = Run{0u, 0u, 0ull};
    const Run carry = seg_op(wpre, ex);
    // walk the items: each run is written at its tail
    uint32_t rc = carry.c;
    uint64_t rs = carry.s;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const uint64_t at = mine + i;
        if (at >= tend) break;
        const uint32_t before = i == 0 ? pred : k[i - 1];
        if (k[i] != before) {
            rc = 0;
            rs = 0;
        }
        rc += 1;
        rs += v[i];
        const bool tile_last = at + 1 == tend;
        const uint32_t after = tile_last ? next_key : (i + 1 < kSortItems ? k[i + 1] : keys[at + 1]);
        const bool tail = k[i] != after;
        if (tail || tile_last) {
            const uint32_t key = k[i];
            const uint32_t d = key >= h.n_bins;
            const uint32_t bin = key - d * h.n_bins;
            const bool shared = (key == prev_key) || (tile_last && key == next_key);
            uint32_t *cp = d ? h.cnt[1] : h.cnt[0];
            uint64_t *bp = d ? h.byt[1] : h.byt[0];
            if (shared) {
                atomicAdd(cp + bin, rc);
                atomicAdd(reinterpret_cast<unsigned long long *>(bp + bin), (unsigned long long)rs);
            } else if (accumulate) {
                cp[bin] += rc;
                bp[bin] += rs;
            } else {
                cp[bin] = rc;
                bp[bin] = rs;
            }
        }
    }
}

}  // namespace

SortPlan plan_sort_reduce(uint64_t n, uint32_t n_bins, bool two_dir) {
    SortPlan p{};
    p.n_emit_max = n * (two_dir ? 2 : 1);
    const uint64_t key_space = 2ull * n_bins;  // keys < 2 * n_bins
    uint32_t bits = 1;
    while (bits < 32 && (1ull << bits) < key_space) bits++;
    p.key_bits = bits;
    p.passes = (bits + 7) / 8;
    const uint64_t quads = n / 4 + 2;
    p.emit_tiles = (quads + kEmitThreads * kEmitQuadsPerThread - 1) / (kEmitThreads * kEmitQuadsPerThread);
    p.sort_tiles = (p.n_emit_max + kSortTile - 1) / kSortTile;
    if (p.sort_tiles == 0) p.sort_tiles = 1;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    p.off_counters = off;
    off += al(16 * 8);
    p.off_hist = off;
    off += al(4 * 256 * 4);
    p.off_emit_status = off;
    off += al(8 * (p.emit_tiles + 1));
    const size_t small_end = off;
    p.off_sort_status = off;
    off += al(8ull * 256 * p.sort_tiles);
    p.off_keys0 = off;
    off += al(4 * p.n_emit_max + 4);
    p.off_vals0 = off;
    off += al(4 * p.n_emit_max + 4);
    p.off_keys1 = off;
    off += al(4 * p.n_emit_max + 4);
    p.off_vals1 = off;
    off += al(4 * p.n_emit_max + 4);
    p.scratch_bytes = off;
    (void)small_end;
    return p;
}

cudaError_t run_sort_reduce(int lk, const RecArgs &r, const TableArgs &t, const HistArgs &h,
                            const SortPlan &plan, void *scratch, bool accumulate,
                            const LaunchCfg &c) {
    uint8_t *base = static_cast<uint8_t *>(scratch);
    SortArgs sa;
    sa.counters = reinterpret_cast<uint64_t *>(base + plan.off_counters);
    sa.digit_hist = reinterpret_cast<uint32_t *>(base + plan.off_hist);
    sa.emit_status = reinterpret_cast<uint64_t *>(base + plan.off_emit_status);
    sa.sort_status = reinterpret_cast<uint64_t *>(base + plan.off_sort_status);
    sa.keys0 = reinterpret_cast<uint32_t *>(base + plan.off_keys0);
    sa.vals0 = reinterpret_cast<uint32_t *>(base + plan.off_vals0);
    sa.keys1 = reinterpret_cast<uint32_t *>(base + plan.off_keys1);
    sa.vals1 = reinterpret_cast<uint32_t *>(base + plan.off_vals1);
    sa.n_bins = h.n_bins;
    sa.passes = plan.passes;
    // counters, digit counts, emit and sort look-back words start at zero
    cudaError_t e = cudaMemsetAsync(base, 0, plan.off_keys0, c.stream);
    if (e != cudaSuccess) return e;
    if (r.g.quads == 0) return cudaSuccess;

    const uint32_t tsm = (lk == LK_INTERVAL || lk == LK_TOGGLE1 || lk == LK_TOGGLE2 ? Classifier<LK_INTERVAL>::smem_bytes(t)
                          : lk == LK_PML    ? Classifier<LK_PML>::smem_bytes(t)
                                            : 0u);
    const size_t smem = ((tsm + 15u) & ~15u) + 8ull * kEmitRecords * (h.two_dir ? 2 : 1);
    switch (lk) {
#define SINET_EMIT(L)                                                                          \
    case L:                                                                                    \
        e = cudaFuncSetAttribute(k_emit<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                        \
        k_emit<L><<<(unsigned)plan.emit_tiles, kEmitThreads, smem, c.stream>>>(r, t, h, sa,    \
                                                                              plan.emit_tiles, c.status); \
        break;
        SINET_EMIT(LK_INTERVAL)
        SINET_EMIT(LK_TOGGLE1)
        SINET_EMIT(LK_TOGGLE2)
        SINET_EMIT(LK_PML)
        SINET_EMIT(LK_INTERVAL_GLOBAL)
        SINET_EMIT(LK_CLASS_IN)
#undef SINET_EMIT
        default:
            return cudaErrorInvalidValue;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    uint32_t *kin = sa.keys0, *vin = sa.vals0, *kout = sa.keys1, *vout = sa.vals1;
    for (uint32_t p = 0; p < plan.passes; ++p) {
        k_radix_pass<<<(unsigned)plan.sort_tiles, kSortThreads, 0, c.stream>>>(sa, p, kin, vin, kout, vout,
                                                                               c.status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        uint32_t *tk = kin, *tv = vin;
        kin = kout;
        vin = vout;
        kout = tk;
        vout = tv;
    }
    k_reduce<<<(unsigned)plan.sort_tiles, kSortThreads, 0, c.stream>>>(sa, kin, vin, h, accumulate ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace sinet
