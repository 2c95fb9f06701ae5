// Discriminate-only and fused discriminate + histogram kernels (sm_103a).
//
// One pass over the SoA records: 128-bit streaming loads of 4 records per
// thread, Algorithm 1 against the shared-memory-staged table, routing by the
// class policy, millisecond binning, and the histogram update of Section 5
// (a merge-scatter with the associative, commutative integer +).
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
    C.init(t, smem, &bar, status);
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

// ---------------------------------------------------------------------------
// Warp run-combining: lanes holding the same (bin, direction) key elect a
// leader that adds the group's count (popc of the peer mask) and byte sum.
// Byte sums are reduced as two 16-bit halves so 32 values of up to 2^32 - 1
// cannot overflow the 32-bit warp reduction; they are recombined in 64 bits.
template <bool AGG>
__device__ __forceinline__ void update_global(const HistArgs &h, uint32_t key, uint32_t b) {
    if (!AGG) {
        if (key != kNoKey) gadd(h, key & 1u, key >> 1, 1u, b);
        return;
    }
    const uint32_t peers = __match_any_sync(kFull, key);
    if (key == kNoKey) return;
    const uint32_t c = __popc(peers);
    uint64_t s = b;
    if (c > 1) {
        const uint32_t lo = __reduce_add_sync(peers, b & 0xFFFFu);
        const uint32_t hi = __reduce_add_sync(peers, b >> 16);
        s = (uint64_t)lo + ((uint64_t)hi << 16);
    }
    if ((threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1)) gadd(h, key & 1u, key >> 1, c, s);
}

template <int LK, bool AGG>
__global__ void __launch_bounds__(256) k_fused_atomic(RecArgs r, TableArgs t, HistArgs h,
                                                      uint32_t *status) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t bar;
    Classifier<LK> C;
    C.init(t, smem, &bar, status);
    const uint64_t pol = policy_evict_first();
    uint32_t cc[4] = {0, 0, 0, 0}, oor[2] = {0, 0};
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // warp-uniform trip count: every lane reaches the warp-synchronous updates
    for (uint64_t q0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) - lane; q0 < r.g.quads;
         q0 += stride) {
        Quad Q;
        load_quad<true, LK != LK_CLASS_IN, true, LK == LK_CLASS_IN>(r, q0 + lane, pol, Q);
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
            update_global<AGG>(h, key, Q.by[j]);
            if (h.two_dir) {
                const bool both = dirs == 3u;
                if (AGG ? __any_sync(kFull, both) : both)
                    update_global<AGG>(h, both ? (bin << 1 | 1u) : kNoKey, Q.by[j]);
            }
        }
    }
    flush_counters(h.stats, cc, oor, true);
}

// ---------------------------------------------------------------------------
// Shared-memory privatised bins. A CTA takes chunks of blockDim * iters quads;
// for each chunk it places a tile of `tile_bins` bins per direction just
// below the chunk's first record (time-sorted input keeps the chunk inside
// it), adds in shared memory, and flushes the non-zero bins with global
// atomics. Records outside the tile go straight to global atomics. With
// `full`, the tile is the whole histogram and is flushed once at the end.
template <int LK>
__global__ void __launch_bounds__(256) k_fused_tile(RecArgs r, TableArgs t, HistArgs h, TileArgs ta,
                                                    uint32_t *status) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t s_base;
    Classifier<LK> C;
    C.init(t, smem, &bar, status);
    const uint32_t T = ta.tile_bins;
    uint8_t *tile_mem = smem + ((Classifier<LK>::smem_bytes(t) + 15u) & ~15u);
    uint64_t *tb = reinterpret_cast<uint64_t *>(tile_mem);            // [2][T] byte sums
    uint32_t *tc = reinterpret_cast<uint32_t *>(tile_mem + 16ull * T);  // [2][T] counts
    for (uint32_t i = threadIdx.x; i < 2 * T; i += blockDim.x) {
        tb[i] = 0;
        tc[i] = 0;
    }
    const uint64_t pol = policy_evict_first();
    uint32_t cc[4] = {0, 0, 0, 0}, oor[2] = {0, 0};
    const uint64_t qpc = (uint64_t)blockDim.x * ta.iters;
    const uint64_t n_chunks = (r.g.quads + qpc - 1) / qpc;
    uint32_t base = 0;
    __syncthreads();

    for (uint64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        if (!ta.full) {
            if (threadIdx.x == 0) {
                int64_t i0 = quad_base(r.g, ch * qpc);
                if (i0 < 0) i0 = 0;
                uint32_t b = 0;
                uint64_t rel = r.ts[i0] - h.t0;
                if (rel < h.span) {
                    b = h.w_is_one ? (uint32_t)rel : (uint32_t)divide(rel, h.div);
                    b = b > ta.margin ? b - ta.margin : 0u;
                }
                s_base = b;
            }
            __syncthreads();
            base = s_base;
        }
        for (uint32_t it = 0; it < ta.iters; ++it) {
            const uint64_t q = ch * qpc + (uint64_t)it * blockDim.x + threadIdx.x;
            Quad Q;
            load_quad<true, LK != LK_CLASS_IN, true, LK == LK_CLASS_IN>(r, q, pol, Q);
            classify_quad<LK>(C, Q);
            // combine runs of equal (bin, direction) inside the quad before
            // touching shared memory (sorted input repeats bins)
            uint32_t pk = kNoKey, pc = 0;
            uint64_t ps = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!(Q.valid >> j & 1u)) continue;
                bump_class(cc, Q.cls[j]);
                uint32_t bin;
                const uint32_t dirs = route(h, Q.cls[j], Q.ts[j], bin, oor);
                if (!dirs) continue;
                const uint32_t key = bin << 1 | (dirs & 1u ? 0u : 1u);
                if (key == pk) {
                    pc++;
                    ps += Q.by[j];
                } else {
                    if (pk != kNoKey) {
                        const uint32_t pd = pk & 1u, off = (pk >> 1) - base;
                        if (off < T) {
                            atomicAdd(tc + pd * T + off, pc);
                            atomicAdd(reinterpret_cast<unsigned long long *>(tb + pd * T + off),
                                      (unsigned long long)ps);
                        } else {
                            gadd(h, pd, pk >> 1, pc, ps);
                        }
                    }
                    pk = key;
                    pc = 1;
                    ps = Q.by[j];
                }
                if (dirs == 3u) {
                    const uint32_t off = bin - base;
                    if (off < T) {
                        atomicAdd(tc + T + off, 1u);
                        atomicAdd(reinterpret_cast<unsigned long long *>(tb + T + off),
                                  (unsigned long long)Q.by[j]);
                    } else {
                        gadd(h, 1u, bin, 1u, Q.by[j]);
                    }
                }
            }
            if (pk != kNoKey) {
                const uint32_t pd = pk & 1u, off = (pk >> 1) - base;
                if (off < T) {
                    atomicAdd(tc + pd * T + off, pc);
                    atomicAdd(reinterpret_cast<unsigned long long *>(tb + pd * T + off),
                              (unsigned long long)ps);
                } else {
                    gadd(h, pd, pk >> 1, pc, ps);
                }
            }
        }
        if (!ta.full) {
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < 2 * T; i += blockDim.x) {
                const uint32_t c = tc[i];
                if (c) {
                    const uint32_t d = i >= T, off = i - d * T;
                    gadd(h, d, base + off, c, tb[i]);
                    tc[i] = 0;
                    tb[i] = 0;
                }
            }
            __syncthreads();
        }
    }
    if (ta.full) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < 2 * T; i += blockDim.x) {
            const uint32_t c = tc[i];
            if (c) {
                const uint32_t d = i >= T, off = i - d * T;
                gadd(h, d, off, c, tb[i]);
            }
        }
    }
    flush_counters(h.stats, cc, oor, true);
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
        SINET_DISC(LK_PML)
        SINET_DISC(LK_INTERVAL_GLOBAL)
#undef SINET_DISC
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t run_fused_atomic(int lk, bool agg, const RecArgs &r, const TableArgs &t,
                             const HistArgs &h, const LaunchCfg &c) {
    int grid = 0;
    cudaError_t e;
#define SINET_ATOM(L, A)                                                                        \
    if (lk == L && agg == A) {                                                                  \
        size_t smem = Classifier<L>::smem_bytes(t);                                             \
        if ((e = launch(k_fused_atomic<L, A>, smem, c, grid)) != cudaSuccess) return e;         \
        k_fused_atomic<L, A><<<grid, c.block, smem, c.stream>>>(r, t, h, c.status);             \
        return cudaGetLastError();                                                              \
    }
    SINET_ATOM(LK_INTERVAL, true)
    SINET_ATOM(LK_INTERVAL, false)
    SINET_ATOM(LK_PML, true)
    SINET_ATOM(LK_PML, false)
    SINET_ATOM(LK_INTERVAL_GLOBAL, true)
    SINET_ATOM(LK_INTERVAL_GLOBAL, false)
    SINET_ATOM(LK_CLASS_IN, true)
    SINET_ATOM(LK_CLASS_IN, false)
#undef SINET_ATOM
    return cudaErrorInvalidValue;
}

cudaError_t run_fused_tile(int lk, const RecArgs &r, const TableArgs &t, const HistArgs &h,
                           const TileArgs &ta, const LaunchCfg &c) {
    int grid = 0;
    cudaError_t e;
    switch (lk) {
#define SINET_TILE(L)                                                                           \
    case L: {                                                                                   \
        size_t smem = ((Classifier<L>::smem_bytes(t) + 15u) & ~15u) + 24ull * ta.tile_bins;     \
        if ((e = launch(k_fused_tile<L>, smem, c, grid)) != cudaSuccess) return e;              \
        k_fused_tile<L><<<grid, c.block, smem, c.stream>>>(r, t, h, ta, c.status);              \
        break;                                                                                  \
    }
        SINET_TILE(LK_INTERVAL)
        SINET_TILE(LK_PML)
        SINET_TILE(LK_INTERVAL_GLOBAL)
        SINET_TILE(LK_CLASS_IN)
#undef SINET_TILE
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sinet
