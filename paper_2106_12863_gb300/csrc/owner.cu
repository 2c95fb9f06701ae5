// OWNER strategy: fused discriminate + histogram for time-sorted input that
// writes every histogram bin exactly once with plain stores.
//
// Chunks of records are taken in ticket order. Each chunk accumulates its
// records in a shared-memory bin tile (as PRIV_TILE does), then learns
// F_prev = 1 + the largest bin any earlier chunk touched (a decoupled
// look-back over per-chunk maxima) and owns the bins [F_prev, F_this), where
// F_this also covers its own records (the last chunk owns up to n_bins). It
// writes its territory with plain stores (empty bins as zeros) and flags it
// done; bins below F_prev that it also touched belong to earlier chunks, so
// it waits for those owners' done flags and adds them with atomics. Records
// outside the tile are re-read and added with atomics at the end. Every bin
// is thus stored once before any atomic reaches it: no separate zeroing and
// no read of the histogram. Correct for any order; fast when each chunk's
// records sit in a narrow time range. All waits are bounded.
#include "launch.h"

namespace sinet {
namespace {

constexpr uint64_t kWordAgg = 1ull << 62;
constexpr uint64_t kWordIncl = 2ull << 62;

__device__ __forceinline__ uint64_t ld_acq64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel64(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acq32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Warp 0: publish this chunk's bound and return the largest bound of all
// earlier chunks (0 if none). Bounds are "largest bin touched + 1".
__device__ uint32_t look_back_max(uint64_t *words, uint64_t ch, uint32_t own, uint32_t *status) {
    const uint32_t lane = threadIdx.x & 31;
    if (lane == 0) st_rel64(words + ch, kWordAgg | own);
    uint32_t acc = 0;
    int64_t p = (int64_t)ch - 1;
    bool ok = true;
    while (p >= 0) {
        const int64_t idx = p - (int64_t)lane;
        uint64_t w = idx >= 0 ? ld_acq64(words + idx) : kWordIncl;
        uint32_t it = 0;
        while (__any_sync(kFull, (w >> 62) == 0)) {
            if (++it >= kSpinLimit) {
                ok = false;
                break;
            }
            if ((w >> 62) == 0) w = ld_acq64(words + idx);
        }
        if (!ok) break;
        const uint32_t incl = __ballot_sync(kFull, (w >> 62) == 2);
        const int first = incl ? __ffs(incl) - 1 : 31;
        const uint32_t v = (int)lane <= first ? (uint32_t)w : 0u;
        acc = max(acc, __reduce_max_sync(kFull, v));
        if (incl) break;
        p -= 32;
    }
    if (!ok && lane == 0) latch_status(status, SINET_ERR_TIMEOUT);
    return acc;
}

template <int LK, bool W1>
__global__ void __launch_bounds__(512, 2) k_fused_owner(RecArgs r, TableArgs t, HistArgs h, OwnerArgs oa,
                                                        uint32_t *status) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ uint64_t s_ch;
    __shared__ uint32_t s_base, s_bmin, s_bmax, s_ovf, s_f0, s_f1;
    __shared__ unsigned long long s_cnt[6];
    Classifier<LK> C;
    C.init(t, smem, &bar, status);
    const uint32_t T = oa.tile_bins;
    uint32_t *tlo = reinterpret_cast<uint32_t *>(smem + ((Classifier<LK>::smem_bytes(t) + 15u) & ~15u));
    uint32_t *thi = tlo + 2 * T;
    for (uint32_t i = threadIdx.x; i < 2 * T; i += blockDim.x) {
        tlo[i] = 0;
        thi[i] = 0;
    }
    if (threadIdx.x < 6) s_cnt[threadIdx.x] = 0;
    const uint64_t pol = policy_evict_first();
    uint64_t ccp = 0;
    uint32_t oorp = 0;
    const uint64_t qpc = (uint64_t)blockDim.x * oa.iters;
    const uint64_t n_chunks = (r.g.quads + qpc - 1) / qpc;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_ch = atomicAdd(reinterpret_cast<unsigned long long *>(oa.ticket), 1ull);
            s_bmin = 0xFFFFFFFFu;
            s_bmax = 0;
            s_ovf = 0;
        }
        __syncthreads();
        const uint64_t ch = s_ch;
        if (ch >= n_chunks) break;

        // --- pass A: the chunk into the tile -------------------------------
        uint32_t base = 0, bmin = 0xFFFFFFFFu, bmax = 0, ovf = 0;
        auto pass_a = [&](const Quad &Q) {
            uint32_t bins[4];
            const uint32_t inr = bin_quad<W1>(h, Q, bins);
            Quad Qc = Q;
            classify_quad<LK>(C, Qc);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!(Qc.valid >> j & 1u)) continue;
                bump_class_packed(ccp, Qc.cls[j]);
                const uint32_t dirs = dirs_of_packed(h, Qc.cls[j], inr >> j & 1u, oorp);
                if (!dirs) continue;
                const uint32_t bin = bins[j];
                bmin = min(bmin, bin);
                bmax = max(bmax, bin);
                const uint32_t off = bin - base;
                if (off < T) {
                    const uint32_t e = (dirs & 1u) ? off : T + off;
                    smem_add_wide(tlo + e, thi + e, Qc.by[j], 1u << 16);
                    if (dirs == 3u) smem_add_wide(tlo + T + off, thi + T + off, Qc.by[j], 1u << 16);
                } else {
                    ovf = 1;
                }
            }
        };
        {
            Quad Q;
            load_quad<true, LK != LK_CLASS_IN, true, LK == LK_CLASS_IN>(r, ch * qpc + threadIdx.x, pol, Q);
            if (threadIdx.x == 0) {
                // the chunk's first record is this thread's first valid one
                const int j0 = Q.valid ? __ffs(Q.valid) - 1 : 0;
                uint32_t b = 0;
                const uint64_t rel = Q.ts[j0] - h.t0;
                if (Q.valid && rel < h.span) {
                    b = W1 ? (uint32_t)rel : (uint32_t)divide(rel, h.div);
                    b = b > oa.margin ? b - oa.margin : 0u;
                }
                s_base = b;
            }
            __syncthreads();
            base = s_base;
            pass_a(Q);
        }
        for (uint32_t it = 1; it < oa.iters; ++it) {
            Quad Q;
            load_quad<true, LK != LK_CLASS_IN, true, LK == LK_CLASS_IN>(
                r, ch * qpc + (uint64_t)it * blockDim.x + threadIdx.x, pol, Q);
            pass_a(Q);
        }
        drain_packed(ccp, oorp, s_cnt);
        bmin = __reduce_min_sync(kFull, bmin);
        bmax = __reduce_max_sync(kFull, bmax);
        ovf = __reduce_or_sync(kFull, ovf);
        if (lane == 0) {
            if (bmin <= bmax) {
                atomicMin(&s_bmin, bmin);
                atomicMax(&s_bmax, bmax);
            }
            if (ovf) s_ovf = 1;
        }
        __syncthreads();
        const uint32_t cmin = s_bmin, cmax = s_bmax;
        const bool any = cmin <= cmax;

        // --- territory ------------------------------------------------------
        if (warp == 0) {
            const uint32_t own = any ? cmax + 1 : 0u;
            const uint32_t prev = look_back_max(oa.words, ch, own, status);
            const uint32_t f1 = max(prev, own);
            if (lane == 0) {
                st_rel64(oa.words + ch, kWordIncl | f1);
                s_f0 = prev;
                s_f1 = (ch + 1 == n_chunks && !oa.accumulate) ? h.n_bins : f1;
            }
        }
        __syncthreads();
        const uint32_t f0 = s_f0, f1 = s_f1;
        // own bins: one plain store each (read-add-write when accumulating)
        for (uint32_t b = f0 + threadIdx.x; b < f1; b += blockDim.x) {
            const uint32_t off = b - base;
#pragma unroll
            for (uint32_t d = 0; d < 2; ++d) {
                uint32_t cnt = 0;
                uint64_t by = 0;
                if (off < T) {
                    const uint32_t vh = thi[d * T + off];
                    if (vh) {
                        cnt = vh >> 16;
                        by = (uint64_t)(vh & 0xFFFFu) << 32 | tlo[d * T + off];
                        thi[d * T + off] = 0;
                        tlo[d * T + off] = 0;
                    }
                }
                uint32_t *cp = d ? h.cnt[1] : h.cnt[0];
                uint64_t *bp = d ? h.byt[1] : h.byt[0];
                if (!oa.accumulate) {
                    cp[b] = cnt;
                    bp[b] = by;
                } else if (cnt) {
                    cp[b] += cnt;
                    bp[b] += by;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_rel32(oa.done + ch, 1u);
        }

        // --- bins owned by earlier chunks ------------------------------------
        if (any && cmin < f0) {
            if (threadIdx.x == 0) {
                // wait for every owner of [cmin, f0): chunks ch-1, ch-2, ...
                bool ok = true;
                for (int64_t c = (int64_t)ch - 1; c >= 0 && ok; --c) {
                    uint32_t it = 0;
                    while (ld_acq32(oa.done + c) == 0u)
                        if (++it >= kSpinLimit) { ok = false; break; }
                    if (!ok || c == 0) break;
                    uint64_t w;
                    it = 0;
                    while (((w = ld_acq64(oa.words + c - 1)) >> 62) != 2)
                        if (++it >= kSpinLimit) { ok = false; break; }
                    if ((uint32_t)w <= cmin) break;  // chunk c's territory starts at or below cmin
                }
                if (!ok) latch_status(status, SINET_ERR_TIMEOUT);
                __threadfence();
            }
            __syncthreads();
            const uint32_t lo = max(cmin, base);
            const uint32_t hi = min(f0, base + T);  // exclusive
            for (uint32_t b = lo + threadIdx.x; b < hi; b += blockDim.x) {
                const uint32_t off = b - base;
#pragma unroll
                for (uint32_t d = 0; d < 2; ++d) {
                    const uint32_t vh = thi[d * T + off];
                    if (vh) {
                        gadd(h, d, b, vh >> 16, (uint64_t)(vh & 0xFFFFu) << 32 | tlo[d * T + off]);
                        thi[d * T + off] = 0;
                        tlo[d * T + off] = 0;
                    }
                }
            }
        }

        // --- records outside the tile: re-read, add with atomics --------------
        if (s_ovf) {
            __syncthreads();
            for (uint32_t it = 0; it < oa.iters; ++it) {
                Quad Q;
                load_quad<true, LK != LK_CLASS_IN, true, LK == LK_CLASS_IN>(
                    r, ch * qpc + (uint64_t)it * blockDim.x + threadIdx.x, pol, Q);
                uint32_t bins[4];
                const uint32_t inr = bin_quad<W1>(h, Q, bins);
                classify_quad<LK>(C, Q);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (!(Q.valid >> j & 1u) || !(inr >> j & 1u)) continue;
                    const uint32_t dirs = (h.policy >> (8 * Q.cls[j])) & 3u;
                    if (!dirs || bins[j] - base < T) continue;
                    gadd(h, (dirs & 1u) ? 0u : 1u, bins[j], 1u, Q.by[j]);
                    if (dirs == 3u) gadd(h, 1u, bins[j], 1u, Q.by[j]);
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 6 && s_cnt[threadIdx.x])
        atomicAdd(reinterpret_cast<unsigned long long *>(h.stats) + threadIdx.x, s_cnt[threadIdx.x]);
}

}  // namespace

cudaError_t run_fused_owner(int lk, const RecArgs &r, const TableArgs &t, const HistArgs &h,
                            const OwnerArgs &oa, const LaunchCfg &c) {
    const bool w1 = h.w_is_one != 0;
    cudaError_t e;
#define SINET_OWNER(L, W)                                                                          \
    if (lk == L && w1 == W) {                                                                      \
        const size_t smem = ((Classifier<L>::smem_bytes(t) + 15u) & ~15u) + 16ull * oa.tile_bins;  \
        e = cudaFuncSetAttribute(k_fused_owner<L, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)smem);                                                       \
        if (e != cudaSuccess) return e;                                                            \
        int per_sm = 0;                                                                            \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_owner<L, W>, c.block, smem); \
        if (e != cudaSuccess) return e;                                                            \
        if (per_sm < 1) return cudaErrorInvalidConfiguration;                                      \
        k_fused_owner<L, W><<<per_sm * c.sm_count, c.block, smem, c.stream>>>(r, t, h, oa, c.status); \
        return cudaGetLastError();                                                                 \
    }
    SINET_OWNER(LK_INTERVAL, true)
    SINET_OWNER(LK_INTERVAL, false)
    SINET_OWNER(LK_PML, true)
    SINET_OWNER(LK_PML, false)
    SINET_OWNER(LK_INTERVAL_GLOBAL, true)
    SINET_OWNER(LK_INTERVAL_GLOBAL, false)
    SINET_OWNER(LK_CLASS_IN, true)
    SINET_OWNER(LK_CLASS_IN, false)
#undef SINET_OWNER
    return cudaErrorInvalidValue;
}

}  // namespace sinet
