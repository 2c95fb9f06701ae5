// Owner-computes discriminate + histogram for time-sorted records (sm_103a).
//
// Section 5 bins sessions by millisecond; with records sorted by timestamp,
// the records that fall into a run of bins are themselves one run. Each CTA
// owns a contiguous block of bin ranges and walks it in order: it classifies
// (Algorithm 1) and bins each range's run into a circular shared-memory tile,
// then stores the bins that are final with plain coalesced stores, including
// the empty ones. The DRAM traffic is the algorithmic one: the records read
// once and every bin written once.
#include <algorithm>

#include "owner.h"

namespace sinet {

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// ---------------------------------------------------------------------------
// Run boundaries: bounds[k] = first record with ts >= t0 + k * T * w for
// 0 < k < n_ranges (binary search over the sorted timestamps), bounds[0] = 0,
// bounds[n_ranges] = n. Records before the window fall into range 0 and
// records past it into the last range (both count as out of window there).
__global__ void __launch_bounds__(256) k_owner_bounds(const uint64_t *ts, uint64_t n, uint64_t t0,
                                                      uint64_t range_ms, uint32_t n_ranges,
                                                      uint64_t *bounds, uint32_t *n_items) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k <= n_ranges; k += stride) {
        uint64_t pos;
        if (k == 0) {
            pos = 0;
            *n_items = 0;
        } else if (k == n_ranges) {
            pos = n;
        } else {
            // k * range_ms < n_bins * w, and t0 + n_bins * w fits in 64 bits
            const uint64_t key = t0 + (uint64_t)k * range_ms;
            uint64_t lo = 0, hi = n;
            while (lo < hi) {
                const uint64_t mid = lo + ((hi - lo) >> 1);
                if (__ldg(ts + mid) < key)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            pos = lo;
        }
        bounds[k] = pos;
    }
}

// In-place prefix maximum over bounds[0..n_ranges] (on unsorted input the
// searched boundaries need not be monotone; the maximum turns them into a
// partition of [0, n) all the same), then the CTA blocks: with the work
// W(k) = bounds[k] + min(k T, n_bins) before range k and N = W(n_ranges),
// part[c] is the first range with W(k) >= floor(c N / G), and part[G] =
// n_ranges. One CTA of 1024 threads; each thread takes a contiguous segment.
__global__ void __launch_bounds__(1024) k_owner_scan(uint64_t *bounds, uint32_t n_ranges, uint32_t T,
                                                     uint32_t n_bins, uint32_t G, uint32_t *part) {
    __shared__ uint64_t s_warp[32];
    const uint32_t count = n_ranges + 1;
    const uint32_t seg = (count + blockDim.x - 1) / blockDim.x;
    const uint32_t i0 = min(count, threadIdx.x * seg), i1 = min(count, i0 + seg);
    uint64_t m = 0;
    for (uint32_t i = i0; i < i1; ++i) m = max(m, bounds[i]);
    // inclusive max-scan over the threads' maxima: within a warp, then over warps
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = m;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t o = __shfl_up_sync(kFull, inc, d);
        if (lane >= (uint32_t)d) inc = max(inc, o);
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t nw = blockDim.x >> 5;
        uint64_t w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t o = __shfl_up_sync(kFull, w, d);
            if (lane >= (uint32_t)d) w = max(w, o);
        }
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    // exclusive prefix of this thread = max over the threads before it
    uint64_t run = __shfl_up_sync(kFull, inc, 1);
    if (lane == 0) run = 0;
    if (warp > 0) run = max(run, s_warp[warp - 1]);

    // N = n + n_bins (bounds[n_ranges] = n is already the maximum, and no
    // thread rewrites it with a different value); c <= chi(W) exactly when
    // floor(c N / G) <= W
    const uint64_t N = bounds[n_ranges] + n_bins;
    auto chi = [&](uint64_t W) { return ((W + 1) * G - 1) / N; };
    for (uint32_t i = i0; i < i1; ++i) {
        const uint64_t prev = run;
        run = max(run, bounds[i]);
        bounds[i] = run;
        const uint64_t W = run + umin64((uint64_t)i * T, n_bins);
        const uint64_t c_from = i == 0 ? 0 : chi(prev + umin64((uint64_t)(i - 1) * T, n_bins)) + 1;
        const uint64_t c_to = umin64(chi(W), (uint64_t)G - 1);
        for (uint64_t c = c_from; c <= c_to; ++c) part[c] = i;
    }
    if (threadIdx.x == 0) part[G] = n_ranges;
}

// ---------------------------------------------------------------------------
// Shared state of the owner and remainder kernels.
struct OwnerArgs {
    const uint64_t *bounds;
    const uint32_t *part;
    OwnerItem *items;
    uint32_t *n_items;
    uint64_t cap_items;
    uint32_t n_ranges;
    uint32_t S;  // tile slots per direction (power of two)
    uint32_t T;  // bins per range
    uint32_t H;  // halo bins on either side of a range
    uint32_t accumulate;
    uint32_t vec;  // output arrays 16-byte aligned
};

// What a pass over records does (owner_records).
enum : int {
    PASS_OWNER = 0,   // count classes and out-of-window records, tile the window's bins, flag strays
    PASS_FULL = 1,    // the same, with strays added by global reductions
    PASS_STRAYS = 2,  // only the strays, by global reductions (the rest was counted and tiled)
};

// A run of records [ra, rb) as quads: quads [qa, qa + nq), the first one
// masked by `first` and the last by `last` (bit j: record j is in the run).
struct QuadRun {
    uint64_t qa;
    uint32_t nq;
    uint32_t masks;  // first | last << 4
};

__device__ __forceinline__ QuadRun quad_run(const QuadGeom &g, uint64_t ra, uint64_t rb) {
    QuadRun q{0, 0, 0};
    if (ra >= rb) return q;
    const uint64_t a = ra + (uint64_t)(-(int64_t)g.shift), b = rb + (uint64_t)(-(int64_t)g.shift);
    q.qa = a >> 2;
    q.nq = (uint32_t)(((b + 3) >> 2) - q.qa);
    const uint32_t first = (0xFu << (a & 3)) & 0xFu;
    const uint32_t last = (b & 3) ? (1u << (b & 3)) - 1u : 0xFu;
    q.masks = first | last << 4;
    return q;
}

// Records of a run against the tile window [wlo, wlo + wlen) (slot = bin mod
// S, direction 1 at slot + S); returns 1 if PASS_OWNER saw a stray.
template <int LK, bool W1, int MODE>
__device__ __forceinline__ uint32_t owner_records(const RecArgs &r, const Classifier<LK> &C,
                                                  const HistArgs &h, const QuadRun run, uint32_t wlo,
                                                  uint32_t wlen, uint32_t S, uint32_t *tlo,
                                                  uint32_t *thi, uint64_t pol, uint64_t &ccp,
                                                  uint32_t &oorp) {
    constexpr bool kCount = MODE != PASS_STRAYS;
    uint32_t stray = 0;
    for (uint32_t dq = threadIdx.x; dq < run.nq; dq += blockDim.x) {
        Quad Q;
        load_quad<true, LK != LK_CLASS_IN, true, LK == LK_CLASS_IN>(r, run.qa + dq, pol, Q);
        if (dq == 0) Q.valid &= run.masks & 0xFu;
        if (dq == run.nq - 1) Q.valid &= run.masks >> 4;
        uint32_t bins[4];
        const uint32_t inr = bin_quad<W1>(h, Q, bins);
        classify_quad<LK>(C, Q);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!(Q.valid >> j & 1u)) continue;
            uint32_t dirs;
            if (kCount) {
                bump_class_packed(ccp, Q.cls[j]);
                dirs = dirs_of_packed(h, Q.cls[j], inr >> j & 1u, oorp);
            } else {
                dirs = (inr >> j & 1u) ? (h.policy >> (8 * Q.cls[j])) & 3u : 0u;
            }
            if (!dirs) continue;
            const uint32_t b = bins[j];
            if (b - wlo < wlen) {
                if (MODE == PASS_STRAYS) continue;  // tiled by the owner
                const uint32_t s = b & (S - 1);
                const uint32_t e = (dirs & 1u) ? s : S + s;
                smem_add_wide(tlo + e, thi + e, Q.by[j], 1u << 16);
                if (dirs == 3u) smem_add_wide(tlo + S + s, thi + S + s, Q.by[j], 1u << 16);
            } else if (MODE == PASS_OWNER) {
                stray = 1;
            } else {
                gadd(h, (dirs & 1u) ? 0u : 1u, b, 1u, Q.by[j]);
                if (dirs == 3u) gadd(h, 1u, b, 1u, Q.by[j]);
            }
        }
    }
    return stray;
}

// Tile entry e as (count, byte sum); the entry is cleared.
__device__ __forceinline__ void take_entry(uint32_t *tlo, uint32_t *thi, uint32_t e, uint32_t &c,
                                           uint64_t &s) {
    const uint32_t lo = tlo[e], hi = thi[e];
    tlo[e] = 0;
    thi[e] = 0;
    c = hi >> 16;
    s = (uint64_t)(hi & 0xFFFFu) << 32 | lo;
}

// The owner's store of bins [slo, shi) of both directions from the tile
// (plain stores; with `accumulate`, added to what the arrays hold); the slots
// are cleared. slo is a multiple of 4; each thread takes 4 consecutive bins,
// with vector accesses when the arrays are 16-byte aligned.
__device__ __forceinline__ void owner_store(const HistArgs &h, const OwnerArgs &oa, uint32_t slo,
                                            uint32_t shi, uint32_t *tlo, uint32_t *thi) {
    const uint32_t S = oa.S;
    const uint32_t nb = shi - slo;
    const uint32_t ng = (nb + 3) >> 2;  // groups of 4 bins per direction
    for (uint32_t i = threadIdx.x; i < 2 * ng; i += blockDim.x) {
        const uint32_t d = i >= ng;
        const uint32_t off = 4 * (i - d * ng);
        const uint32_t b = slo + off;
        const uint32_t e = d * S + (b & (S - 1));  // 4 slots in a row: b is a multiple of 4
        uint32_t *cp = (d ? h.cnt[1] : h.cnt[0]) + b;
        uint64_t *bp = (d ? h.byt[1] : h.byt[0]) + b;
        if (oa.vec && off + 4 <= nb) {
            const uint4 lo = *reinterpret_cast<const uint4 *>(tlo + e);
            const uint4 hi = *reinterpret_cast<const uint4 *>(thi + e);
            *reinterpret_cast<uint4 *>(tlo + e) = make_uint4(0, 0, 0, 0);
            *reinterpret_cast<uint4 *>(thi + e) = make_uint4(0, 0, 0, 0);
            uint4 c = make_uint4(hi.x >> 16, hi.y >> 16, hi.z >> 16, hi.w >> 16);
            if (oa.accumulate) {
                const uint4 oc = *reinterpret_cast<const uint4 *>(cp);
                c.x += oc.x; c.y += oc.y; c.z += oc.z; c.w += oc.w;
            }
            *reinterpret_cast<uint4 *>(cp) = c;
            ulonglong2 s01 = make_ulonglong2((uint64_t)(hi.x & 0xFFFFu) << 32 | lo.x,
                                             (uint64_t)(hi.y & 0xFFFFu) << 32 | lo.y);
            if (oa.accumulate) {
                const ulonglong2 o = *reinterpret_cast<const ulonglong2 *>(bp);
                s01.x += o.x; s01.y += o.y;
            }
            *reinterpret_cast<ulonglong2 *>(bp) = s01;
            ulonglong2 s23 = make_ulonglong2((uint64_t)(hi.z & 0xFFFFu) << 32 | lo.z,
                                             (uint64_t)(hi.w & 0xFFFFu) << 32 | lo.w);
            if (oa.accumulate) {
                const ulonglong2 o = *reinterpret_cast<const ulonglong2 *>(bp + 2);
                s23.x += o.x; s23.y += o.y;
            }
            *reinterpret_cast<ulonglong2 *>(bp + 2) = s23;
        } else {
            for (uint32_t j = 0; j < 4 && off + j < nb; ++j) {
                uint32_t c;
                uint64_t s;
                take_entry(tlo, thi, e + j, c, s);
                if (!oa.accumulate) {
                    cp[j] = c;
                    bp[j] = s;
                } else if (c) {
                    cp[j] += c;
                    bp[j] += s;
                }
            }
        }
    }
}

// Owner kernel (REM = false): CTA c walks ranges [part[c], part[c + 1]).
// For range k (bins [b0, b1)) the tile window is [max(lo, b0 - H),
// min(hi, b1 + H)) with [lo, hi) the bins of the CTA's block; after the run,
// the bins below b1 - H are final (no later run of the block reaches them)
// and are stored, the last range of the block storing up to hi.
// Remainder kernel (REM = true): the items the owners queued, added with
// global reductions after every owner has stored its bins.
template <int LK, bool W1, bool REM>
__global__ void __launch_bounds__(512, 2) k_fused_owner(RecArgs r, TableArgs t, HistArgs h, OwnerArgs oa,
                                                        uint32_t *status) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ unsigned long long s_cnt[6];
    __shared__ uint32_t s_item, s_m;
    __shared__ uint64_t s_run[2][2];  // owner: run bounds by range parity
    __shared__ OwnerItem s_it;        // remainder: the current item
    uint32_t k0 = 0, k1 = 0;          // owner: this CTA's ranges; remainder: the items
    if (REM) {
        k1 = (uint32_t)umin64(*oa.n_items, oa.cap_items);
        k0 = blockIdx.x;
    } else {
        k0 = oa.part[blockIdx.x];
        k1 = oa.part[blockIdx.x + 1];
    }
    if (k0 >= k1) return;  // for sorted input the remainder kernel usually ends here
    Classifier<LK> C;
    if (!C.init(t, smem, &bar, status)) return;  // table not staged: the status word says so
    const uint32_t S = oa.S;
    uint32_t *tlo = reinterpret_cast<uint32_t *>(smem + ((Classifier<LK>::smem_bytes(t) + 15u) & ~15u));
    uint32_t *thi = tlo + 2 * S;
    for (uint32_t i = threadIdx.x; i < 2 * S; i += blockDim.x) {
        tlo[i] = 0;
        thi[i] = 0;
    }
    if (threadIdx.x < 6) s_cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        if (REM) {
            s_it = oa.items[k0];
        } else {
            s_run[0][0] = oa.bounds[k0];
            s_run[0][1] = oa.bounds[k0 + 1];
        }
    }
    __syncthreads();
    const uint64_t pol = policy_evict_first();
    uint64_t ccp = 0;
    uint32_t oorp = 0;

    if (!REM) {
        const uint32_t T = oa.T, H = oa.H;
        const uint32_t lo = k0 * T;
        const uint32_t hi = (uint32_t)umin64((uint64_t)k1 * T, h.n_bins);
        uint32_t par = 0;
        for (uint32_t k = k0; k < k1; ++k) {
            const uint32_t b0 = k * T;
            const uint32_t b1 = (uint32_t)umin64((uint64_t)b0 + T, h.n_bins);
            const uint32_t wlo = max(lo, b0 >= H ? b0 - H : 0u);
            const uint32_t whi = (uint32_t)umin64(hi, (uint64_t)b1 + H);
            uint32_t stray;
            {
                // the run's bounds are read from shared memory where they are
                // needed, not kept in registers across the record loop
                const uint64_t ra = s_run[par][0];
                const uint64_t rb = umin64(s_run[par][1], ra + kOwnerCap);
                stray = owner_records<LK, W1, PASS_OWNER>(r, C, h, quad_run(r.g, ra, rb), wlo, whi - wlo, S,
                                                          tlo, thi, pol, ccp, oorp);
            }
            drain_packed(ccp, oorp, s_cnt);
            const int any_stray = __syncthreads_or(stray);
            uint64_t nra = 0, nrb = 0;
            if (threadIdx.x == 0 && k + 1 < k1) {
                nra = oa.bounds[k + 1];
                nrb = oa.bounds[k + 2];
            }
            owner_store(h, oa, wlo, k + 1 < k1 ? b1 - H : hi, tlo, thi);
            const uint64_t ra = s_run[par][0], rb_run = s_run[par][1];
            const uint64_t rb = umin64(rb_run, ra + kOwnerCap);
            if (threadIdx.x == 0) {
                // the buffer of the other parity was last read before the barrier above
                s_run[par ^ 1][0] = nra;
                s_run[par ^ 1][1] = nrb;
                // queue a second look at this run (strays first) and the rest of the run
                const uint64_t m = (any_stray ? 1u : 0u) + (rb_run - rb + kOwnerCap - 1) / kOwnerCap;
                uint32_t first = 0, fit = 0;
                if (m) {
                    // the list holds every item by construction (plan_owner)
                    first = atomicAdd(oa.n_items, (uint32_t)m);
                    fit = first < oa.cap_items ? (uint32_t)umin64(m, oa.cap_items - first) : 0u;
                    if (fit < m) latch_status(status, SINET_ERR_DEVICE_CHECK);
                }
                s_item = first;
                s_m = fit;
            }
            __syncthreads();
            par ^= 1u;
            const uint32_t first = s_item, m = s_m;
            const uint32_t s0 = any_stray ? 1u : 0u;
            for (uint32_t j = threadIdx.x; j < m; j += blockDim.x) {
                OwnerItem it;
                it.k = k;
                if (j < s0) {
                    it.x = ra;
                    it.y = rb;
                    it.mode = OWN_STRAYS;
                    it.wlo = wlo;
                    it.wlen = whi - wlo;
                } else {
                    it.x = rb + (uint64_t)(j - s0) * kOwnerCap;
                    it.y = umin64(rb_run, it.x + kOwnerCap);
                    it.mode = OWN_FULL;
                    it.wlo = b0;
                    it.wlen = b1 - b0;
                }
                oa.items[first + j] = it;
            }
        }
    } else {
        for (uint32_t w = k0; w < k1; w += gridDim.x) {
            const OwnerItem it = s_it;
            __syncthreads();  // every thread has read the item
            if (threadIdx.x == 0 && w + gridDim.x < k1) s_it = oa.items[w + gridDim.x];
            const bool ok = it.k < oa.n_ranges && it.x <= it.y && it.y <= r.g.n && it.wlen <= oa.S &&
                            (uint64_t)it.wlo + it.wlen <= h.n_bins;
            if (ok) {
                const QuadRun run = quad_run(r.g, it.x, it.y);
                if (it.mode == OWN_STRAYS) {
                    owner_records<LK, W1, PASS_STRAYS>(r, C, h, run, it.wlo, it.wlen, S, tlo, thi, pol, ccp,
                                                       oorp);
                } else {
                    owner_records<LK, W1, PASS_FULL>(r, C, h, run, it.wlo, it.wlen, S, tlo, thi, pol, ccp,
                                                     oorp);
                    drain_packed(ccp, oorp, s_cnt);
                    __syncthreads();
                    for (uint32_t i = threadIdx.x; i < 2 * it.wlen; i += blockDim.x) {
                        const uint32_t d = i >= it.wlen;
                        const uint32_t b = it.wlo + i - d * it.wlen;
                        const uint32_t e = d * S + (b & (S - 1));
                        if (thi[e] | tlo[e]) {
                            uint32_t c;
                            uint64_t sum;
                            take_entry(tlo, thi, e, c, sum);
                            gadd(h, d, b, c, sum);
                        }
                    }
                }
            } else if (threadIdx.x == 0) {
                latch_status(status, SINET_ERR_DEVICE_CHECK);  // a queued item out of range cannot occur
            }
            __syncthreads();  // the next item is in place, the tile is clear
        }
    }
    __syncthreads();
    if (threadIdx.x < 6 && s_cnt[threadIdx.x])
        atomicAdd(reinterpret_cast<unsigned long long *>(h.stats) + threadIdx.x, s_cnt[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// Host side.

OwnerPlan plan_owner(uint64_t n, uint32_t n_bins, uint32_t slots, uint32_t grid) {
    OwnerPlan p{};
    uint32_t S = 16;
    while (S * 2 <= slots) S *= 2;
    p.slots = S;
    p.range_bins = S / 2;
    p.halo_bins = S / 4;
    p.n_ranges = (uint32_t)(((uint64_t)n_bins + p.range_bins - 1) / p.range_bins);
    p.grid = grid;
    // at most one stray item per range, and the overflow items of a run of L
    // records number ceil(L / cap) - 1 <= L / cap, n / cap in all
    p.cap_items = (uint64_t)p.n_ranges + n / kOwnerCap + 1;
    size_t off = 0;
    p.off_bounds = off;
    off += ((size_t)p.n_ranges + 1) * sizeof(uint64_t);
    off = (off + 255) & ~(size_t)255;
    p.off_part = off;
    off += ((size_t)grid + 1) * sizeof(uint32_t);
    off = (off + 255) & ~(size_t)255;
    p.off_items = off;
    off += (size_t)p.cap_items * sizeof(OwnerItem);
    off = (off + 255) & ~(size_t)255;
    p.off_count = off;
    off += 256;
    p.scratch_bytes = off;
    return p;
}

template <typename K>
static cudaError_t kernel_grid(K kernel, size_t smem, const LaunchCfg &c, int &grid) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, c.block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    grid = c.grid > 0 ? c.grid : per_sm * c.sm_count;
    return cudaSuccess;
}

template <int LK>
static size_t owner_smem(const TableArgs &t, uint32_t S) {
    return ((Classifier<LK>::smem_bytes(t) + 15u) & ~15u) + 16ull * S;
}

template <int LK, bool W1>
static cudaError_t launch_owner_pair(const RecArgs &r, const TableArgs &t, const HistArgs &h,
                                     const OwnerArgs &oa, uint32_t grid, const LaunchCfg &c) {
    const size_t smem = owner_smem<LK>(t, oa.S);
    int g = 0;
    cudaError_t e = kernel_grid(k_fused_owner<LK, W1, false>, smem, c, g);
    if (e != cudaSuccess) return e;
    k_fused_owner<LK, W1, false><<<grid, c.block, smem, c.stream>>>(r, t, h, oa, c.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = kernel_grid(k_fused_owner<LK, W1, true>, smem, c, g);
    if (e != cudaSuccess) return e;
    k_fused_owner<LK, W1, true><<<g, c.block, smem, c.stream>>>(r, t, h, oa, c.status);
    return cudaGetLastError();
}

#define SINET_OWN_FORMS(X)        \
    X(LK_INTERVAL, true)          \
    X(LK_INTERVAL, false)         \
    X(LK_TOGGLE1, true)           \
    X(LK_TOGGLE1, false)          \
    X(LK_TOGGLE2, true)           \
    X(LK_TOGGLE2, false)          \
    X(LK_PML, true)               \
    X(LK_PML, false)              \
    X(LK_INTERVAL_GLOBAL, true)   \
    X(LK_INTERVAL_GLOBAL, false)  \
    X(LK_CLASS_IN, true)          \
    X(LK_CLASS_IN, false)

cudaError_t owner_grid(int lk, bool w1, const TableArgs &t, uint32_t slots, const LaunchCfg &c, int *grid) {
#define SINET_OWN_GRID(L, W) \
    if (lk == L && w1 == W) return kernel_grid(k_fused_owner<L, W, false>, owner_smem<L>(t, slots), c, *grid);
    SINET_OWN_FORMS(SINET_OWN_GRID)
#undef SINET_OWN_GRID
    return cudaErrorInvalidValue;
}

cudaError_t run_fused_owner(int lk, const RecArgs &r, const TableArgs &t, const HistArgs &h,
                            uint64_t bin_width, const OwnerPlan &plan, void *scratch,
                            bool accumulate, bool vec_ok, const LaunchCfg &c) {
    if (c.block <= 0 || c.block > 512 || c.block % 32 || plan.grid == 0) return cudaErrorInvalidConfiguration;
    uint8_t *s = static_cast<uint8_t *>(scratch);
    uint64_t *bounds = reinterpret_cast<uint64_t *>(s + plan.off_bounds);
    uint32_t *part = reinterpret_cast<uint32_t *>(s + plan.off_part);
    OwnerArgs oa{};
    oa.bounds = bounds;
    oa.part = part;
    oa.items = reinterpret_cast<OwnerItem *>(s + plan.off_items);
    oa.n_items = reinterpret_cast<uint32_t *>(s + plan.off_count);
    oa.cap_items = plan.cap_items;
    oa.n_ranges = plan.n_ranges;
    oa.S = plan.slots;
    oa.T = plan.range_bins;
    oa.H = plan.halo_bins;
    oa.accumulate = accumulate ? 1u : 0u;
    oa.vec = vec_ok ? 1u : 0u;

    const uint32_t count = plan.n_ranges + 1;
    const int bgrid = (int)std::min<uint32_t>((count + 255) / 256, 8u * (uint32_t)c.sm_count);
    k_owner_bounds<<<bgrid, 256, 0, c.stream>>>(r.ts, r.g.n, h.t0, (uint64_t)plan.range_bins * bin_width,
                                                 plan.n_ranges, bounds, oa.n_items);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_owner_scan<<<1, 1024, 0, c.stream>>>(bounds, plan.n_ranges, plan.range_bins, h.n_bins, plan.grid,
                                           part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    const bool w1 = h.w_is_one != 0;
#define SINET_OWN_RUN(L, W) \
    if (lk == L && w1 == W) return launch_owner_pair<L, W>(r, t, h, oa, plan.grid, c);
    SINET_OWN_FORMS(SINET_OWN_RUN)
#undef SINET_OWN_RUN
    return cudaErrorInvalidValue;
}

#undef SINET_OWN_FORMS

}  // namespace sinet
