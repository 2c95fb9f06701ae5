// C ABI: argument validation, table upload, strategy dispatch, scratch.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "api_internal.h"
#include "owner.h"
#include "partition.h"

namespace sinet {

static std::mutex g_mu;
static DeviceState g_dev[64];
static thread_local int t_last_cuda = 0;

sinet_status cuda_fail(cudaError_t e) {
    t_last_cuda = (int)e;
    return e == cudaErrorMemoryAllocation ? SINET_ERR_OOM : SINET_ERR_CUDA;
}


sinet_status device_state(DeviceState **out) {
    int dev = 0;
    SINET_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SINET_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState &d = g_dev[dev];
    if (!d.ready) {
        int v = 0;
        SINET_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
        d.sm_count = v;
        SINET_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        d.smem_optin = (size_t)v;
        SINET_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        d.smem_per_sm = (size_t)v;
        SINET_CUDA(cudaMalloc(&d.status, 256));
        SINET_CUDA(cudaMemset(d.status, 0, 256));
        // keep stream-ordered scratch cached in the device's default pool
        // between calls instead of returning it at every synchronisation
        cudaMemPool_t pool = nullptr;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        d.ready = true;
    }
    *out = &d;
    return SINET_OK;
}

// Host side of the invariant-integer divider (Granlund & Montgomery 1994).
Divider make_divider(uint64_t w) {
    Divider d{};
    uint32_t l = 0;
    while (l < 64 && (((unsigned __int128)1) << l) < w) l++;
    const unsigned __int128 two64 = ((unsigned __int128)1) << 64;
    d.m = (uint64_t)((two64 * ((((unsigned __int128)1) << l) - w)) / w + 1);
    d.sh1 = l < 1 ? l : 1;
    d.sh2 = l >= 1 ? l - 1 : 0;
    return d;
}

// Quad geometry: pick the first record index (<= 0) at which every stream is
// 16-byte aligned (4-byte for byte streams), or fall back to scalar loads.
QuadGeom make_geom(uint64_t n, std::initializer_list<Stream> streams) {
    QuadGeom g{};
    g.n = n;
    g.shift = 0;
    g.vec = 0;
    for (int s = 0; s >= -3; --s) {
        bool ok = true;
        for (const Stream &st : streams) {
            if (!st.p) continue;
            const uint64_t a = (uint64_t)(uintptr_t)st.p + (uint64_t)((int64_t)s * (int64_t)st.esize);
            const uint64_t al = st.esize == 1 ? 4 : 16;
            if (a % al) ok = false;
        }
        if (ok) {
            g.shift = s;
            g.vec = 1;
            break;
        }
    }
    g.quads = n == 0 ? 0 : (n + (uint64_t)(-g.shift) + 3) / 4;
    return g;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

sinet_status check_params(const sinet_hist_params *p) {
    if (!p) return SINET_ERR_INVALID_ARG;
    if (p->bin_width_ms == 0 || p->n_bins == 0 || p->n_bins > 0x7FFFFFFFull) return SINET_ERR_INVALID_ARG;
    const unsigned __int128 end = (unsigned __int128)p->t0_ms + (unsigned __int128)p->n_bins * p->bin_width_ms;
    if (end > (unsigned __int128)UINT64_MAX) return SINET_ERR_INVALID_ARG;
    for (int c = 0; c < 4; ++c)
        if (p->policy[c] > 3) return SINET_ERR_INVALID_ARG;
    if (p->strategy < SINET_STRAT_AUTO || p->strategy > SINET_STRAT_PARTITION) return SINET_ERR_INVALID_ARG;
    if (p->lookup < SINET_LOOKUP_AUTO || p->lookup > SINET_LOOKUP_PML) return SINET_ERR_INVALID_ARG;
    if (p->block_threads && (p->block_threads > 1024 || p->block_threads % 32)) return SINET_ERR_INVALID_ARG;
    return SINET_OK;
}

sinet_status check_out(const sinet_hist_out *o) {
    if (!o || !o->count[0] || !o->count[1] || !o->bytes[0] || !o->bytes[1] || !o->stats)
        return SINET_ERR_INVALID_ARG;
    if (!aligned(o->count[0], 4) || !aligned(o->count[1], 4) || !aligned(o->bytes[0], 8) ||
        !aligned(o->bytes[1], 8) || !aligned(o->stats, 8))
        return SINET_ERR_INVALID_ARG;
    return SINET_OK;
}

HistArgs make_hist(const sinet_hist_params *p, const sinet_hist_out *o) {
    HistArgs h{};
    h.cnt[0] = o->count[0];
    h.cnt[1] = o->count[1];
    h.byt[0] = o->bytes[0];
    h.byt[1] = o->bytes[1];
    h.stats = o->stats;
    h.t0 = p->t0_ms;
    h.span = p->n_bins * p->bin_width_ms;
    h.div = make_divider(p->bin_width_ms);
    h.w_is_one = p->bin_width_ms == 1;
    h.policy = 0;
    h.two_dir = 0;
    for (int c = 0; c < 4; ++c) {
        h.policy |= (uint32_t)p->policy[c] << (8 * c);
        if (p->policy[c] == 3) h.two_dir = 1;
    }
    h.n_bins = (uint32_t)p->n_bins;
    return h;
}

sinet_status zero_outputs(const sinet_hist_params *p, const sinet_hist_out *o, cudaStream_t s) {
    if (p->accumulate) return SINET_OK;
    SINET_CUDA(cudaMemsetAsync(o->count[0], 0, 4 * p->n_bins, s));
    SINET_CUDA(cudaMemsetAsync(o->count[1], 0, 4 * p->n_bins, s));
    SINET_CUDA(cudaMemsetAsync(o->bytes[0], 0, 8 * p->n_bins, s));
    SINET_CUDA(cudaMemsetAsync(o->bytes[1], 0, 8 * p->n_bins, s));
    SINET_CUDA(cudaMemsetAsync(o->stats, 0, 64, s));
    return SINET_OK;
}

// Lookup form for a table: the staged interval form when it fits shared
// memory, the per-length form on request, else global-memory intervals.
int pick_lookup(const sinet_prefix_table *t, int32_t lookup, sinet_status *err) {
    *err = SINET_OK;
    if (lookup == SINET_LOOKUP_PML) {
        if (!t->img.pml_fits_smem) *err = SINET_ERR_UNSUPPORTED;
        return LK_PML;
    }
    if (!t->img.iv_fits_smem) return LK_INTERVAL_GLOBAL;
    return t->host.toggle_form == 1 ? LK_TOGGLE1 : t->host.toggle_form == 2 ? LK_TOGGLE2 : LK_INTERVAL;
}

static uint32_t table_smem(const sinet_prefix_table *t, int lk) {
    if (!t) return 0;
    if (lk == LK_INTERVAL || lk == LK_TOGGLE1 || lk == LK_TOGGLE2) return t->img.iv_bytes;
    if (lk == LK_PML) return t->img.pml_bytes;
    return 0;
}

// Histograms at least this large (24 bytes per bin) default to the cell
// scratch when the input is not time-sorted: well beyond L2, unsorted updates
// miss, and one sector per update instead of two halves the DRAM traffic.
static const uint64_t kCellMinHistBytes = 256ull << 20;

// Hot-key cache of the warp-aggregated atomic kernel: 2^9 sets x 4 ways
// (32 KB of shared memory per CTA).
static const uint32_t kCacheSetBits = 9;

// Bins per direction that fit a shared-memory tile (8 bytes per bin and
// direction) after the staged table and the kernel's static shared memory.
static uint32_t tile_capacity(const DeviceState *ds, uint32_t tsm) {
    const size_t reserve = 1024;
    const size_t used = ((tsm + 15u) & ~15u) + reserve;
    if (ds->smem_optin <= used) return 0;
    return (uint32_t)((ds->smem_optin - used) / 16) & ~3u;
}

// Tile bins that still let two CTAs share one SM's shared memory.
static uint32_t tile_capacity_pair(const DeviceState *ds, uint32_t tsm) {
    const size_t reserve = 2048;  // static shared memory and per-CTA reservation
    const size_t per_cta = ds->smem_per_sm / 2;
    const size_t used = ((tsm + 15u) & ~15u) + reserve;
    if (per_cta <= used) return 0;
    return (uint32_t)((per_cta - used) / 16) & ~3u;
}

// What AUTO runs without a measurement: the whole-histogram tile for small
// histograms, the chunk tile for time-sorted input, the cells for unsorted
// input over a histogram far beyond L2, warp combining otherwise.
// The cell strategy: zeroed cells, the combining kernel into them, then the
// expansion into the outputs.
static cudaError_t run_cells(int lk, const RecArgs &r, const TableArgs &ta_tab, HistArgs h,
                             const sinet_hist_params *p, const LaunchCfg &c, cudaStream_t s,
                             const TableArgs *watch = nullptr) {
    const size_t cell_bytes = 32 * (size_t)p->n_bins;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&h.cells), cell_bytes, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(h.cells, 0, cell_bytes, s);
    if (e == cudaSuccess) e = run_fused_atomic(lk, true, r, ta_tab, h, kCacheSetBits, c, watch);
    if (e == cudaSuccess) e = run_cells_expand(h, p->accumulate != 0, c);
    const cudaError_t e2 = cudaFreeAsync(h.cells, s);
    return e == cudaSuccess ? e2 : e;
}

static int auto_rule(const sinet_hist_params *p, const RecArgs &r, uint32_t cap, int lk, uint32_t tsm,
                     const HistArgs &h, const DeviceState *ds) {
    if (2ull * p->n_bins <= 8192 && p->n_bins <= cap) return SINET_STRAT_SMEM_FULL;
    // the tile strategy: measured faster than OWNER on the paper-shaped day
    // (about 4.6 records per ms bin, +-500 ms disorder)
    if (p->hints & SINET_HINT_TIME_SORTED) return SINET_STRAT_PRIV_TILE;
    // unsorted input over a histogram far beyond L2: the hot/cold partition
    // (measured 1.9x faster than the cells on the Zipf-skewed heavy day),
    // else the cells
    if (24 * p->n_bins >= kCellMinHistBytes && r.g.n >= p->n_bins / 4) {
        PartPlan probe{};
        if (plan_partition(lk, tsm, r, h, 0, ds->sm_count, ds->smem_optin, &probe) == cudaSuccess)
            return SINET_STRAT_PARTITION;
        return SINET_STRAT_ATOMIC_CELL;
    }
    return SINET_STRAT_GLOBAL_ATOMIC;
}

// Strategies a measured AUTO times for a call like this one.
static int auto_candidates(const sinet_hist_params *p, const RecArgs &r, uint32_t cap, int lk, uint32_t tsm,
                           const HistArgs &h, const DeviceState *ds, int out[4]) {
    int k = 0;
    if (2ull * p->n_bins <= 8192 && p->n_bins <= cap) {
        out[k++] = SINET_STRAT_SMEM_FULL;
        out[k++] = SINET_STRAT_GLOBAL_ATOMIC;
        return k;
    }
    if (p->hints & SINET_HINT_TIME_SORTED) {
        out[k++] = SINET_STRAT_PRIV_TILE;
        out[k++] = SINET_STRAT_OWNER;
    }
    out[k++] = SINET_STRAT_GLOBAL_ATOMIC;
    if (24 * p->n_bins >= kCellMinHistBytes) out[k++] = SINET_STRAT_ATOMIC_CELL;
    PartPlan probe{};
    if (k < 4 && !(p->hints & SINET_HINT_TIME_SORTED) &&
        plan_partition(lk, tsm, r, h, 0, ds->sm_count, ds->smem_optin, &probe) == cudaSuccess)
        out[k++] = SINET_STRAT_PARTITION;
    return k;
}

// Process-wide cache of measured AUTO choices, by device and input class.
static std::mutex g_auto_mu;
static std::map<std::string, int> g_auto;

static std::string auto_key(int dev, int lk, const sinet_hist_params *p, const RecArgs &r, const HistArgs &h) {
    auto lg = [](uint64_t v) {
        uint32_t l = 0;
        while (v > 1) {
            v >>= 1;
            ++l;
        }
        return l;
    };
    char b[128];
    std::snprintf(b, sizeof b, "d%d/lk%d/sorted%u/bins2^%u/n2^%u/w1%u/two%u", dev, lk,
                  (p->hints & SINET_HINT_TIME_SORTED) ? 1u : 0u, lg(p->n_bins), lg(r.g.n + 1), h.w_is_one,
                  h.two_dir);
    return b;
}

static sinet_status run_hist(const sinet_prefix_table *t, int lk, const RecArgs &r,
                             const sinet_hist_params *p, const sinet_hist_out *o, cudaStream_t s);

// Measured AUTO: time every candidate once on this call's own input (each
// overwrites the outputs in full), keep the fastest for the class. The
// caller then runs the winner, which leaves the outputs right.
static sinet_status measure_auto(const sinet_prefix_table *t, int lk, const RecArgs &r, const sinet_hist_params *p,
                                 const sinet_hist_out *o, cudaStream_t s, const int *cands, int nc, int *best) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SINET_CUDA(cudaEventCreate(&e0));
    SINET_CUDA(cudaEventCreate(&e1));
    float best_ms = 0.f;
    *best = -1;
    sinet_status st = SINET_OK;
    for (int i = 0; i < nc && st == SINET_OK; ++i) {
        sinet_hist_params pc = *p;
        pc.strategy = cands[i];
        pc.hints &= ~SINET_HINT_TUNE;
        cudaError_t e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            st = run_hist(t, lk, r, &pc, o, s);
            if (st == SINET_ERR_UNSUPPORTED) {  // not for this input: not a candidate
                st = SINET_OK;
                continue;
            }
        }
        if (e == cudaSuccess && st == SINET_OK) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess && st == SINET_OK) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess && st == SINET_OK) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) st = cuda_fail(e);
        if (st == SINET_OK && (*best < 0 || ms < best_ms)) {
            *best = cands[i];
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// The histogram step for every strategy (records already validated).
static sinet_status run_hist(const sinet_prefix_table *t, int lk, const RecArgs &r,
                             const sinet_hist_params *p, const sinet_hist_out *o, cudaStream_t s) {
    DeviceState *ds = nullptr;
    sinet_status st = device_state(&ds);
    if (st != SINET_OK) return st;
    HistArgs h = make_hist(p, o);
    h.status = ds->status;
    TableArgs ta_tab{};
    if (t) ta_tab = t->args;
    LaunchCfg c;
    c.block = p->block_threads ? (int)p->block_threads : 256;
    c.stream = s;
    c.status = ds->status;
    c.sm_count = ds->sm_count;
    const uint32_t tsm = table_smem(t, lk);
    const uint32_t cap = tile_capacity(ds, tsm);

    int strat = p->strategy;
    const TableArgs *watch = p->watch ? &p->watch->args : nullptr;
    if (watch && (lk == LK_PML || lk == LK_CLASS_IN)) return SINET_ERR_UNSUPPORTED;
    if (watch && strat != SINET_STRAT_AUTO && strat != SINET_STRAT_GLOBAL_ATOMIC &&
        strat != SINET_STRAT_ATOMIC_NOAGG && strat != SINET_STRAT_ATOMIC_CELL)
        return SINET_ERR_UNSUPPORTED;
    // a watch list keeps few records (a blocklist): the plain combining kernel
    if (strat == SINET_STRAT_AUTO && watch) strat = SINET_STRAT_GLOBAL_ATOMIC;
    if (strat == SINET_STRAT_AUTO) {
        strat = auto_rule(p, r, cap, lk, tsm, h, ds);
        int dev = 0;
        cudaGetDevice(&dev);
        const std::string key = auto_key(dev, lk, p, r, h);
        bool cached = false;
        {
            std::lock_guard<std::mutex> lk_(g_auto_mu);
            auto it = g_auto.find(key);
            if (it != g_auto.end()) {
                strat = it->second;
                cached = true;
            }
        }
        if (!cached && (p->hints & SINET_HINT_TUNE) && !p->accumulate && r.g.n > 0) {
            int cands[4];
            const int nc = auto_candidates(p, r, cap, lk, tsm, h, ds, cands);
            int best = -1;
            st = measure_auto(t, lk, r, p, o, s, cands, nc, &best);
            if (st != SINET_OK) return st;
            if (best >= 0) {
                strat = best;
                std::lock_guard<std::mutex> lk_(g_auto_mu);
                g_auto[key] = best;
            }
        }
    }

    // launch shapes first, so an unsupported combination fails before anything is enqueued
    TileArgs ta{};
    LaunchCfg ct = c;
    if (strat == SINET_STRAT_PRIV_TILE || strat == SINET_STRAT_SMEM_FULL) {
        ct.block = p->block_threads ? (int)p->block_threads : 512;
        if (strat == SINET_STRAT_SMEM_FULL) {
            ta.tile_bins = (uint32_t)((p->n_bins + 3) & ~3ull);  // whole histogram
            if (ta.tile_bins > cap) return SINET_ERR_UNSUPPORTED;
            ta.full = 1;
            ta.margin = 0;
            ta.iters = (uint32_t)(2048 / ct.block);
        } else {
            // default: as many bins as let two CTAs share an SM (at most
            // 4,096), and chunks of about three records per tile bin (fewer,
            // longer chunks amortise the per-chunk flush; much longer ones
            // span more bins than the tile holds where records are sparse)
            uint32_t T = p->tile_bins ? p->tile_bins : std::min<uint32_t>(4096, tile_capacity_pair(ds, tsm));
            if (T > cap) T = cap;
            T &= ~255u;
            if (T == 0) return SINET_ERR_UNSUPPORTED;
            ta.tile_bins = T;
            ta.full = 0;
            ta.margin = T / 6;
            ta.iters = (uint32_t)std::max<uint64_t>(1, (3ull * T) / (4ull * ct.block));
        }
        // a chunk stays within 65,535 records: a tile entry counts in 16 bits
        while ((uint64_t)ct.block * 4 * ta.iters > 65535 && ta.iters > 1) ta.iters--;
        if (ta.iters == 0) ta.iters = 1;
    }
    if (strat == SINET_STRAT_SORT_REDUCE && r.g.n * (h.two_dir ? 2ull : 1ull) >= 0xFFFFFFF0ull)
        return SINET_ERR_UNSUPPORTED;
    PartPlan pplan{};
    if (strat == SINET_STRAT_PARTITION) {
        if (watch) return SINET_ERR_UNSUPPORTED;
        uint32_t bb = 0;
        if (p->tile_bins) {
            if (p->tile_bins & (p->tile_bins - 1)) return SINET_ERR_INVALID_ARG;
            while ((1u << bb) < p->tile_bins) ++bb;
            if (bb > 20) return SINET_ERR_UNSUPPORTED;
        }
        if (plan_partition(lk, tsm, r, h, bb, ds->sm_count, ds->smem_optin, &pplan) != cudaSuccess)
            return SINET_ERR_UNSUPPORTED;
    }
    OwnerPlan oplan{};
    LaunchCfg co = c;
    if (strat == SINET_STRAT_OWNER) {
        // tile slots as for PRIV_TILE's tile (two CTAs of 512 threads per SM)
        co.block = p->block_threads ? (int)p->block_threads : 512;
        if (co.block > 512) return SINET_ERR_UNSUPPORTED;
        uint32_t S = p->tile_bins ? p->tile_bins : std::min<uint32_t>(4096, tile_capacity_pair(ds, tsm));
        if (S > cap) S = cap;
        if (S < 16) return SINET_ERR_UNSUPPORTED;
        oplan = plan_owner(r.g.n, h.n_bins, S, 0);
        int g = 0;
        const cudaError_t eg = owner_grid(lk, h.w_is_one != 0, ta_tab, oplan.slots, co, &g);
        if (eg != cudaSuccess) return cuda_fail(eg);
        oplan = plan_owner(r.g.n, h.n_bins, S, (uint32_t)g);
    }

    if ((strat == SINET_STRAT_ATOMIC_CELL || strat == SINET_STRAT_OWNER || strat == SINET_STRAT_PARTITION) &&
        !p->accumulate && r.g.n > 0) {
        // the expansion (cells), the owners or the cold pass write every bin;
        // only the counters start at zero
        cudaError_t ez = cudaMemsetAsync(o->stats, 0, 64, s);
        if (ez != cudaSuccess) return cuda_fail(ez);
    } else {
        st = zero_outputs(p, o, s);
        if (st != SINET_OK) return st;
    }
    if (r.g.n == 0) return SINET_OK;

    cudaError_t e = cudaSuccess;
    switch (strat) {
        case SINET_STRAT_GLOBAL_ATOMIC:
            e = run_fused_atomic(lk, true, r, ta_tab, h, kCacheSetBits, c, watch);
            break;
        case SINET_STRAT_ATOMIC_NOAGG:
            e = run_fused_atomic(lk, false, r, ta_tab, h, 0, c, watch);
            break;
        case SINET_STRAT_ATOMIC_CELL:
            e = run_cells(lk, r, ta_tab, h, p, c, s, watch);
            break;
        case SINET_STRAT_PRIV_TILE:
        case SINET_STRAT_SMEM_FULL:
            e = run_fused_tile(lk, r, ta_tab, h, ta, ct);
            break;
        case SINET_STRAT_OWNER: {
            void *scratch = nullptr;
            e = cudaMallocAsync(&scratch, oplan.scratch_bytes, s);
            if (e != cudaSuccess) return cuda_fail(e);
            const bool vec = aligned(o->count[0], 16) && aligned(o->count[1], 16) &&
                             aligned(o->bytes[0], 16) && aligned(o->bytes[1], 16);
            e = run_fused_owner(lk, r, ta_tab, h, p->bin_width_ms, oplan, scratch, p->accumulate != 0,
                                vec, co);
            const cudaError_t e2 = cudaFreeAsync(scratch, s);
            if (e == cudaSuccess) e = e2;
            break;
        }
        case SINET_STRAT_PARTITION: {
            void *scratch = nullptr;
            e = cudaMallocAsync(&scratch, pplan.scratch_bytes, s);
            if (e != cudaSuccess && p->strategy == SINET_STRAT_AUTO) {
                // AUTO's choice does not fit the free memory: the cells need
                // far less scratch and zero the same outputs (none)
                cudaGetLastError();
                e = run_cells(lk, r, ta_tab, h, p, c, s);
                break;
            }
            if (e != cudaSuccess) return cuda_fail(e);
            e = run_partition(lk, r, ta_tab, h, pplan, scratch, p->accumulate != 0, c);
            const cudaError_t e2 = cudaFreeAsync(scratch, s);
            if (e == cudaSuccess) e = e2;
            break;
        }
        case SINET_STRAT_SORT_REDUCE: {
            SortPlan plan = plan_sort_reduce(r.g.n, h.n_bins, h.two_dir);
            void *scratch = nullptr;
            e = cudaMallocAsync(&scratch, plan.scratch_bytes, s);
            if (e != cudaSuccess) return cuda_fail(e);
            e = run_sort_reduce(lk, r, ta_tab, h, plan, scratch, p->accumulate != 0, c);
            cudaError_t e2 = cudaFreeAsync(scratch, s);
            if (e == cudaSuccess) e = e2;
            break;
        }
        default:
            e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    return SINET_OK;
}

}  // namespace sinet

using namespace sinet;

extern "C" {

uint32_t sinet_version(void) { return 0x000100u; }

const char *sinet_status_string(sinet_status s) {
    switch (s) {
        case SINET_OK: return "ok";
        case SINET_ERR_INVALID_ARG: return "invalid argument";
        case SINET_ERR_CUDA: return "CUDA error";
        case SINET_ERR_OOM: return "out of device memory";
        case SINET_ERR_BUDGET: return "over memory budget";
        case SINET_ERR_TIMEOUT: return "device-side wait timed out";
        case SINET_ERR_TABLE_TOO_LARGE: return "prefix table too large";
        case SINET_ERR_DEVICE_CHECK: return "device-side check failed";
        case SINET_ERR_UNSUPPORTED: return "unsupported option combination";
    }
    return "unknown status";
}

int sinet_last_cuda_error(void) { return t_last_cuda; }

void sinet_default_params(sinet_hist_params *p, uint64_t t0_ms, uint64_t bin_width_ms, uint64_t n_bins) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->t0_ms = t0_ms;
    p->bin_width_ms = bin_width_ms;
    p->n_bins = n_bins;
    p->policy[0] = 0;
    p->policy[1] = SINET_DIR_OUT;
    p->policy[2] = SINET_DIR_IN;
    p->policy[3] = 0;
}

sinet_status sinet_parse_cidr(const char *text, uint32_t *net, uint8_t *len) {
    if (!text || !net || !len) return SINET_ERR_INVALID_ARG;
    uint32_t oct[4];
    const char *s = text;
    for (int i = 0; i < 4; ++i) {
        if (*s < '0' || *s > '9') return SINET_ERR_INVALID_ARG;
        uint32_t v = 0;
        int digits = 0;
        while (*s >= '0' && *s <= '9') {
            v = v * 10 + (uint32_t)(*s - '0');
            if (++digits > 3 || v > 255) return SINET_ERR_INVALID_ARG;
            ++s;
        }
        oct[i] = v;
        if (i < 3) {
            if (*s != '.') return SINET_ERR_INVALID_ARG;
            ++s;
        }
    }
    uint32_t z = 32;
    if (*s == '/') {
        ++s;
        if (*s < '0' || *s > '9') return SINET_ERR_INVALID_ARG;
        z = 0;
        int digits = 0;
        while (*s >= '0' && *s <= '9') {
            z = z * 10 + (uint32_t)(*s - '0');
            if (++digits > 2) return SINET_ERR_INVALID_ARG;
            ++s;
        }
        if (z > 32) return SINET_ERR_INVALID_ARG;
    }
    if (*s != '\0') return SINET_ERR_INVALID_ARG;
    *net = oct[0] << 24 | oct[1] << 16 | oct[2] << 8 | oct[3];
    *len = (uint8_t)z;
    return SINET_OK;
}

sinet_status sinet_build_prefix_table(const uint32_t *h_net, const uint8_t *h_len, uint32_t n,
                                      sinet_stream_t stream, sinet_prefix_table **out) {
    SINET_TRACE();
    if (!out) return SINET_ERR_INVALID_ARG;
    *out = nullptr;
    sinet_prefix_table *t = new (std::nothrow) sinet_prefix_table();
    if (!t) return SINET_ERR_OOM;
    int rc = compile_table(h_net, h_len, n, 0, t->host);
    if (rc != SINET_OK) {
        delete t;
        return (sinet_status)rc;
    }
    std::vector<uint8_t> buf = serialise(t->host, t->img);
    cudaError_t e = cudaGetDevice(&t->device);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_image, buf.size());
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->d_image, buf.data(), buf.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // host buffer goes out of scope
    if (e != cudaSuccess) {
        if (t->d_image) cudaFree(t->d_image);
        delete t;
        return cuda_fail(e);
    }
    TableArgs &a = t->args;
    a.image = t->d_image;
    a.iv_bytes = t->img.iv_bytes;
    a.off_blocks = t->img.off_blocks;
    a.off_desc = t->img.off_desc;
    a.desc_bits = t->host.desc_bits;
    a.toggle_form = t->host.toggle_form;
    a.off_lo = t->img.off_lo;
    a.off_hi = t->img.off_hi;
    a.off_idx32 = t->img.off_idx32;
    a.n_iv = (uint32_t)t->host.lo.size();
    a.index_bits = t->host.index_bits;
    a.off_nets = t->img.off_nets;
    a.off_groups = t->img.off_groups;
    a.pml_bytes = t->img.pml_bytes;
    a.n_groups = (uint32_t)t->host.groups.size();
    *out = t;
    return SINET_OK;
}

sinet_status sinet_destroy_prefix_table(sinet_prefix_table *t) {
    if (!t) return SINET_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaError_t e = cudaSuccess;
    if (cur != t->device) cudaSetDevice(t->device);
    e = cudaDeviceSynchronize();
    if (t->d_image) {
        cudaError_t e2 = cudaFree(t->d_image);
        if (e == cudaSuccess) e = e2;
    }
    if (cur != t->device) cudaSetDevice(cur);
    delete t;
    return e == cudaSuccess ? SINET_OK : cuda_fail(e);
}

sinet_status sinet_discriminate(const sinet_prefix_table *t, const uint32_t *d_src, const uint32_t *d_dst,
                                uint64_t n, uint8_t *d_class, uint64_t *d_class_counts, int32_t lookup,
                                sinet_stream_t stream) {
    SINET_TRACE();
    if (!t || !d_class_counts || !aligned(d_class_counts, 8)) return SINET_ERR_INVALID_ARG;
    if (n > kMaxN) return SINET_ERR_INVALID_ARG;
    if (n && (!d_src || !d_dst || !aligned(d_src, 4) || !aligned(d_dst, 4))) return SINET_ERR_INVALID_ARG;
    if (lookup < SINET_LOOKUP_AUTO || lookup > SINET_LOOKUP_PML) return SINET_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    sinet_status st = device_state(&ds);
    if (st != SINET_OK) return st;
    const int lk = pick_lookup(t, lookup, &st);
    if (st != SINET_OK) return st;
    SINET_CUDA(cudaMemsetAsync(d_class_counts, 0, 32, stream));
    if (n == 0) return SINET_OK;
    RecArgs r{};
    r.src = d_src;
    r.dst = d_dst;
    r.cls_out = d_class;
    r.g = make_geom(n, {{d_src, 4}, {d_dst, 4}, {d_class, 1}});
    LaunchCfg c;
    c.stream = stream;
    c.status = ds->status;
    c.sm_count = ds->sm_count;
    SINET_CUDA(run_discriminate(lk, r, t->args, d_class_counts, c));
    return SINET_OK;
}

sinet_status sinet_bin(const uint64_t *d_ts, uint64_t n, uint64_t t0_ms, uint64_t bin_width_ms, uint64_t n_bins,
                       uint32_t *d_bin, sinet_stream_t stream) {
    SINET_TRACE();
    sinet_hist_params p;
    sinet_default_params(&p, t0_ms, bin_width_ms, n_bins);
    sinet_status st = check_params(&p);
    if (st != SINET_OK) return st;
    if (n > kMaxN) return SINET_ERR_INVALID_ARG;
    if (n && (!d_ts || !d_bin || !aligned(d_ts, 8) || !aligned(d_bin, 4))) return SINET_ERR_INVALID_ARG;
    if (n == 0) return SINET_OK;
    DeviceState *ds = nullptr;
    if ((st = device_state(&ds)) != SINET_OK) return st;
    HistArgs h{};
    h.t0 = t0_ms;
    h.span = n_bins * bin_width_ms;
    h.div = make_divider(bin_width_ms);
    LaunchCfg c;
    c.stream = stream;
    c.sm_count = ds->sm_count;
    SINET_CUDA(run_bin(d_ts, n, h, d_bin, c));
    return SINET_OK;
}

sinet_status sinet_histogram(const uint64_t *d_ts, const uint32_t *d_bytes, const uint8_t *d_class, uint64_t n,
                             const sinet_hist_params *p, const sinet_hist_out *o, sinet_stream_t stream) {
    SINET_TRACE();
    sinet_status st = check_params(p);
    if (st != SINET_OK) return st;
    if ((st = check_out(o)) != SINET_OK) return st;
    if (n > kMaxN) return SINET_ERR_INVALID_ARG;
    if (n && (!d_ts || !d_bytes || !d_class || !aligned(d_ts, 8) || !aligned(d_bytes, 4)))
        return SINET_ERR_INVALID_ARG;
    if (p->watch) return SINET_ERR_UNSUPPORTED;  // the class input has no addresses to test
    RecArgs r{};
    r.ts = d_ts;
    r.bytes = d_bytes;
    r.cls_in = d_class;
    r.g = make_geom(n, {{d_ts, 8}, {d_bytes, 4}, {d_class, 1}});
    return run_hist(nullptr, LK_CLASS_IN, r, p, o, stream);
}

sinet_status sinet_discriminate_histogram(const sinet_prefix_table *t, const uint64_t *d_ts, const uint32_t *d_src,
                                          const uint32_t *d_dst, const uint32_t *d_bytes, uint64_t n,
                                          const sinet_hist_params *p, const sinet_hist_out *o,
                                          sinet_stream_t stream) {
    SINET_TRACE();
    if (!t) return SINET_ERR_INVALID_ARG;
    sinet_status st = check_params(p);
    if (st != SINET_OK) return st;
    if ((st = check_out(o)) != SINET_OK) return st;
    if (n > kMaxN) return SINET_ERR_INVALID_ARG;
    if (n && (!d_ts || !d_src || !d_dst || !d_bytes || !aligned(d_ts, 8) || !aligned(d_src, 4) ||
              !aligned(d_dst, 4) || !aligned(d_bytes, 4)))
        return SINET_ERR_INVALID_ARG;
    const int lk = pick_lookup(t, p->lookup, &st);
    if (st != SINET_OK) return st;
    RecArgs r{};
    r.ts = d_ts;
    r.src = d_src;
    r.dst = d_dst;
    r.bytes = d_bytes;
    r.g = make_geom(n, {{d_ts, 8}, {d_src, 4}, {d_dst, 4}, {d_bytes, 4}});
    return run_hist(t, lk, r, p, o, stream);
}

sinet_status sinet_auto_strategy(const sinet_prefix_table *t, uint64_t n, const sinet_hist_params *p,
                                 int32_t *strategy) {
    if (!t || !strategy) return SINET_ERR_INVALID_ARG;
    sinet_status st = check_params(p);
    if (st != SINET_OK) return st;
    if (n > kMaxN) return SINET_ERR_INVALID_ARG;
    const int lk = pick_lookup(t, p->lookup, &st);
    if (st != SINET_OK) return st;
    DeviceState *ds = nullptr;
    if ((st = device_state(&ds)) != SINET_OK) return st;
    if (p->strategy != SINET_STRAT_AUTO) {
        *strategy = p->strategy;
        return SINET_OK;
    }
    if (p->watch) {
        *strategy = SINET_STRAT_GLOBAL_ATOMIC;
        return SINET_OK;
    }
    RecArgs r{};
    r.g.n = n;
    sinet_hist_out o{};
    HistArgs h = make_hist(p, &o);
    const uint32_t tsm = table_smem(t, lk);
    *strategy = auto_rule(p, r, tile_capacity(ds, tsm), lk, tsm, h, ds);
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk_(g_auto_mu);
    auto it = g_auto.find(auto_key(dev, lk, p, r, h));
    if (it != g_auto.end()) *strategy = it->second;
    return SINET_OK;
}

sinet_status sinet_device_status(sinet_stream_t stream, uint32_t *device_code) {
    if (!device_code) return SINET_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    sinet_status st = device_state(&ds);
    if (st != SINET_OK) return st;
    SINET_CUDA(cudaStreamSynchronize(stream));
    uint32_t v = 0;
    SINET_CUDA(cudaMemcpy(&v, ds->status, 4, cudaMemcpyDeviceToHost));
    SINET_CUDA(cudaMemset(ds->status, 0, 4));
    *device_code = v;
    return SINET_OK;
}

}  // extern "C"
