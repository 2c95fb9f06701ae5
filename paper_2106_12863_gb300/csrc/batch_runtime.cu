// Batched launch runtime: slice planning, the strategy autotuner and its
// cache, the device engine (descriptors + CUDA graph), and the batch C ABI.
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

#include "batch_internal.h"

namespace sinet {

uint32_t batch_smem(const DeviceState *ds) {
    // two CTAs per SM; 1 KB per CTA is reserved by the hardware, and the
    // kernel's static shared memory (descriptor copy, slice starts, counters)
    // stays below 5 KB
    const size_t per_cta = ds->smem_per_sm / 2;
    size_t v = per_cta > 6144 ? per_cta - 6144 : 0;
    v = std::min(v, ds->smem_optin);
    return (uint32_t)(v & ~(size_t)15);
}

uint32_t batch_grid(const DeviceState *ds) { return 2u * (uint32_t)ds->sm_count; }

uint32_t batch_scheme(int32_t strategy) {
    switch (strategy) {
        case SINET_STRAT_SMEM_FULL: return BS_TILE;
        case SINET_STRAT_ATOMIC_NOAGG:
        case SINET_STRAT_SORT_REDUCE: return BS_NOAGG;  // the plain path takes no work items
        default: return BS_AGG;
    }
}

bool sort_feasible(const PlannedSlice &ps) {
    return ps.d.r.g.n * (ps.d.h.two_dir ? 2ull : 1ull) < 0xFFFFFFF0ull;
}

static uint32_t round16(uint32_t v) { return (v + 15u) & ~15u; }

uint32_t item_quads_for(uint64_t quads, uint32_t scheme, uint32_t grid) {
    if (scheme == BS_TILE || grid == 0) return kItemQuads;
    const uint64_t q = (quads + grid - 1) / grid;
    return (uint32_t)std::min<uint64_t>(kItemQuads, std::max<uint64_t>(kMinItemQuads, q));
}

void set_strategy(PlannedSlice &ps, int32_t strategy, uint32_t grid) {
    ps.strategy = strategy;
    ps.d.strat = batch_scheme(strategy);
    ps.d.item_quads = item_quads_for(ps.d.r.g.quads, ps.d.strat, grid);
    ps.items = strategy == SINET_STRAT_SORT_REDUCE
                   ? 0u
                   : (uint32_t)((ps.d.r.g.quads + ps.d.item_quads - 1) / ps.d.item_quads);
}

sinet_status check_slice(const sinet_batch_slice &u) {
    if (!u.table) return SINET_ERR_INVALID_ARG;
    sinet_status st = check_params(&u.params);
    if (st != SINET_OK) return st;
    if ((st = check_out(&u.out)) != SINET_OK) return st;
    if (u.n > kMaxN) return SINET_ERR_INVALID_ARG;
    if (u.n && (!u.ts || !u.src || !u.dst || !u.bytes || !aligned(u.ts, 8) || !aligned(u.src, 4) ||
                !aligned(u.dst, 4) || !aligned(u.bytes, 4)))
        return SINET_ERR_INVALID_ARG;
    const int32_t s = u.params.strategy;
    if (s != SINET_STRAT_AUTO && s != SINET_STRAT_GLOBAL_ATOMIC && s != SINET_STRAT_ATOMIC_NOAGG &&
        s != SINET_STRAT_SMEM_FULL && s != SINET_STRAT_SORT_REDUCE)
        return SINET_ERR_UNSUPPORTED;
    if (u.params.lookup == SINET_LOOKUP_PML || u.params.watch) return SINET_ERR_UNSUPPORTED;
    return SINET_OK;
}

sinet_status plan_slice(const sinet_batch_slice &u, const DeviceState *ds, uint32_t smem, PlannedSlice &ps) {
    const sinet_prefix_table *t = u.table;
    BatchSlice &d = ps.d;
    std::memset(&d, 0, sizeof d);
    d.r.ts = u.ts;
    d.r.src = u.src;
    d.r.dst = u.dst;
    d.r.bytes = u.bytes;
    d.r.g = make_geom(u.n, {{u.ts, 8}, {u.src, 4}, {u.dst, 4}, {u.bytes, 4}});
    d.t = t->args;
    d.h = make_hist(&u.params, &u.out);
    d.h.status = ds->status;
    // the toggle form is staged when it leaves room for the hot-key cache
    uint32_t staged = 0;
    if (t->img.iv_fits_smem && round16(t->img.iv_bytes) + kBatchCacheBytes <= smem) {
        staged = round16(t->img.iv_bytes);
        d.lk = t->host.toggle_form == 1 ? LK_TOGGLE1 : t->host.toggle_form == 2 ? LK_TOGGLE2 : LK_INTERVAL;
    } else {
        d.lk = LK_INTERVAL_GLOBAL;
    }
    const uint64_t T = (u.params.n_bins + 3) & ~3ull;
    d.tile_bins = (uint32_t)std::min<uint64_t>(T, 0xFFFFFFFFull);
    ps.tile_fits = staged + 16 * T <= smem;
    d.zero = u.params.accumulate ? 0u : 1u;
    d.ready = u.ready;
    d.ready_value = u.ready_value;
    if (u.params.strategy == SINET_STRAT_SMEM_FULL && !ps.tile_fits) return SINET_ERR_UNSUPPORTED;
    if (u.params.strategy == SINET_STRAT_SORT_REDUCE && !sort_feasible(ps)) return SINET_ERR_UNSUPPORTED;
    set_strategy(ps, u.params.strategy, batch_grid(ds));  // AUTO: resolved later
    ps.zero_items = d.zero ? (uint32_t)((u.params.n_bins + kZeroBins - 1) / kZeroBins) : 0u;
    return SINET_OK;
}

// ---------------------------------------------------------------------------
// Engine.

sinet_status BatchEngine::init(uint32_t capacity, const DeviceState *ds, uint32_t smem_bytes) {
    SINET_CUDA(cudaGetDevice(&device));
    cap = capacity;
    smem = smem_bytes;
    int per_sm = 0;
    SINET_CUDA(batch_occupancy(smem, &per_sm));
    if (per_sm < 1) return SINET_ERR_UNSUPPORTED;
    grid = per_sm * ds->sm_count;
    zgrid = 4 * ds->sm_count;
    sm_count = ds->sm_count;
    off_item = sizeof(BatchHeader);
    off_zero = off_item + 4 * ((size_t)cap + 1);
    off_slices = (off_zero + 4 * ((size_t)cap + 1) + 15) & ~(size_t)15;
    bytes = off_slices + sizeof(BatchSlice) * (size_t)cap;
    SINET_CUDA(cudaMalloc(&d_mem, bytes));
    SINET_CUDA(cudaMemset(d_mem, 0, bytes));
    uint8_t *m = static_cast<uint8_t *>(d_mem);
    args.hdr = reinterpret_cast<BatchHeader *>(m);
    args.item_start = reinterpret_cast<const uint32_t *>(m + off_item);
    args.zero_start = reinterpret_cast<const uint32_t *>(m + off_zero);
    args.slices = reinterpret_cast<const BatchSlice *>(m + off_slices);
    return SINET_OK;
}

void BatchEngine::image(const std::vector<PlannedSlice> &v, std::vector<uint8_t> &buf) const {
    const uint32_t n = (uint32_t)v.size();
    buf.assign(off_slices + sizeof(BatchSlice) * (size_t)n, 0);
    BatchHeader hdr{};
    uint32_t *item = reinterpret_cast<uint32_t *>(buf.data() + off_item);
    uint32_t *zero = reinterpret_cast<uint32_t *>(buf.data() + off_zero);
    uint64_t ti = 0, tz = 0;
    for (uint32_t i = 0; i < n; ++i) {
        item[i] = (uint32_t)ti;
        zero[i] = (uint32_t)tz;
        ti += v[i].items;
        tz += v[i].zero_items;
        std::memcpy(buf.data() + off_slices + sizeof(BatchSlice) * i, &v[i].d, sizeof(BatchSlice));
    }
    item[n] = (uint32_t)ti;
    zero[n] = (uint32_t)tz;
    hdr.n_slices = n;
    hdr.wait_ns = wait_ns;
    hdr.total_items = (uint32_t)ti;
    hdr.total_zero = (uint32_t)tz;
    std::memcpy(buf.data(), &hdr, sizeof hdr);
}

sinet_status BatchEngine::plan_sorts(const std::vector<PlannedSlice> &v, const DeviceState *ds) {
    (void)ds;
    for (const PlannedSlice &ps : v) {
        if (ps.strategy != SINET_STRAT_SORT_REDUCE) continue;
        SortJob j;
        j.r = ps.d.r;
        j.t = ps.d.t;
        j.h = ps.d.h;
        j.lk = (int)ps.d.lk;
        j.plan = plan_sort_reduce(ps.d.r.g.n, ps.d.h.n_bins, ps.d.h.two_dir != 0);
        SINET_CUDA(cudaMalloc(&j.scratch, std::max<size_t>(j.plan.scratch_bytes, 256)));
        sorts.push_back(j);
    }
    return SINET_OK;
}

sinet_status BatchEngine::capture(uint32_t *status) {
    cudaStream_t cs = nullptr;
    SINET_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = run_batch_zero(args, zgrid, cs);
        cudaError_t e2 = e1 == cudaSuccess ? run_batch(args, smem, grid, cs, status) : e1;
        // slices on the plain path: their outputs were zeroed (or are
        // accumulated into) like every other slice's, so the chain adds
        LaunchCfg lc;
        lc.stream = cs;
        lc.status = status;
        for (const SortJob &j : sorts) {
            if (e2 != cudaSuccess) break;
            lc.sm_count = sm_count;
            e2 = run_sort_reduce(j.lk, j.r, j.t, j.h, j.plan, j.scratch, true, lc);
        }
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    cudaStreamDestroy(cs);
    return e == cudaSuccess ? SINET_OK : cuda_fail(e);
}

sinet_status BatchEngine::launch(cudaStream_t s) const {
    SINET_CUDA(cudaGraphLaunch(exec, s));
    return SINET_OK;
}

void BatchEngine::release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (d_mem) cudaFree(d_mem);
    for (SortJob &j : sorts)
        if (j.scratch) cudaFree(j.scratch);
    sorts.clear();
    exec = nullptr;
    graph = nullptr;
    d_mem = nullptr;
}

// ---------------------------------------------------------------------------
// Autotuner. A class groups slices whose best strategy should agree; its
// representative (largest slice) is timed with every candidate.

namespace {

std::mutex g_tune_mu;
bool g_tune_loaded = false;
std::map<std::string, int32_t> g_tune;

const char *strategy_name(int32_t s) {
    switch (s) {
        case SINET_STRAT_GLOBAL_ATOMIC: return "global_atomic";
        case SINET_STRAT_ATOMIC_NOAGG: return "atomic_noagg";
        case SINET_STRAT_SMEM_FULL: return "smem_full";
        case SINET_STRAT_SORT_REDUCE: return "sort_reduce";
    }
    return "auto";
}

int32_t strategy_from_name(const char *s) {
    if (!std::strcmp(s, "global_atomic")) return SINET_STRAT_GLOBAL_ATOMIC;
    if (!std::strcmp(s, "atomic_noagg")) return SINET_STRAT_ATOMIC_NOAGG;
    if (!std::strcmp(s, "smem_full")) return SINET_STRAT_SMEM_FULL;
    if (!std::strcmp(s, "sort_reduce")) return SINET_STRAT_SORT_REDUCE;
    return -1;
}

uint32_t ceil_log2(uint64_t v) {
    uint32_t l = 0;
    while (l < 64 && (1ull << l) < v) ++l;
    return l;
}

uint32_t floor_log2(uint64_t v) {
    uint32_t l = 0;
    while (v > 1) {
        v >>= 1;
        ++l;
    }
    return l;
}

std::string class_key(const PlannedSlice &ps, const DeviceState *ds) {
    char b[160];
    std::snprintf(b, sizeof b, "sm%d/lk%u/tile%d/bins2^%u/n2^%u/w1%u/two%u", ds->sm_count, ps.d.lk,
                  ps.tile_fits ? 1 : 0, ceil_log2(ps.d.h.n_bins), floor_log2(ps.d.r.g.n + 1),
                  ps.d.h.w_is_one, ps.d.h.two_dir);
    return b;
}

void load_cache_file() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("SINET_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char key[200], name[40];
    while (std::fscanf(f, "%199s %39s%*[^\n]", key, name) == 2) {
        const int32_t s = strategy_from_name(name);
        if (s >= 0) g_tune[key] = s;
    }
    std::fclose(f);
}

void append_cache_file(const std::string &key, int32_t s, float ns_per_record) {
    const char *path = std::getenv("SINET_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %s %.4f\n", key.c_str(), strategy_name(s), ns_per_record);
    std::fclose(f);
}

// The rule for a class nobody has tuned: the tile when the histogram fits
// and the slice has a few records per bin, warp combining when the
// histogram is small enough to stay in L2, plain atomics otherwise.
int32_t fixed_rule(const PlannedSlice &ps) {
    const uint64_t n = ps.d.r.g.n, bins = ps.d.h.n_bins;
    if (ps.tile_fits && n >= 4 * bins) return SINET_STRAT_SMEM_FULL;
    if (24 * bins <= (64ull << 20)) return SINET_STRAT_GLOBAL_ATOMIC;
    return SINET_STRAT_ATOMIC_NOAGG;
}

// Time the candidates on one representative slice; returns the fastest per
// record. A batch keeps every CTA busy, so each candidate runs on enough
// copies of the slice (its first kTuneRecords records) to give the grid two
// work items per CTA: timed alone, a slice cut into few large items would
// leave most of the GPU idle and look slower than it is inside a batch. The
// copies write separate scratch outputs when those stay small, else share one.
sinet_status tune_one(const PlannedSlice &rep, const DeviceState *ds, uint32_t smem, cudaStream_t s,
                      BatchEngine &eng, int32_t *best, float *best_ns) {
    PlannedSlice ps = rep;
    const uint64_t n = std::min<uint64_t>(rep.d.r.g.n, kTuneRecords);
    ps.d.r.g = make_geom(n, {{ps.d.r.ts, 8}, {ps.d.r.src, 4}, {ps.d.r.dst, 4}, {ps.d.r.bytes, 4}});
    const uint32_t nb = ps.d.h.n_bins;
    const size_t out_bytes = (((size_t)8 * nb + 15) & ~(size_t)15) + (size_t)16 * nb + 64;
    ps.d.zero = 1;
    ps.zero_items = (nb + kZeroBins - 1) / kZeroBins;
    int32_t cands[3] = {SINET_STRAT_GLOBAL_ATOMIC, SINET_STRAT_ATOMIC_NOAGG, SINET_STRAT_SMEM_FULL};
    const int nc = ps.tile_fits ? 3 : 2;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SINET_CUDA(cudaEventCreate(&e0));
    SINET_CUDA(cudaEventCreate(&e1));
    *best = -1;
    *best_ns = 0.f;
    std::vector<uint8_t> buf;
    sinet_status st = SINET_OK;
    for (int c = 0; c < nc && st == SINET_OK; ++c) {
        set_strategy(ps, cands[c], (uint32_t)eng.grid);
        uint32_t copies = ps.items ? (uint32_t)((2ull * eng.grid + ps.items - 1) / ps.items) : 1u;
        copies = std::max<uint32_t>(1, std::min<uint32_t>({copies, eng.cap,
                                                           (uint32_t)std::max<uint64_t>(1, (4 * kTuneRecords) / std::max<uint64_t>(n, 1))}));
        const bool separate = (size_t)copies * out_bytes <= (512ull << 20);
        void *scratch = nullptr;
        cudaError_t e = cudaMalloc(&scratch, separate ? copies * out_bytes : out_bytes);
        std::vector<PlannedSlice> v(copies, ps);
        for (uint32_t k = 0; k < copies && e == cudaSuccess; ++k) {
            uint8_t *m = static_cast<uint8_t *>(scratch) + (separate ? k * out_bytes : 0);
            HistArgs &h = v[k].d.h;
            h.cnt[0] = reinterpret_cast<uint32_t *>(m);
            h.cnt[1] = h.cnt[0] + nb;
            h.byt[0] = reinterpret_cast<uint64_t *>(m + (((size_t)8 * nb + 15) & ~(size_t)15));
            h.byt[1] = h.byt[0] + nb;
            h.stats = h.byt[1] + nb;
            if (!separate && k) v[k].zero_items = 0;  // zeroed once
        }
        if (e == cudaSuccess) {
            eng.image(v, buf);
            e = cudaMemcpyAsync(eng.d_mem, buf.data(), buf.size(), cudaMemcpyHostToDevice, s);
        }
        float ms = 1e30f;
        for (int rep_i = 0; rep_i < 4 && e == cudaSuccess; ++rep_i) {
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = run_batch_zero(eng.args, eng.zgrid, s);
            if (e == cudaSuccess) e = run_batch(eng.args, smem, eng.grid, s, ds->status);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess && rep_i > 0) ms = std::min(ms, t);  // the first run warms up
        }
        if (scratch) {
            const cudaError_t e2 = cudaFree(scratch);
            if (e == cudaSuccess) e = e2;
        }
        if (e != cudaSuccess) {
            st = cuda_fail(e);
            break;
        }
        const float ns = ms * 1e6f / (float)((double)copies * (double)std::max<uint64_t>(n, 1));
        if (*best < 0 || ns < *best_ns) {
            *best = cands[c];
            *best_ns = ns;
        }
    }
    // the plain path: its own chain of kernels over the slice's first n
    // records into scratch outputs, timed the same way (best of three after a
    // warm-up run)
    if (st == SINET_OK && sort_feasible(ps)) {
        const SortPlan plan = plan_sort_reduce(n, nb, ps.d.h.two_dir != 0);
        void *scratch = nullptr, *outs = nullptr;
        cudaError_t e = cudaMalloc(&scratch, std::max<size_t>(plan.scratch_bytes, 256));
        if (e == cudaSuccess) e = cudaMalloc(&outs, out_bytes);
        HistArgs h = ps.d.h;
        if (e == cudaSuccess) {
            uint8_t *m = static_cast<uint8_t *>(outs);
            h.cnt[0] = reinterpret_cast<uint32_t *>(m);
            h.cnt[1] = h.cnt[0] + nb;
            h.byt[0] = reinterpret_cast<uint64_t *>(m + (((size_t)8 * nb + 15) & ~(size_t)15));
            h.byt[1] = h.byt[0] + nb;
            h.stats = h.byt[1] + nb;
        }
        LaunchCfg lc;
        lc.stream = s;
        lc.status = ds->status;
        lc.sm_count = ds->sm_count;
        float ms = 1e30f;
        for (int rep_i = 0; rep_i < 4 && e == cudaSuccess; ++rep_i) {
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(outs, 0, out_bytes, s);
            if (e == cudaSuccess) e = run_sort_reduce((int)ps.d.lk, ps.d.r, ps.d.t, h, plan, scratch, true, lc);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess && rep_i > 0) ms = std::min(ms, t);
        }
        if (scratch) cudaFree(scratch);
        if (outs) cudaFree(outs);
        if (e != cudaSuccess) {
            st = cuda_fail(e);
        } else {
            const float ns = ms * 1e6f / (float)std::max<uint64_t>(n, 1);
            if (*best < 0 || ns < *best_ns) {
                *best = SINET_STRAT_SORT_REDUCE;
                *best_ns = ns;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // namespace

sinet_status resolve_strategies(std::vector<PlannedSlice> &v, bool tune, const DeviceState *ds,
                                uint32_t smem, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_cache_file();
    // classes of the AUTO slices and their largest member
    std::map<std::string, size_t> rep;
    std::vector<std::string> keys(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        if (v[i].strategy != SINET_STRAT_AUTO) continue;
        keys[i] = class_key(v[i], ds);
        auto it = rep.find(keys[i]);
        if (it == rep.end() || v[i].d.r.g.n > v[it->second].d.r.g.n) rep[keys[i]] = i;
    }
    if (tune) {
        bool any = false;
        for (auto &kv : rep) any = any || !g_tune.count(kv.first);
        if (any) {
            BatchEngine eng;
            sinet_status st = eng.init(kTuneCopies, ds, smem);
            for (auto &kv : rep) {
                if (st != SINET_OK) break;
                if (g_tune.count(kv.first)) continue;
                int32_t best = -1;
                float ns = 0.f;
                st = tune_one(v[kv.second], ds, smem, s, eng, &best, &ns);
                if (st == SINET_OK && best >= 0) {
                    g_tune[kv.first] = best;
                    append_cache_file(kv.first, best, ns);
                }
            }
            eng.release();
            if (st != SINET_OK) return st;
        }
    }
    for (size_t i = 0; i < v.size(); ++i) {
        if (v[i].strategy != SINET_STRAT_AUTO) continue;
        auto it = g_tune.find(keys[i]);
        int32_t s_ = it != g_tune.end() ? it->second : fixed_rule(v[i]);
        if (s_ == SINET_STRAT_SMEM_FULL && !v[i].tile_fits) s_ = fixed_rule(v[i]);
        if (s_ == SINET_STRAT_SORT_REDUCE && !sort_feasible(v[i])) s_ = fixed_rule(v[i]);
        set_strategy(v[i], s_, batch_grid(ds));
    }
    return SINET_OK;
}

}  // namespace sinet

struct sinet_batch {
    sinet::BatchEngine eng;
    std::vector<int32_t> strategy;  // per caller slice
    uint64_t items = 0, records = 0;
};

using namespace sinet;

extern "C" {

sinet_status sinet_batch_create(const sinet_batch_slice *slices, uint32_t n_slices, uint32_t flags,
                                sinet_stream_t stream, sinet_batch **out) {
    SINET_TRACE();
    if (!out) return SINET_ERR_INVALID_ARG;
    *out = nullptr;
    if (!slices || n_slices == 0 || n_slices > 65536 || (flags & ~SINET_BATCH_AUTOTUNE))
        return SINET_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < n_slices; ++i) {
        const sinet_status st = check_slice(slices[i]);
        if (st != SINET_OK) return st;
    }
    DeviceState *ds = nullptr;
    sinet_status st = device_state(&ds);
    if (st != SINET_OK) return st;
    const uint32_t smem = batch_smem(ds);
    std::vector<PlannedSlice> v(n_slices);
    uint64_t records = 0;
    for (uint32_t i = 0; i < n_slices; ++i) {
        if ((st = plan_slice(slices[i], ds, smem, v[i])) != SINET_OK) return st;
        v[i].user_index = i;
        records += slices[i].n;
    }
    if ((st = resolve_strategies(v, (flags & SINET_BATCH_AUTOTUNE) != 0, ds, smem, stream)) != SINET_OK)
        return st;
    uint64_t items = 0, zitems = 0;
    for (const PlannedSlice &ps : v) {
        items += ps.items;
        zitems += ps.zero_items;
    }
    if (items >= 0xFFFFFFFFull || zitems >= 0xFFFFFFFFull) return SINET_ERR_UNSUPPORTED;
    // largest slices first: the last work items handed out are the small ones
    std::stable_sort(v.begin(), v.end(), [](const PlannedSlice &a, const PlannedSlice &b) {
        return a.d.r.g.quads > b.d.r.g.quads;
    });
    sinet_batch *b = new (std::nothrow) sinet_batch();
    if (!b) return SINET_ERR_OOM;
    b->strategy.resize(n_slices);
    for (const PlannedSlice &ps : v) b->strategy[ps.user_index] = ps.strategy;
    b->items = items;
    b->records = records;
    st = b->eng.init(n_slices, ds, smem);
    if (st == SINET_OK) st = b->eng.plan_sorts(v, ds);
    std::vector<uint8_t> buf;
    if (st == SINET_OK) {
        b->eng.image(v, buf);
        cudaError_t e = cudaMemcpyAsync(b->eng.d_mem, buf.data(), buf.size(), cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // host image goes out of scope
        if (e != cudaSuccess) st = cuda_fail(e);
    }
    if (st == SINET_OK) st = b->eng.capture(ds->status);
    if (st != SINET_OK) {
        b->eng.release();
        delete b;
        return st;
    }
    *out = b;
    return SINET_OK;
}

sinet_status sinet_batch_run(sinet_batch *b, sinet_stream_t stream) {
    SINET_TRACE();
    if (!b) return SINET_ERR_INVALID_ARG;
    int dev = 0;
    SINET_CUDA(cudaGetDevice(&dev));
    if (dev != b->eng.device) return SINET_ERR_INVALID_ARG;
    return b->eng.launch(stream);
}

sinet_status sinet_batch_set_wait(sinet_batch *b, uint64_t wait_ns) {
    if (!b) return SINET_ERR_INVALID_ARG;
    b->eng.wait_ns = wait_ns;
    SINET_CUDA(cudaMemcpy(reinterpret_cast<uint8_t *>(b->eng.d_mem) + offsetof(BatchHeader, wait_ns), &wait_ns,
                          sizeof wait_ns, cudaMemcpyHostToDevice));
    return SINET_OK;
}

sinet_status sinet_batch_strategy(const sinet_batch *b, uint32_t i, int32_t *strategy) {
    if (!b || !strategy || i >= b->strategy.size()) return SINET_ERR_INVALID_ARG;
    *strategy = b->strategy[i];
    return SINET_OK;
}

sinet_status sinet_batch_info(const sinet_batch *b, uint64_t *work_items, uint64_t *records) {
    if (!b) return SINET_ERR_INVALID_ARG;
    if (work_items) *work_items = b->items;
    if (records) *records = b->records;
    return SINET_OK;
}

sinet_status sinet_batch_destroy(sinet_batch *b) {
    if (!b) return SINET_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != b->eng.device) cudaSetDevice(b->eng.device);
    const cudaError_t e = cudaDeviceSynchronize();
    b->eng.release();
    if (cur != b->eng.device) cudaSetDevice(cur);
    delete b;
    return e == cudaSuccess ? SINET_OK : cuda_fail(e);
}

}  // extern "C"
