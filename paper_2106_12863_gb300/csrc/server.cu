// Serving loop with continuous batching: tenants with resident histograms, a
// device arena for the records of admitted requests, and a worker thread that
// admits requests in arrival order, overlaps their host-to-device copies with
// the running launch, and starts the next batched launch over every request
// that is ready (Section 4's bounded work queue, on one GPU).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda.h>

#include "batch_internal.h"

namespace sinet {
namespace {

// The driver's stream write (a front-end operation: it needs no SM) ends a
// request's copies by setting its ready word, so a launch can start while
// the copies are still landing.
typedef CUresult (*StreamWriteValue32)(CUstream, CUdeviceptr, cuuint32_t, unsigned int);

StreamWriteValue32 stream_write_fn() {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue32", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return reinterpret_cast<StreamWriteValue32>(fn);
}

// Value of a request's ready word: never 0 (the words start at 0), and
// distinct for tickets less than 2^32 - 1 apart.
uint32_t ready_value(uint64_t ticket) { return 1u + (uint32_t)(ticket % 0xFFFFFFFFull); }

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Device bytes of a request's records: four streams, each 16-byte aligned.
size_t record_bytes(uint64_t n) { return round_up(8 * n, 16) + 3 * round_up(4 * n, 16); }

// First-fit allocator of byte ranges of the device arena (256-byte granules),
// coalescing freed neighbours.
class Arena {
  public:
    void init(size_t bytes) {
        free_.clear();
        total_ = bytes & ~(size_t)255;
        if (total_) free_[0] = total_;
    }
    size_t total() const { return total_; }
    bool alloc(size_t bytes, size_t *off) {
        bytes = round_up(std::max<size_t>(bytes, 1), 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t o = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[o + bytes] = rest;
            *off = o;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = round_up(std::max<size_t>(bytes, 1), 256);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<size_t, size_t> free_;  // offset -> size
    size_t total_ = 0;
};

struct Request {
    uint64_t ticket = 0;
    uint32_t tenant = 0;
    const uint64_t *ts = nullptr;
    const uint32_t *src = nullptr, *dst = nullptr, *by = nullptr;
    uint64_t n = 0;
    size_t off = 0, bytes = 0;
    uint32_t slot = 0;  // index of its ready word
    uint64_t submit_ns = 0, done_ns = 0, launch = 0;
    bool done = false;
};

struct Tenant {
    const sinet_prefix_table *table = nullptr;
    sinet_hist_params params{};
    int32_t strategy = SINET_STRAT_AUTO;
    sinet_hist_out out{};
};

}  // namespace
}  // namespace sinet

struct sinet_server {
    int device = 0;
    sinet_server_config cfg{};
    std::vector<sinet::Tenant> tenants;
    sinet::DeviceState *ds = nullptr;
    uint32_t smem = 0;
    uint8_t *arena_mem = nullptr;
    sinet::Arena arena;
    sinet::BatchEngine eng;
    uint8_t *stage = nullptr;  // pinned host image of the launch's descriptors
    cudaStream_t copy_stream = nullptr, compute_stream = nullptr;
    cudaEvent_t copied = nullptr, launch_done = nullptr;
    uint32_t *flags = nullptr;          // ready words, one per admission slot
    std::vector<uint32_t> free_slots;   // admission slots not in use
    sinet::StreamWriteValue32 write32 = nullptr;  // null: launches wait on the copy event instead

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<sinet::Request *> pending;   // submitted, waiting for arena space
    std::vector<sinet::Request *> ready;    // records copied (or in flight), not launched
    std::vector<sinet::Request *> inflight; // in the running launch
    std::unordered_map<uint64_t, sinet::Request *> by_ticket;
    uint64_t next_ticket = 1;
    uint64_t outstanding = 0;  // submitted, not done
    bool stop = false;
    bool launch_active = false;
    uint64_t launch_start_ns = 0;
    sinet_status error = SINET_OK;  // sticky worker failure

    uint64_t launches = 0, requests_done = 0, records_done = 0, busy_ns = 0;
    std::vector<uint64_t> latencies;
    std::thread worker;
};

namespace sinet {
namespace {

// Descriptors of one launch: one slice per request, accumulating into its
// tenant's resident histogram.
sinet_status plan_launch(sinet_server *s, const std::vector<Request *> &reqs, std::vector<PlannedSlice> &v) {
    v.resize(reqs.size());
    for (size_t i = 0; i < reqs.size(); ++i) {
        const Request *r = reqs[i];
        const Tenant &t = s->tenants[r->tenant];
        sinet_batch_slice u{};
        uint8_t *base = s->arena_mem + r->off;
        u.ts = reinterpret_cast<const uint64_t *>(base);
        u.src = reinterpret_cast<const uint32_t *>(base + round_up(8 * r->n, 16));
        u.dst = reinterpret_cast<const uint32_t *>(base + round_up(8 * r->n, 16) + round_up(4 * r->n, 16));
        u.bytes = reinterpret_cast<const uint32_t *>(base + round_up(8 * r->n, 16) + 2 * round_up(4 * r->n, 16));
        u.n = r->n;
        u.table = t.table;
        u.params = t.params;
        u.params.strategy = t.strategy;
        u.out = t.out;
        if (s->write32 && r->n) {
            u.ready = s->flags + r->slot;
            u.ready_value = ready_value(r->ticket);
        }
        const sinet_status st = plan_slice(u, s->ds, s->smem, v[i]);
        if (st != SINET_OK) return st;
    }
    return SINET_OK;
}

void finish_launch(sinet_server *s) {
    const uint64_t t = now_ns();
    s->busy_ns += t - s->launch_start_ns;
    for (Request *r : s->inflight) {
        r->done = true;
        r->done_ns = t;
        s->arena.release(r->off, r->bytes);
        s->free_slots.push_back(r->slot);
        s->latencies.push_back(t - r->submit_ns);
        s->requests_done++;
        s->records_done += r->n;
        s->outstanding--;
    }
    s->inflight.clear();
    s->launch_active = false;
    s->cv_done.notify_all();
}

void worker_main(sinet_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    std::vector<PlannedSlice> plan;
    std::vector<uint8_t> img;
    while (!s->stop) {
        bool progressed = false;
        // admission in arrival order while the arena has room; the copies go
        // out on the copy stream and overlap the running launch
        while (!s->pending.empty() && s->error == SINET_OK) {
            Request *r = s->pending.front();
            size_t off = 0;
            if (s->free_slots.empty()) break;  // admission by slot ...
            if (r->n && !s->arena.alloc(r->bytes, &off)) break;  // ... and by HBM budget
            r->off = off;
            r->slot = s->free_slots.back();
            s->free_slots.pop_back();
            s->pending.pop_front();
            if (r->n) {
                uint8_t *base = s->arena_mem + off;
                const size_t o1 = round_up(8 * r->n, 16), o2 = o1 + round_up(4 * r->n, 16),
                             o3 = o2 + round_up(4 * r->n, 16);
                lk.unlock();  // a copy from pageable memory blocks the thread
                cudaError_t e = cudaMemcpyAsync(base, r->ts, 8 * r->n, cudaMemcpyHostToDevice, s->copy_stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(base + o1, r->src, 4 * r->n, cudaMemcpyHostToDevice, s->copy_stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(base + o2, r->dst, 4 * r->n, cudaMemcpyHostToDevice, s->copy_stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(base + o3, r->by, 4 * r->n, cudaMemcpyHostToDevice, s->copy_stream);
                if (e == cudaSuccess && s->write32 &&
                    s->write32(reinterpret_cast<CUstream>(s->copy_stream),
                               reinterpret_cast<CUdeviceptr>(s->flags + r->slot), ready_value(r->ticket),
                               CU_STREAM_WRITE_VALUE_DEFAULT) != CUDA_SUCCESS)
                    e = cudaErrorUnknown;
                lk.lock();
                if (e != cudaSuccess) s->error = cuda_fail(e);
            }
            s->ready.push_back(r);
            progressed = true;
        }
        if (s->launch_active) {
            const cudaError_t q = cudaEventQuery(s->launch_done);
            if (q == cudaSuccess) {
                finish_launch(s);
                progressed = true;
            } else if (q != cudaErrorNotReady) {
                s->error = cuda_fail(q);
            }
        }
        if (!s->launch_active && !s->ready.empty() && s->error == SINET_OK) {
            TraceRange range("sinet_server_launch");
            const size_t take = std::min<size_t>(s->ready.size(), s->cfg.max_requests_per_launch);
            std::vector<Request *> batch(s->ready.begin(), s->ready.begin() + take);
            s->ready.erase(s->ready.begin(), s->ready.begin() + take);
            sinet_status st = plan_launch(s, batch, plan);
            cudaError_t e = cudaSuccess;
            if (st == SINET_OK) {
                s->eng.image(plan, img);
                std::memcpy(s->stage, img.data(), img.size());
                // the launch starts at once and each request's work waits for
                // its ready word; without stream writes it waits for every
                // copy issued so far
                if (!s->write32) {
                    e = cudaEventRecord(s->copied, s->copy_stream);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->compute_stream, s->copied, 0);
                }
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(s->eng.d_mem, s->stage, img.size(), cudaMemcpyHostToDevice,
                                        s->compute_stream);
                if (e == cudaSuccess) st = s->eng.launch(s->compute_stream);
                if (e == cudaSuccess && st == SINET_OK) e = cudaEventRecord(s->launch_done, s->compute_stream);
            }
            if (st == SINET_OK && e != cudaSuccess) st = cuda_fail(e);
            if (st != SINET_OK) {
                s->error = st;
            } else {
                s->launches++;
                for (Request *r : batch) r->launch = s->launches;
                s->inflight = std::move(batch);
                s->launch_active = true;
                s->launch_start_ns = now_ns();
            }
            progressed = true;
        }
        if (s->error != SINET_OK) s->cv_done.notify_all();
        if (!progressed) s->cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
}

}  // namespace
}  // namespace sinet

using namespace sinet;

extern "C" {

sinet_status sinet_server_create(const sinet_server_config *cfg, const sinet_tenant *tenants, uint32_t n_tenants,
                                 sinet_server **out) {
    SINET_TRACE();
    if (!out) return SINET_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || !tenants || n_tenants == 0 || cfg->inflight_budget_bytes < (1u << 20) ||
        cfg->max_requests_per_launch == 0 || cfg->max_requests_per_launch > 4096 || cfg->max_queued == 0)
        return SINET_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < n_tenants; ++i) {
        sinet_batch_slice u{};
        u.table = tenants[i].table;
        u.params = tenants[i].params;
        u.params.accumulate = 1;
        u.out.count[0] = u.out.count[1] = reinterpret_cast<uint32_t *>(16);  // checked below, allocated later
        u.out.bytes[0] = u.out.bytes[1] = reinterpret_cast<uint64_t *>(16);
        u.out.stats = reinterpret_cast<uint64_t *>(16);
        const sinet_status st = check_slice(u);
        if (st != SINET_OK) return st;
        // requests join shared launches of the batch kernel: the plain path,
        // a chain of its own per slice, is not run by the server
        if (u.params.strategy == SINET_STRAT_SORT_REDUCE) return SINET_ERR_UNSUPPORTED;
    }
    DeviceState *ds = nullptr;
    sinet_status st = device_state(&ds);
    if (st != SINET_OK) return st;
    sinet_server *s = new (std::nothrow) sinet_server();
    if (!s) return SINET_ERR_OOM;
    s->cfg = *cfg;
    s->ds = ds;
    s->smem = batch_smem(ds);
    cudaError_t e = cudaGetDevice(&s->device);
    s->tenants.resize(n_tenants);
    for (uint32_t i = 0; i < n_tenants && e == cudaSuccess; ++i) {
        Tenant &t = s->tenants[i];
        t.table = tenants[i].table;
        t.params = tenants[i].params;
        t.params.accumulate = 1;
        const uint64_t nb = t.params.n_bins;
        uint8_t *m = nullptr;
        const size_t bytes = round_up(8 * nb, 16) + 16 * nb + 64;
        e = cudaMalloc(&m, bytes);
        if (e == cudaSuccess) e = cudaMemset(m, 0, bytes);
        if (e != cudaSuccess) break;
        t.out.count[0] = reinterpret_cast<uint32_t *>(m);
        t.out.count[1] = t.out.count[0] + nb;
        t.out.bytes[0] = reinterpret_cast<uint64_t *>(m + round_up(8 * nb, 16));
        t.out.bytes[1] = t.out.bytes[0] + nb;
        t.out.stats = t.out.bytes[1] + nb;
        // the strategy: as given, or tile / combining / plain atomics by size
        sinet_batch_slice u{};
        u.table = t.table;
        u.params = t.params;
        u.out = t.out;
        PlannedSlice ps;
        if ((st = plan_slice(u, ds, s->smem, ps)) != SINET_OK) break;
        t.strategy = t.params.strategy;
        if (t.strategy == SINET_STRAT_AUTO)
            t.strategy = ps.tile_fits ? SINET_STRAT_SMEM_FULL
                         : 24 * nb <= (64ull << 20) ? SINET_STRAT_GLOBAL_ATOMIC
                                                    : SINET_STRAT_ATOMIC_NOAGG;
    }
    // admission slots (each with a ready word): four launches' worth
    const uint32_t slots = 4 * cfg->max_requests_per_launch;
    if (e == cudaSuccess && st == SINET_OK) e = cudaMalloc(&s->flags, 4 * (size_t)slots);
    if (e == cudaSuccess && st == SINET_OK) e = cudaMemset(s->flags, 0, 4 * (size_t)slots);
    for (uint32_t i = 0; i < slots; ++i) s->free_slots.push_back(slots - 1 - i);
    if (e == cudaSuccess && st == SINET_OK) e = cudaMalloc(&s->arena_mem, cfg->inflight_budget_bytes);
    if (e == cudaSuccess) s->arena.init(cfg->inflight_budget_bytes);
    if (e == cudaSuccess && st == SINET_OK) st = s->eng.init(cfg->max_requests_per_launch, ds, s->smem);
    // a request's items may wait behind every copy admitted before it
    s->eng.wait_ns = 30000000000ull;
    if (e == cudaSuccess && st == SINET_OK) e = cudaMallocHost(&s->stage, s->eng.bytes);
    if (e == cudaSuccess && st == SINET_OK) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && st == SINET_OK) e = cudaStreamCreateWithFlags(&s->compute_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && st == SINET_OK) e = cudaEventCreateWithFlags(&s->copied, cudaEventDisableTiming);
    if (e == cudaSuccess && st == SINET_OK) e = cudaEventCreateWithFlags(&s->launch_done, cudaEventDisableTiming);
    if (e == cudaSuccess && st == SINET_OK) st = s->eng.capture(ds->status);
    if (e == cudaSuccess && st == SINET_OK) {
        // stream writes in use only if one goes through here
        s->write32 = stream_write_fn();
        if (s->write32 &&
            (s->write32(reinterpret_cast<CUstream>(s->copy_stream), reinterpret_cast<CUdeviceptr>(s->flags), 0,
                        CU_STREAM_WRITE_VALUE_DEFAULT) != CUDA_SUCCESS ||
             cudaStreamSynchronize(s->copy_stream) != cudaSuccess))
            s->write32 = nullptr;
    }
    if (e != cudaSuccess && st == SINET_OK) st = cuda_fail(e);
    if (st == SINET_OK) {
        s->worker = std::thread(worker_main, s);
        *out = s;
        return SINET_OK;
    }
    sinet_server_destroy(s);
    return st;
}

sinet_status sinet_server_submit(sinet_server *s, uint32_t tenant, const uint64_t *h_ts, const uint32_t *h_src,
                                 const uint32_t *h_dst, const uint32_t *h_bytes, uint64_t n, uint64_t *ticket) {
    if (!s || !ticket || tenant >= s->tenants.size() || n > kMaxN) return SINET_ERR_INVALID_ARG;
    if (n && (!h_ts || !h_src || !h_dst || !h_bytes || !aligned(h_ts, 8) || !aligned(h_src, 4) ||
              !aligned(h_dst, 4) || !aligned(h_bytes, 4)))
        return SINET_ERR_INVALID_ARG;
    const size_t bytes = n ? record_bytes(n) : 0;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error != SINET_OK) return s->error;
    if (bytes > s->arena.total() || s->outstanding >= s->cfg.max_queued) return SINET_ERR_BUDGET;
    Request *r = new (std::nothrow) Request();
    if (!r) return SINET_ERR_OOM;
    r->ticket = s->next_ticket++;
    r->tenant = tenant;
    r->ts = h_ts;
    r->src = h_src;
    r->dst = h_dst;
    r->by = h_bytes;
    r->n = n;
    r->bytes = bytes;
    r->submit_ns = now_ns();
    s->pending.push_back(r);
    s->by_ticket[r->ticket] = r;
    s->outstanding++;
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return SINET_OK;
}

sinet_status sinet_server_wait(sinet_server *s, uint64_t ticket, uint32_t timeout_ms, sinet_request_info *info) {
    if (!s) return SINET_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->by_ticket.find(ticket);
    if (it == s->by_ticket.end()) return SINET_ERR_INVALID_ARG;
    Request *r = it->second;
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return r->done || s->error != SINET_OK; });
    if (!r->done) return ok ? s->error : SINET_ERR_TIMEOUT;
    if (info) {
        info->n = r->n;
        info->launch = r->launch;
        info->latency_ns = r->done_ns - r->submit_ns;
    }
    s->by_ticket.erase(it);
    delete r;
    return SINET_OK;
}

sinet_status sinet_server_drain(sinet_server *s, uint32_t timeout_ms) {
    if (!s) return SINET_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return s->outstanding == 0 || s->error != SINET_OK; });
    if (s->error != SINET_OK) return s->error;
    return ok ? SINET_OK : SINET_ERR_TIMEOUT;
}

sinet_status sinet_server_tenant_output(sinet_server *s, uint32_t tenant, sinet_hist_out *out) {
    if (!s || !out || tenant >= s->tenants.size()) return SINET_ERR_INVALID_ARG;
    *out = s->tenants[tenant].out;
    return SINET_OK;
}

sinet_status sinet_server_export(sinet_server *s, uint32_t tenant, uint32_t *h_count, uint64_t *h_bytes,
                                 uint64_t *h_stats) {
    SINET_TRACE();
    if (!s || tenant >= s->tenants.size() || !h_count || !h_bytes || !h_stats) return SINET_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);  // no launch starts meanwhile
    const Tenant &t = s->tenants[tenant];
    const uint64_t nb = t.params.n_bins;
    SINET_CUDA(cudaStreamSynchronize(s->compute_stream));
    SINET_CUDA(cudaMemcpy(h_count, t.out.count[0], 8 * nb, cudaMemcpyDeviceToHost));
    SINET_CUDA(cudaMemcpy(h_bytes, t.out.bytes[0], 16 * nb, cudaMemcpyDeviceToHost));
    SINET_CUDA(cudaMemcpy(h_stats, t.out.stats, 64, cudaMemcpyDeviceToHost));
    return SINET_OK;
}

sinet_status sinet_server_import(sinet_server *s, uint32_t tenant, const uint32_t *h_count, const uint64_t *h_bytes,
                                 const uint64_t *h_stats) {
    SINET_TRACE();
    if (!s || tenant >= s->tenants.size() || !h_count || !h_bytes || !h_stats) return SINET_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);  // no launch starts meanwhile
    const Tenant &t = s->tenants[tenant];
    const uint64_t nb = t.params.n_bins;
    SINET_CUDA(cudaStreamSynchronize(s->compute_stream));
    SINET_CUDA(cudaMemcpy(t.out.count[0], h_count, 8 * nb, cudaMemcpyHostToDevice));
    SINET_CUDA(cudaMemcpy(t.out.bytes[0], h_bytes, 16 * nb, cudaMemcpyHostToDevice));
    SINET_CUDA(cudaMemcpy(t.out.stats, h_stats, 64, cudaMemcpyHostToDevice));
    return SINET_OK;
}

sinet_status sinet_server_stats(sinet_server *s, int reset, sinet_server_counters *st) {
    if (!s || !st) return SINET_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(st, 0, sizeof *st);
    st->requests_done = s->requests_done;
    st->records_done = s->records_done;
    st->launches = s->launches;
    st->busy_ns = s->busy_ns;
    std::vector<uint64_t> l = s->latencies;
    if (!l.empty()) {
        const size_t i50 = (l.size() - 1) / 2, i99 = (size_t)((double)(l.size() - 1) * 0.99);
        std::nth_element(l.begin(), l.begin() + i50, l.end());
        st->p50_latency_ns = l[i50];
        std::nth_element(l.begin(), l.begin() + i99, l.end());
        st->p99_latency_ns = l[i99];
        st->max_latency_ns = *std::max_element(l.begin(), l.end());
    }
    if (reset) {
        s->latencies.clear();
        s->requests_done = s->records_done = s->launches = s->busy_ns = 0;
    }
    return SINET_OK;
}

sinet_status sinet_server_destroy(sinet_server *s) {
    if (!s) return SINET_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    if (s->compute_stream) cudaStreamSynchronize(s->compute_stream);
    if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
    for (auto &kv : s->by_ticket) delete kv.second;
    for (Tenant &t : s->tenants)
        if (t.out.count[0]) cudaFree(t.out.count[0]);
    if (s->arena_mem) cudaFree(s->arena_mem);
    if (s->flags) cudaFree(s->flags);
    s->eng.release();
    if (s->stage) cudaFreeHost(s->stage);
    if (s->copied) cudaEventDestroy(s->copied);
    if (s->launch_done) cudaEventDestroy(s->launch_done);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->compute_stream) cudaStreamDestroy(s->compute_stream);
    if (cur != s->device) cudaSetDevice(cur);
    delete s;
    return SINET_OK;
}

}  // extern "C"
