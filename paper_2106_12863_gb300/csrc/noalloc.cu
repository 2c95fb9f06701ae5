// Allocation-free entry point: the plain discriminate -> radix sort ->
// reduce-by-key path with its scratch in a fixed, file-scope device array
// instead of memory allocated per call.
//
// Who needs it: callers that must not allocate device memory on the call
// path, such as a host application whose memory manager owns every device
// allocation, or a latency-bound loop that cannot afford an allocator call
// (which may synchronise or fail under fragmentation). They pass inputs and
// outputs; everything else this path needs lives in the array below.
#include <mutex>

#include "api_internal.h"

namespace sinet {
namespace {

// Scratch for the plain path: about 16.5 bytes per routed record, so a
// little over 2 M records with a one-direction policy (half that when a
// class routes to both directions). Every GPU that loads the library holds
// this array until the process exits.
constexpr size_t kNoAllocScratchBytes = 32ull << 20;
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
    bool ready = false;
    int sm_count = 0;
    void *scratch = nullptr;  // device address of g_noalloc_scratch on this device
};

std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[64];

// Once per device, with that device current: look up the array's device
// address. In host code the name g_noalloc_scratch is only a host-side stand-in,
// so only this looked-up address is ever passed to a kernel.
sinet_status noalloc_setup(NoAllocDevice **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SINET_ERR_CUDA;
    if (dev < 0 || dev >= 64) return SINET_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDevice &d = g_noalloc_dev[dev];
    if (!d.ready) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return SINET_ERR_CUDA;
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
            return SINET_ERR_CUDA;
        d.sm_count = v;
        d.scratch = p;
        d.ready = true;
    }
    *out = &d;
    return SINET_OK;
}

}  // namespace
}  // namespace sinet

using namespace sinet;

extern "C" sinet_status sinet_discriminate_histogram_noalloc(
    const sinet_prefix_table *t, const uint64_t *d_ts, const uint32_t *d_src, const uint32_t *d_dst,
    const uint32_t *d_bytes, uint64_t n, const sinet_hist_params *p, const sinet_hist_out *o,
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
    if (p->watch) return SINET_ERR_UNSUPPORTED;
    HistArgs h = make_hist(p, o);
    if (n * (h.two_dir ? 2ull : 1ull) >= 0xFFFFFFF0ull) return SINET_ERR_BUDGET;
    const SortPlan plan = plan_sort_reduce(n, h.n_bins, h.two_dir);
    if (plan.scratch_bytes > kNoAllocScratchBytes) return SINET_ERR_BUDGET;

    NoAllocDevice *d = nullptr;
    if ((st = noalloc_setup(&d)) != SINET_OK) return st;
    // this call's device-side status starts clear, accumulating or not, so a
    // failure latched by an earlier call is not reported again
    if (cudaMemsetAsync(o->stats + 7, 0, 4, stream) != cudaSuccess) return SINET_ERR_CUDA;
    if ((st = zero_outputs(p, o, stream)) != SINET_OK) return st;
    if (n == 0) return SINET_OK;

    RecArgs r{};
    r.ts = d_ts;
    r.src = d_src;
    r.dst = d_dst;
    r.bytes = d_bytes;
    r.g = make_geom(n, {{d_ts, 8}, {d_src, 4}, {d_dst, 4}, {d_bytes, 4}});
    LaunchCfg c;
    c.stream = stream;
    c.sm_count = d->sm_count;
    // device-side failures of this call latch into the low word of stats[7]
    c.status = reinterpret_cast<uint32_t *>(o->stats + 7);
    // run_sort_reduce clears the counters, digit counts and look-back words
    // at the start of the scratch before any kernel reads them
    const cudaError_t e = run_sort_reduce(lk, r, t->args, h, plan, d->scratch, p->accumulate != 0, c);
    return e == cudaSuccess ? SINET_OK : SINET_ERR_CUDA;
}
