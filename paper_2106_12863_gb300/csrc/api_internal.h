// Host helpers shared by the C-ABI translation units.
#pragma once
#include <initializer_list>

#include <nvtx3/nvToolsExt.h>

#include "launch.h"
#include "table_host.h"

struct sinet_prefix_table {
    int device;
    sinet::TableHost host;
    sinet::TableImage img;
    uint8_t *d_image;
    sinet::TableArgs args;
};

namespace sinet {

constexpr uint64_t kMaxN = 1ull << 40;

// Per-device facts and the device status word, set up on first use.
struct DeviceState {
    bool ready = false;
    int sm_count = 0;
    size_t smem_optin = 0;
    size_t smem_per_sm = 0;
    uint32_t *status = nullptr;  // device status word
};
sinet_status device_state(DeviceState **out);
// Map a failed CUDA call to a status (and remember it for sinet_last_cuda_error).
sinet_status cuda_fail(cudaError_t e);

#define SINET_CUDA(x)                                          \
    do {                                                       \
        cudaError_t e_ = (x);                                  \
        if (e_ != cudaSuccess) return ::sinet::cuda_fail(e_);  \
    } while (0)

// A profiler-visible range around a C-ABI call (NVTX; it costs nothing when
// no tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
#define SINET_TRACE() ::sinet::TraceRange sinet_trace_range_(__func__)

struct Stream {
    const void *p;
    uint32_t esize;
};

Divider make_divider(uint64_t w);
QuadGeom make_geom(uint64_t n, std::initializer_list<Stream> streams);
bool aligned(const void *p, size_t a);
sinet_status check_params(const sinet_hist_params *p);
sinet_status check_out(const sinet_hist_out *o);
HistArgs make_hist(const sinet_hist_params *p, const sinet_hist_out *o);
sinet_status zero_outputs(const sinet_hist_params *p, const sinet_hist_out *o, cudaStream_t s);
int pick_lookup(const sinet_prefix_table *t, int32_t lookup, sinet_status *err);

}  // namespace sinet
