// Host helpers shared by the C-ABI translation units.
#pragma once
#include <initializer_list>

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
