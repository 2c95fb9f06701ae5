// Histogram post-processing on the device: roll-up into coarser bins and
// sparse compaction of the non-empty bins (the downstream views of
// Section 6 use hourly and ten-minute bins; the reduce-by-key of Section 5
// yields only the present keys).
#include <algorithm>

#include "api_internal.h"

namespace sinet {
namespace {

constexpr uint32_t kPostBlock = 256;
constexpr uint32_t kRollPer = 16;       // input bins per thread
constexpr uint32_t kSparseTile = 4096;  // bins per compaction tile (16 per thread)

// Exact warp sum of 64-bit values over the lanes in `g`: three 22/22/20-bit
// slices, each summed in 32 bits without overflow (32 x 2^22 < 2^32), then
// recombined modulo 2^64.
__device__ __forceinline__ uint64_t reduce_add_u64(uint32_t g, uint64_t v) {
    const uint32_t a = __reduce_add_sync(g, (uint32_t)(v & 0x3FFFFFu));
    const uint32_t b = __reduce_add_sync(g, (uint32_t)((v >> 22) & 0x3FFFFFu));
    const uint32_t c = __reduce_add_sync(g, (uint32_t)(v >> 44));
    return (uint64_t)a + ((uint64_t)b << 22) + ((uint64_t)c << 44);
}

// Each thread sums kRollPer consecutive input bins per output bin and adds a
// run to the outputs when it ends inside its range; the run it holds at the
// end is combined with the lanes that hold the same output bin (consecutive
// lanes), and their leader adds it.
__global__ void __launch_bounds__(kPostBlock) k_rollup(HistArgs in, uint64_t factor, HistArgs out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * kRollPer;
    const uint64_t n = in.n_bins;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x * kRollPer; base < n; base += stride) {
        const uint64_t first = base + (uint64_t)threadIdx.x * kRollPer;
        uint32_t cur = first < n ? (uint32_t)(first / factor) : kNoKey;
        uint32_t sc0 = 0, sc1 = 0;
        uint64_t sb0 = 0, sb1 = 0;
        for (uint32_t k = 0; k < kRollPer; ++k) {
            const uint64_t i = first + k;
            if (i >= n) break;
            const uint32_t o = (uint32_t)(i / factor);
            if (o != cur) {
                red_add_u32(out.cnt[0] + cur, sc0);
                red_add_u32(out.cnt[1] + cur, sc1);
                red_add_u64(out.byt[0] + cur, sb0);
                red_add_u64(out.byt[1] + cur, sb1);
                sc0 = sc1 = 0;
                sb0 = sb1 = 0;
                cur = o;
            }
            sc0 += in.cnt[0][i];
            sc1 += in.cnt[1][i];
            sb0 += in.byt[0][i];
            sb1 += in.byt[1][i];
        }
        const uint32_t g = __match_any_sync(kFull, cur);
        sc0 = __reduce_add_sync(g, sc0);
        sc1 = __reduce_add_sync(g, sc1);
        sb0 = reduce_add_u64(g, sb0);
        sb1 = reduce_add_u64(g, sb1);
        if (cur != kNoKey && (threadIdx.x & 31) == (uint32_t)(__ffs(g) - 1)) {
            red_add_u32(out.cnt[0] + cur, sc0);
            red_add_u32(out.cnt[1] + cur, sc1);
            red_add_u64(out.byt[0] + cur, sb0);
            red_add_u64(out.byt[1] + cur, sb1);
        }
    }
}

__device__ __forceinline__ bool nonempty(const HistArgs &h, uint64_t i) {
    return (h.cnt[0][i] | h.cnt[1][i]) != 0 || (h.byt[0][i] | h.byt[1][i]) != 0;
}

// Sparse pass 1: non-empty bins per tile.
__global__ void __launch_bounds__(kPostBlock) k_sparse_count(HistArgs h, uint32_t *tile_count) {
    __shared__ uint32_t s_n;
    const uint64_t tiles = (h.n_bins + kSparseTile - 1) / kSparseTile;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        uint32_t c = 0;
        for (uint32_t k = threadIdx.x; k < kSparseTile; k += blockDim.x) {
            const uint64_t i = t * kSparseTile + k;
            if (i < h.n_bins && nonempty(h, i)) c++;
        }
        c = __reduce_add_sync(kFull, c);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_n, c);
        __syncthreads();
        if (threadIdx.x == 0) tile_count[t] = s_n;
        __syncthreads();
    }
}

// Sparse pass 2: exclusive scan of the tile counts by one CTA (u64 offsets)
// and the total.
__global__ void __launch_bounds__(1024) k_sparse_scan(const uint32_t *tile_count, uint64_t tiles,
                                                      uint64_t *tile_off, uint64_t *total) {
    __shared__ uint64_t s_warp[32];
    __shared__ uint64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t b = 0; b < tiles; b += blockDim.x) {
        const uint64_t t = b + threadIdx.x;
        const uint64_t v = t < tiles ? tile_count[t] : 0;
        uint64_t x = v;  // inclusive scan within the warp
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint64_t w = lane < (blockDim.x >> 5) ? s_warp[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(kFull, w, o);
                if (lane >= (uint32_t)o) w += y;
            }
            s_warp[lane] = w;  // inclusive totals of warps
        }
        __syncthreads();
        const uint64_t before = s_carry + (warp ? s_warp[warp - 1] : 0) + x - v;
        if (t < tiles) tile_off[t] = before;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_warp[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = s_carry;
}

// Sparse pass 3: each tile writes its non-empty bins in order at its offset
// (warp ballots give the order inside a warp, a shared scan across warps).
__global__ void __launch_bounds__(kPostBlock) k_sparse_write(HistArgs h, const uint64_t *tile_off, uint64_t cap,
                                                             uint32_t *o_bin, uint32_t *o_c0, uint32_t *o_c1,
                                                             uint64_t *o_b0, uint64_t *o_b1) {
    __shared__ uint32_t s_warp[kPostBlock / 32];
    __shared__ uint64_t s_base;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t tiles = (h.n_bins + kSparseTile - 1) / kSparseTile;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        if (threadIdx.x == 0) s_base = tile_off[t];
        __syncthreads();
        for (uint32_t k0 = 0; k0 < kSparseTile; k0 += blockDim.x) {
            const uint64_t i = t * kSparseTile + k0 + threadIdx.x;
            const bool keep = i < h.n_bins && nonempty(h, i);
            const uint32_t bal = __ballot_sync(kFull, keep);
            if (lane == 0) s_warp[warp] = __popc(bal);
            __syncthreads();
            uint32_t before = 0, all = 0;
            for (uint32_t w = 0; w < blockDim.x / 32; ++w) {
                if (w < warp) before += s_warp[w];
                all += s_warp[w];
            }
            if (keep) {
                const uint64_t pos = s_base + before + __popc(bal & ((1u << lane) - 1));
                if (pos < cap) {
                    o_bin[pos] = (uint32_t)i;
                    o_c0[pos] = h.cnt[0][i];
                    o_c1[pos] = h.cnt[1][i];
                    o_b0[pos] = h.byt[0][i];
                    o_b1[pos] = h.byt[1][i];
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) s_base += all;
            __syncthreads();
        }
    }
}

HistArgs view(const sinet_hist_out *o, uint64_t n_bins) {
    HistArgs h{};
    h.cnt[0] = o->count[0];
    h.cnt[1] = o->count[1];
    h.byt[0] = o->bytes[0];
    h.byt[1] = o->bytes[1];
    h.stats = o->stats;
    h.n_bins = (uint32_t)n_bins;
    return h;
}

bool out_arrays_ok(const sinet_hist_out *o) {
    return o && o->count[0] && o->count[1] && o->bytes[0] && o->bytes[1] && aligned(o->count[0], 4) &&
           aligned(o->count[1], 4) && aligned(o->bytes[0], 8) && aligned(o->bytes[1], 8);
}

}  // namespace
}  // namespace sinet

using namespace sinet;

extern "C" {

sinet_status sinet_histogram_rollup(const sinet_hist_out *in, uint64_t n_bins, uint64_t factor, int accumulate,
                                    const sinet_hist_out *out, sinet_stream_t stream) {
    SINET_TRACE();
    if (!out_arrays_ok(in) || !out_arrays_ok(out) || n_bins == 0 || n_bins > 0x7FFFFFFFull || factor == 0)
        return SINET_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    sinet_status st = device_state(&ds);
    if (st != SINET_OK) return st;
    const uint64_t n_out = (n_bins + factor - 1) / factor;
    if (!accumulate) {
        SINET_CUDA(cudaMemsetAsync(out->count[0], 0, 4 * n_out, stream));
        SINET_CUDA(cudaMemsetAsync(out->count[1], 0, 4 * n_out, stream));
        SINET_CUDA(cudaMemsetAsync(out->bytes[0], 0, 8 * n_out, stream));
        SINET_CUDA(cudaMemsetAsync(out->bytes[1], 0, 8 * n_out, stream));
    }
    if (in->stats && out->stats && in->stats != out->stats)
        SINET_CUDA(cudaMemcpyAsync(out->stats, in->stats, 64, cudaMemcpyDeviceToDevice, stream));
    const uint64_t threads = (n_bins + kRollPer - 1) / kRollPer;
    const int grid = (int)std::min<uint64_t>((threads + kPostBlock - 1) / kPostBlock, 8ull * ds->sm_count);
    k_rollup<<<grid, kPostBlock, 0, stream>>>(view(in, n_bins), factor, view(out, n_out));
    SINET_CUDA(cudaGetLastError());
    return SINET_OK;
}

sinet_status sinet_histogram_sparse(const sinet_hist_out *in, uint64_t n_bins, uint32_t *d_bin, uint32_t *d_count0,
                                    uint32_t *d_count1, uint64_t *d_bytes0, uint64_t *d_bytes1, uint64_t cap,
                                    uint64_t *d_n_out, sinet_stream_t stream) {
    SINET_TRACE();
    if (!out_arrays_ok(in) || n_bins == 0 || n_bins > 0x7FFFFFFFull || !d_n_out || !aligned(d_n_out, 8))
        return SINET_ERR_INVALID_ARG;
    if (cap && (!d_bin || !d_count0 || !d_count1 || !d_bytes0 || !d_bytes1 || !aligned(d_bin, 4) ||
                !aligned(d_count0, 4) || !aligned(d_count1, 4) || !aligned(d_bytes0, 8) || !aligned(d_bytes1, 8)))
        return SINET_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    sinet_status st = device_state(&ds);
    if (st != SINET_OK) return st;
    const uint64_t tiles = (n_bins + kSparseTile - 1) / kSparseTile;
    void *scratch = nullptr;
    SINET_CUDA(cudaMallocAsync(&scratch, 12 * tiles + 16, stream));
    uint64_t *tile_off = static_cast<uint64_t *>(scratch);
    uint32_t *tile_count = reinterpret_cast<uint32_t *>(tile_off + tiles);
    const HistArgs h = view(in, n_bins);
    const int grid = (int)std::min<uint64_t>(tiles, 8ull * ds->sm_count);
    k_sparse_count<<<grid, kPostBlock, 0, stream>>>(h, tile_count);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_sparse_scan<<<1, 1024, 0, stream>>>(tile_count, tiles, tile_off, d_n_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_sparse_write<<<grid, kPostBlock, 0, stream>>>(h, tile_off, cap, d_bin, d_count0, d_count1, d_bytes0,
                                                        d_bytes1);
        e = cudaGetLastError();
    }
    const cudaError_t e2 = cudaFreeAsync(scratch, stream);
    if (e == cudaSuccess) e = e2;
    return e == cudaSuccess ? SINET_OK : cuda_fail(e);
}

}  // extern "C"
