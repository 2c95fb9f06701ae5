// Update-combining pieces shared by the fused and batched kernels: the
// per-CTA hot-key cache, warp run-combining, and in-quad run merging.
#pragma once
#include "records.cuh"

namespace sinet {

// Per-CTA cache of hot (bin, direction) keys in shared memory: 4-way set
// associative, a key claims an empty way the first time it is seen and keeps
// it until the cache is flushed (skewed input puts its hottest keys in first);
// a key that finds its set full goes to global atomics. The fused kernel
// flushes it once per CTA, the batched kernel once per work item.
struct HotCache {
    uint32_t *keys;  // [ways * sets], kNoKey when empty
    uint32_t *cnt;
    uint32_t *lo;    // byte sums: low words
    uint32_t *hi;    // byte sums: high words
    uint32_t set_bits;

    static constexpr uint32_t kWays = 4;
    static constexpr uint32_t kSlotBytes = 16;

    __device__ __forceinline__ bool add(uint32_t key, uint32_t c, uint64_t s) {
        const uint32_t set = (key * 0x9E3779B1u) >> (32 - set_bits);
        uint32_t *kp = keys + kWays * set;
        uint4 k4;
        asm volatile("ld.volatile.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(k4.x), "=r"(k4.y), "=r"(k4.z), "=r"(k4.w)
                     : "r"(smem_u32(kp)));
        int way = k4.x == key ? 0 : k4.y == key ? 1 : k4.z == key ? 2 : k4.w == key ? 3 : -1;
        if (way < 0) {
            const uint32_t cur[4] = {k4.x, k4.y, k4.z, k4.w};
            bool tried = false;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                if (way < 0 && cur[w] == kNoKey) {
                    tried = true;
                    const uint32_t old = atomicCAS(kp + w, kNoKey, key);
                    if (old == kNoKey || old == key) way = w;
                }
            }
            // a claim lost to a racing lane may have put this key in another
            // way; a full set (the common miss once warm) tried no claim
            if (way < 0 && tried) {
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    if (way < 0 && *reinterpret_cast<volatile uint32_t *>(kp + w) == key) way = w;
            }
        }
        if (way < 0) return false;
        const uint32_t i = kWays * set + way;
        atomicAdd(cnt + i, c);
        smem_add_wide(lo + i, hi + i, s, 0u);
        return true;
    }
};

// Warp run-combining: lanes holding the same (bin, direction) key elect a
// leader that adds the group's count (popc of the peer mask) and byte sum.
// Byte sums are reduced as two 16-bit halves so 32 values of up to 2^32 - 1
// cannot overflow the 32-bit warp reduction; they are recombined in 64 bits.
__device__ __forceinline__ void update_agg(const HistArgs &h, HotCache &hc, uint32_t key, uint32_t b) {
    const uint32_t peers = __match_any_sync(kFull, key);
    if (key == kNoKey) return;
    const uint32_t c = __popc(peers);
    uint64_t s = b;
    if (c > 1) {
        const uint32_t lo = __reduce_add_sync(peers, b & 0xFFFFu);
        const uint32_t hi = __reduce_add_sync(peers, b >> 16);
        s = (uint64_t)lo + ((uint64_t)hi << 16);
    }
    if ((threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1)) {
        if (!hc.add(key, c, s)) gadd(h, key & 1u, key >> 1, c, s);
    }
}

// Walk a quad's records in order; consecutive records with the same (bin,
// direction) are merged in registers (time-sorted input repeats bins) and each
// run goes to `emit(key, count, bytes)` with key = bin << 1 | direction.
template <typename Emit>
__device__ __forceinline__ void combine_quad(const HistArgs &h, const Quad &Q, uint32_t cc[4],
                                             uint32_t oor[2], Emit &&emit) {
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
            if (pk != kNoKey) emit(pk, pc, ps);
            pk = key;
            pc = 1;
            ps = Q.by[j];
        }
        if (dirs == 3u) emit(bin << 1 | 1u, 1u, (uint64_t)Q.by[j]);
    }
    if (pk != kNoKey) emit(pk, pc, ps);
}

}  // namespace sinet
