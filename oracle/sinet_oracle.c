/*
 * Plain CPU oracle for session discrimination and millisecond histogramming.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library. The product path never does, and this
 * file shares no code, header, table or helper with the CUDA library.
 *
 * What it computes, in the paper's notation (Algorithm 1 and Section 5):
 *   - bitmask(X, Z) keeps the top Z bits of the 32-bit address X (first octet
 *     most significant); Z = 0 keeps nothing. (Algorithm 1, Fig. 4.)
 *   - For a CIDR entry Y/Z of the list and an address X: SB = bitmask(X, Z),
 *     CB = bitmask(Y, Z), result = SB - CB; a zero result is a match.
 *     (Algorithm 1.) An address is "in the list" when any entry matches
 *     (the input is a CIDR list: membership in the union).
 *   - Each record gets class = src_in | dst_in << 1 (0 neither, 1 src inside =
 *     outgoing, 2 dst inside = ingoing, 3 both). A 4-entry policy maps a class
 *     to a set of directions (bit 0 = outgoing, bit 1 = ingoing); the literal
 *     Algorithm 1 (mark outgoing when the source matches, else ingoing) is the
 *     policy {IN, OUT, IN, OUT}.
 *   - Histogram (Section 5, "Pairwise Reduction" and "Merge Scatter": maps
 *     <timestamp,count> and <timestamp,bytes> at 1 ms granularity): for each
 *     routed direction d, if t0 <= ts < t0 + n_bins * w then
 *     count[d][(ts - t0) / w] += 1 (uint32, wraps) and
 *     bytes[d][(ts - t0) / w] += bytes (uint64); otherwise oor[d] += 1.
 *   - stats[0..3] = records per class, stats[4..5] = out-of-range per direction.
 *   - Watch list (the blocklist analyses of Section 6, as a filter): with a
 *     second CIDR list, a record whose src and dst are both outside it is not
 *     classified or binned at all; it only counts in stats[6].
 *
 * Every loop is the definition written out: a loop over records, and for each
 * record a loop over EVERY table entry. No index, no sorting, no early exit.
 * Classification runs in parallel over records (OpenMP); the histogram pass is
 * a single sequential loop.
 *
 * ORACLE_MUTANT (compile-time, tests only) plants one known mistake so the
 * test suite can show that its pins catch it; the default build has none.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* bitmask(X, Z) of Algorithm 1: the top Z bits of X, the rest zero. */
uint32_t oracle_bitmask(uint32_t x, uint32_t z) {
#if ORACLE_MUTANT == 1
    /* planted: one bit too few */
    if (z <= 1) return 0;
    return x & (0xFFFFFFFFu << (33 - z));
#elif ORACLE_MUTANT == 2
    /* planted: Z = 0 behaves like a 32-bit shift that wraps (keeps all bits) */
    if (z == 0) return x;
    return x & (0xFFFFFFFFu << (32 - z));
#else
    if (z == 0) return 0u; /* a 32-bit shift by 32 is undefined in C */
    return x & (0xFFFFFFFFu << (32 - z));
#endif
}

/* 1 if X matches any CIDR entry Y/Z of the list (Algorithm 1, per entry). */
int oracle_in_list(uint32_t x, const uint32_t *net, const uint8_t *len, uint32_t n_entries) {
    int hit = 0;
    for (uint32_t p = 0; p < n_entries; p++) {
        uint32_t SB = oracle_bitmask(x, len[p]);
#if ORACLE_MUTANT == 3
        uint32_t CB = net[p]; /* planted: the CIDR's host bits are not masked */
#else
        uint32_t CB = oracle_bitmask(net[p], len[p]);
#endif
        uint32_t result = SB - CB;
        hit |= (result == 0u);
    }
    return hit;
}

/* class of one record */
static uint8_t classify_one(uint32_t s, uint32_t d, const uint32_t *net, const uint8_t *len,
                            uint32_t n_entries) {
    int s_in = oracle_in_list(s, net, len, n_entries);
    int d_in = oracle_in_list(d, net, len, n_entries);
#if ORACLE_MUTANT == 4
    return (uint8_t)(d_in | (s_in << 1)); /* planted: src and dst bits swapped */
#elif ORACLE_MUTANT == 5
    (void)d_in;
    return (uint8_t)(s_in); /* planted: destination never tested */
#else
    return (uint8_t)(s_in | (d_in << 1));
#endif
}

/* class[i] for every record. */
void oracle_classify(const uint32_t *net, const uint8_t *len, uint32_t n_entries,
                     const uint32_t *src, const uint32_t *dst, uint64_t n, uint8_t *cls) {
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < (int64_t)n; i++) cls[i] = classify_one(src[i], dst[i], net, len, n_entries);
}

/* One record's contribution to the histogram (shared by the full and the
 * sampled forms below, which differ only in which bins they keep). */
static int bin_of(uint64_t ts, uint64_t t0, uint64_t w, uint64_t n_bins, uint64_t *bin) {
#if ORACLE_MUTANT == 6
    /* planted: the window's right edge is included */
    if (ts < t0) return 0;
    uint64_t b = (ts - t0) / w;
    if (b > n_bins) return 0;
    if (b == n_bins) b = n_bins - 1;
    *bin = b;
    return 1;
#elif ORACLE_MUTANT == 7
    /* planted: records before t0 wrap around instead of being out of range */
    uint64_t b = (uint64_t)((int64_t)(ts - t0) / (int64_t)w) % n_bins;
    *bin = b;
    return 1;
#else
    if (ts < t0) return 0;
    uint64_t b = (ts - t0) / w;
    if (b >= n_bins) return 0;
    *bin = b;
    return 1;
#endif
}

static inline uint8_t directions(const uint8_t *policy, uint8_t c) {
#if ORACLE_MUTANT == 8
    return policy[3 - c]; /* planted: policy read backwards */
#else
    return policy[c];
#endif
}

static inline void add_bytes(uint64_t *dst, uint32_t b) {
#if ORACLE_MUTANT == 9
    *dst = (uint32_t)(*dst + b); /* planted: byte sums kept in 32 bits */
#else
    *dst += b;
#endif
}

/*
 * Histogram of classified records, accumulating into caller arrays
 * (count[d] u32[n_bins], bytes[d] u64[n_bins], stats u64[8]); the caller
 * zeroes them for a fresh histogram. Sequential.
 */
void oracle_histogram(const uint64_t *ts, const uint32_t *bytes, const uint8_t *cls, uint64_t n,
                      uint64_t t0, uint64_t w, uint64_t n_bins, const uint8_t *policy,
                      uint32_t *count0, uint32_t *count1, uint64_t *bytes0, uint64_t *bytes1,
                      uint64_t *stats) {
    uint32_t *count[2] = {count0, count1};
    uint64_t *bsum[2] = {bytes0, bytes1};
    for (uint64_t i = 0; i < n; i++) {
        uint8_t c = cls[i];
        stats[c] += 1;
        uint8_t dirs = directions(policy, c);
        for (int d = 0; d < 2; d++) {
            if (!((dirs >> d) & 1u)) continue;
            uint64_t b;
            if (bin_of(ts[i], t0, w, n_bins, &b)) {
                count[d][b] += 1u;
                add_bytes(&bsum[d][b], bytes[i]);
            } else {
                stats[4 + d] += 1;
            }
        }
    }
}

/*
 * Classification plus histogram over a record stream (the whole hot path),
 * processed in chunks so the class array stays small. Accumulates like
 * oracle_histogram.
 */
int oracle_discriminate_histogram(const uint32_t *net, const uint8_t *len, uint32_t n_entries,
                                  const uint64_t *ts, const uint32_t *src, const uint32_t *dst,
                                  const uint32_t *bytes, uint64_t n, uint64_t t0, uint64_t w,
                                  uint64_t n_bins, const uint8_t *policy, uint32_t *count0,
                                  uint32_t *count1, uint64_t *bytes0, uint64_t *bytes1,
                                  uint64_t *stats) {
    const uint64_t chunk = 1u << 22;
    uint8_t *cls = (uint8_t *)malloc(chunk);
    if (!cls) return -1;
    for (uint64_t s = 0; s < n; s += chunk) {
        uint64_t m = n - s < chunk ? n - s : chunk;
        oracle_classify(net, len, n_entries, src + s, dst + s, m, cls);
        oracle_histogram(ts + s, bytes + s, cls, m, t0, w, n_bins, policy, count0, count1, bytes0,
                         bytes1, stats);
    }
    free(cls);
    return 0;
}

/*
 * Classification plus histogram of the records whose src or dst is in the
 * watch list (membership as above, against the second list); every other
 * record only adds one to stats[6]. Accumulates like oracle_histogram.
 */
int oracle_discriminate_histogram_watch(const uint32_t *net, const uint8_t *len, uint32_t n_entries,
                                        const uint32_t *wnet, const uint8_t *wlen, uint32_t w_entries,
                                        const uint64_t *ts, const uint32_t *src, const uint32_t *dst,
                                        const uint32_t *bytes, uint64_t n, uint64_t t0, uint64_t w,
                                        uint64_t n_bins, const uint8_t *policy, uint32_t *count0,
                                        uint32_t *count1, uint64_t *bytes0, uint64_t *bytes1,
                                        uint64_t *stats) {
    const uint64_t chunk = 1u << 22;
    uint8_t *cls = (uint8_t *)malloc(chunk);
    uint8_t *wcls = (uint8_t *)malloc(chunk);
    if (!cls || !wcls) {
        free(cls);
        free(wcls);
        return -1;
    }
    for (uint64_t s = 0; s < n; s += chunk) {
        uint64_t m = n - s < chunk ? n - s : chunk;
        oracle_classify(wnet, wlen, w_entries, src + s, dst + s, m, wcls);
        oracle_classify(net, len, n_entries, src + s, dst + s, m, cls);
        for (uint64_t i = 0; i < m; i++) {
            if (wcls[i] == 0) {
                stats[6] += 1;
                continue;
            }
            oracle_histogram(ts + s + i, bytes + s + i, cls + i, 1, t0, w, n_bins, policy, count0, count1,
                             bytes0, bytes1, stats);
        }
    }
    free(cls);
    free(wcls);
    return 0;
}

/*
 * The same histogram, restricted to a sorted list of bins `keep[0..m)`
 * (each < n_bins): out_count[d * m + j] and out_bytes[d * m + j] receive the
 * full-workload values of bin keep[j]. Records in other bins are skipped
 * before classification, so this answers sampled bins of a large workload.
 * Accumulates into the caller's arrays. Parallel over records.
 */
void oracle_histogram_bins(const uint32_t *net, const uint8_t *len, uint32_t n_entries,
                           const uint64_t *ts, const uint32_t *src, const uint32_t *dst,
                           const uint32_t *bytes, uint64_t n, uint64_t t0, uint64_t w,
                           uint64_t n_bins, const uint8_t *policy, const uint64_t *keep, uint64_t m,
                           uint32_t *out_count, uint64_t *out_bytes) {
#pragma omp parallel
    {
        uint32_t *lc = (uint32_t *)calloc(2 * m + 1, sizeof(uint32_t));
        uint64_t *lb = (uint64_t *)calloc(2 * m + 1, sizeof(uint64_t));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < (int64_t)n; i++) {
            uint64_t b;
            if (!bin_of(ts[i], t0, w, n_bins, &b)) continue;
            uint64_t lo = 0, hi = m; /* binary search of b in keep */
            while (lo < hi) {
                uint64_t mid = (lo + hi) / 2;
                if (keep[mid] < b) lo = mid + 1; else hi = mid;
            }
            if (lo == m || keep[lo] != b) continue;
            uint8_t dirs = directions(policy, classify_one(src[i], dst[i], net, len, n_entries));
            for (int d = 0; d < 2; d++) {
                if (!((dirs >> d) & 1u)) continue;
                lc[d * m + lo] += 1u;
                add_bytes(&lb[d * m + lo], bytes[i]);
            }
        }
#pragma omp critical
        for (uint64_t j = 0; j < 2 * m; j++) {
            out_count[j] += lc[j];
            out_bytes[j] += lb[j];
        }
        free(lc);
        free(lb);
    }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int oracle_mutant(void) { return ORACLE_MUTANT; }
