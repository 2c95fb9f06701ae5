/*
 * Seeded synthetic inputs: CIDR prefix tables and IPv4 session records.
 *
 * This module shapes inputs only. It never decides whether an address is
 * inside a table (no mask/compare membership test), never bins, never counts:
 * both the CPU oracle and the CUDA path consume its buffers, and neither takes
 * an expected value from it.
 *
 * Every draw is counter based: value = splitmix64 finaliser applied to
 * (per-stream key + golden-ratio step * (index + 1)), so any sub-range of a
 * workload can be regenerated on its own and the bytes do not depend on how
 * the work is split across threads.
 *
 * Shapes (after the paper's workloads: Table 1 fields capture_time, source_ip,
 * destination_ip and bytes; Table 2's 1.3-1.6 billion sessions per day; the
 * diurnal pattern of its Figs. 6-7):
 *   - class mix: a record's intended class (neither / src inside / dst inside /
 *     both) is drawn first with caller-given probabilities;
 *   - inside address: a table prefix (uniform, or a Zipf-ranked host pool) with
 *     uniform host bits;
 *   - outside address: first octet drawn from the octets that no table prefix
 *     starts with, lower 24 bits uniform; table prefixes all have length >= 8,
 *     so such an address lies outside every prefix by construction;
 *   - bytes: min(floor(exp(N(mu, sigma))), 2^32 - 1);
 *   - timestamps: uniform, diurnal sorted with jitter, or Zipf-ranked bins
 *     under an affine permutation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define GEN_PI 3.14159265358979323846

static inline uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xbf58476d1ce4e5b9ULL;
    z ^= z >> 27;
    z *= 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return z;
}

/* Key of stream `s` under `seed`. */
static inline uint64_t stream_key(uint64_t seed, uint64_t s) {
    return mix64(seed ^ mix64(0x2545F4914F6CDD1DULL + s * 0xD1B54A32D192ED03ULL));
}

/* Draw number i of a stream. */
static inline uint64_t draw(uint64_t key, uint64_t i) {
    return mix64(key + 0x9E3779B97F4A7C15ULL * (i + 1));
}

/* Uniform in [0, 1). */
static inline double unit(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

/* Uniform integer in [0, n) (multiply-shift; n >= 1). */
static inline uint64_t below(uint64_t x, uint64_t n) {
    return (uint64_t)(((unsigned __int128)x * n) >> 64);
}

enum {
    S_CLASS = 1, S_SRC_PICK, S_SRC_HOST, S_DST_PICK, S_DST_HOST, S_TS, S_TS2,
    S_BYTES1, S_BYTES2, S_JITTER, S_TABLE_LEN, S_TABLE_NET, S_POOL_IN_PICK,
    S_POOL_IN_HOST, S_POOL_OUT, S_ZIPF_SRC, S_ZIPF_DST, S_ZIPF_TS, S_PERM
};

/* ------------------------------------------------------------------------ */
/* Zipf(s) over {1..n} by rejection-inversion (Hoermann & Derflinger, 1996,
 * "Rejection-inversion to generate variates from monotone discrete
 * distributions"), s > 0, s != 1.                                           */

typedef struct {
    double s, hx1, hn, sconst;
    uint64_t n;
} zipf_t;

static double zh(double s, double x) { return exp(-s * log(x)); }            /* x^-s */
static double zH(double s, double x) {                                         /* int x^-s */
    double lx = log(x), y = (1.0 - s) * lx;
    double r = fabs(y) > 1e-8 ? expm1(y) / y : 1.0 + 0.5 * y;
    return r * lx;
}
static double zHinv(double s, double v) {
    double y = (1.0 - s) * v;
    double r = fabs(y) > 1e-8 ? log1p(y) / y : 1.0 - 0.5 * y;
    return exp(r * v);
}
static zipf_t zipf_init(double s, uint64_t n) {
    zipf_t z;
    z.s = s;
    z.n = n;
    z.hx1 = zH(s, 1.5) - 1.0;
    z.hn = zH(s, (double)n + 0.5);
    z.sconst = 2.0 - zHinv(s, zH(s, 2.5) - zh(s, 2.0));
    return z;
}
/* Rank in [1, n]; attempt a uses draw (i * 64 + a) of the stream. */
static uint64_t zipf_draw(const zipf_t *z, uint64_t key, uint64_t i) {
    for (uint64_t a = 0; a < 64; a++) {
        double u = z->hn + unit(draw(key, i * 64 + a)) * (z->hx1 - z->hn);
        double x = zHinv(z->s, u);
        double kd = floor(x + 0.5);
        if (kd < 1.0) kd = 1.0;
        if (kd > (double)z->n) kd = (double)z->n;
        if (kd - x <= z->sconst || u >= zH(z->s, kd + 0.5) - zh(z->s, kd)) return (uint64_t)kd;
    }
    return 1;
}

uint64_t gen_zipf(double s, uint64_t n, uint64_t seed, uint64_t first, uint64_t count, uint64_t *out) {
    zipf_t z = zipf_init(s, n);
    uint64_t key = stream_key(seed, S_ZIPF_TS);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)count; i++) out[i] = zipf_draw(&z, key, first + (uint64_t)i);
    return count;
}

/* ------------------------------------------------------------------------ */
/* Tables. */

/* Prefix lengths: uniform in [len_lo, len_hi]; with weighted != 0, lengths
 * 16..24 carry weight 4 and the others weight 1. Networks lie inside
 * 0.0.0.0/1 with their host bits cleared. Requires 8 <= len_lo <= len_hi <= 32. */
int gen_table(uint64_t seed, uint32_t n, uint32_t len_lo, uint32_t len_hi, int weighted,
              uint32_t *net, uint8_t *len) {
    if (len_lo < 8 || len_hi > 32 || len_lo > len_hi) return -1;
    double w[33] = {0}, tot = 0;
    for (uint32_t l = len_lo; l <= len_hi; l++) {
        w[l] = (weighted && l >= 16 && l <= 24) ? 4.0 : 1.0;
        tot += w[l];
    }
    uint64_t kl = stream_key(seed, S_TABLE_LEN), kn = stream_key(seed, S_TABLE_NET);
    for (uint32_t p = 0; p < n; p++) {
        double u = unit(draw(kl, p)) * tot, acc = 0;
        uint32_t l = len_hi;
        for (uint32_t c = len_lo; c <= len_hi; c++) {
            acc += w[c];
            if (u < acc) { l = c; break; }
        }
        uint32_t r = (uint32_t)(draw(kn, p) >> 32) & 0x7FFFFFFFu;
        uint32_t keep = 32 - l;                       /* host-bit count, <= 24 */
        net[p] = keep ? (r >> keep) << keep : r;
        len[p] = (uint8_t)l;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Records. */

typedef struct {
    uint64_t seed;
    uint64_t n_total;      /* records in the whole workload (for sorted kinds) */
    double   class_p[4];   /* P(neither), P(src inside), P(dst inside), P(both) */
    double   bytes_mu, bytes_sigma;
    int32_t  ts_kind;      /* 0 uniform [t_lo,t_hi); 1 diurnal sorted + jitter; 2 Zipf bins */
    int32_t  host_kind;    /* 0 prefix + uniform host bits; 1 Zipf over host pools */
    uint64_t t_lo, t_hi;   /* uniform range; diurnal day = [t_lo, t_hi) */
    uint64_t jitter;       /* +-jitter ms on the diurnal kind */
    double   peak_frac;    /* diurnal peak position as a fraction of the day */
    double   zipf_s;       /* Zipf exponent for ts bins and host ranks */
    uint64_t zipf_bins;    /* bins for the Zipf ts kind */
    uint64_t zipf_w;       /* bin width (ms) for the Zipf ts kind */
    uint32_t pool_size;    /* hosts per pool (inside and outside) */
    uint32_t reserved;
} gen_params;

/* Diurnal rate r(t) ~ 2 + cos(2 pi (t - tp) / D): cumulative fraction F(t). */
static double diurnal_F(double t, double D, double tp) {
    double c = D / (2.0 * GEN_PI);
    return (2.0 * t + c * (sin(2.0 * GEN_PI * (t - tp) / D) + sin(2.0 * GEN_PI * tp / D))) / (2.0 * D);
}
static double diurnal_f(double t, double D, double tp) {
    return (2.0 + cos(2.0 * GEN_PI * (t - tp) / D)) / (2.0 * D);
}
#define DI_KNOTS 65536
static void diurnal_knots(double D, double tp, double *knot) {
    /* knot[j] = F^-1(j / DI_KNOTS), by bisection to full precision */
    for (int j = 0; j <= DI_KNOTS; j++) {
        double u = (double)j / DI_KNOTS, lo = 0, hi = D;
        for (int it = 0; it < 80; it++) {
            double mid = 0.5 * (lo + hi);
            if (diurnal_F(mid, D, tp) < u) lo = mid; else hi = mid;
        }
        knot[j] = 0.5 * (lo + hi);
    }
}
static double diurnal_inv(double u, double D, double tp, const double *knot) {
    double x = u * DI_KNOTS;
    int j = (int)x;
    if (j >= DI_KNOTS) j = DI_KNOTS - 1;
    double t = knot[j] + (x - j) * (knot[j + 1] - knot[j]);
    for (int it = 0; it < 1; it++) {          /* fixed Newton steps: same result for any split */
        t -= (diurnal_F(t, D, tp) - u) / diurnal_f(t, D, tp);
        if (t < 0) t = 0;
        if (t > D) t = D;
    }
    return t;
}

static inline uint32_t host_bits(uint64_t x, uint32_t len) {
    uint32_t k = 32 - len;                     /* number of host bits, <= 24 here */
    uint32_t r = (uint32_t)(x >> 32);
    return k ? (r & ((1u << k) - 1u)) : 0u;
}

typedef struct {
    const uint32_t *net;
    const uint8_t *len;
    uint32_t P;
    uint8_t free_octet[256];
    uint32_t n_free;
} addr_ctx;

static inline uint32_t inside_addr(const addr_ctx *a, uint64_t xpick, uint64_t xhost) {
    uint32_t p = (uint32_t)below(xpick, a->P);
    return a->net[p] | host_bits(xhost, a->len[p]);
}
static inline uint32_t outside_addr(const addr_ctx *a, uint64_t x) {
    uint32_t o = a->free_octet[below(x, a->n_free)];
    return (o << 24) | ((uint32_t)x & 0xFFFFFFu);
}

/*
 * Fill records [first, first + n) of a workload. Outputs may be NULL to skip
 * a field; intended_class (optional) receives the construction class
 * (bit0 = src drawn inside, bit1 = dst drawn inside).
 * Returns 0, or -1 on a bad argument (a prefix shorter than /8, no free first
 * octet, empty table while inside addresses are requested).
 */
int gen_records(const gen_params *g, const uint32_t *net, const uint8_t *len, uint32_t P,
                uint64_t first, uint64_t n, uint64_t *ts, uint32_t *src, uint32_t *dst,
                uint32_t *bytes, uint8_t *intended_class) {
    addr_ctx a;
    a.net = net;
    a.len = len;
    a.P = P;
    uint8_t used[256];
    memset(used, 0, sizeof used);
    for (uint32_t p = 0; p < P; p++) {
        if (len[p] < 8 || len[p] > 32) return -1;
        used[net[p] >> 24] = 1;
    }
    a.n_free = 0;
    for (int o = 0; o < 256; o++)
        if (!used[o]) a.free_octet[a.n_free++] = (uint8_t)o;
    if (a.n_free == 0) return -1;
    int need_inside = g->class_p[1] > 0 || g->class_p[2] > 0 || g->class_p[3] > 0;
    if (need_inside && P == 0) return -1;

    const uint64_t seed = g->seed;
    const uint64_t kc = stream_key(seed, S_CLASS), ksp = stream_key(seed, S_SRC_PICK),
                   ksh = stream_key(seed, S_SRC_HOST), kdp = stream_key(seed, S_DST_PICK),
                   kdh = stream_key(seed, S_DST_HOST), kt = stream_key(seed, S_TS),
                   kt2 = stream_key(seed, S_TS2), kb1 = stream_key(seed, S_BYTES1),
                   kb2 = stream_key(seed, S_BYTES2), kj = stream_key(seed, S_JITTER),
                   kzs = stream_key(seed, S_ZIPF_SRC), kzd = stream_key(seed, S_ZIPF_DST),
                   kzt = stream_key(seed, S_ZIPF_TS);

    /* host pools for the Zipf host kind */
    uint32_t *pool_in = NULL, *pool_out = NULL;
    zipf_t zpool;
    if (g->host_kind == 1) {
        uint32_t m = g->pool_size ? g->pool_size : 1;
        pool_in = (uint32_t *)malloc(sizeof(uint32_t) * m);
        pool_out = (uint32_t *)malloc(sizeof(uint32_t) * m);
        if (!pool_in || !pool_out) { free(pool_in); free(pool_out); return -1; }
        uint64_t kpp = stream_key(seed, S_POOL_IN_PICK), kph = stream_key(seed, S_POOL_IN_HOST),
                 kpo = stream_key(seed, S_POOL_OUT);
        for (uint32_t h = 0; h < m; h++) {
            pool_in[h] = P ? inside_addr(&a, draw(kpp, h), draw(kph, h)) : 0;
            pool_out[h] = outside_addr(&a, draw(kpo, h));
        }
        zpool = zipf_init(g->zipf_s, m);
    }

    /* timestamp machinery */
    double *knot = NULL;
    double D = (double)(g->t_hi - g->t_lo), tp = g->peak_frac * D;
    if (g->ts_kind == 1) {
        knot = (double *)malloc(sizeof(double) * (DI_KNOTS + 1));
        if (!knot) { free(pool_in); free(pool_out); return -1; }
        diurnal_knots(D, tp, knot);
    }
    zipf_t zts;
    uint64_t perm_a = 1, perm_b = 0;
    if (g->ts_kind == 2) {
        zts = zipf_init(g->zipf_s, g->zipf_bins);
        /* affine permutation of ranks onto bins: multiplier coprime to the bin count */
        uint64_t nb = g->zipf_bins;
        perm_a = 1000003ULL % nb;
        for (;;) {
            uint64_t x = perm_a, y = nb;
            while (y) { uint64_t t = x % y; x = y; y = t; }
            if (x == 1 || nb == 1) break;
            perm_a = (perm_a + 1) % nb;
        }
        perm_b = below(draw(stream_key(seed, S_PERM), 0), nb);
    }

    const double c1 = g->class_p[0], c2 = c1 + g->class_p[1], c3 = c2 + g->class_p[2];
    const uint64_t span = g->t_hi - g->t_lo;

#pragma omp parallel for schedule(static)
    for (int64_t ii = 0; ii < (int64_t)n; ii++) {
        const uint64_t i = first + (uint64_t)ii;
        double u = unit(draw(kc, i));
        uint32_t cls = u < c1 ? 0u : u < c2 ? 1u : u < c3 ? 2u : 3u;
        uint32_t s, d;
        if (g->host_kind == 1) {
            uint64_t rs = zipf_draw(&zpool, kzs, i) - 1, rd = zipf_draw(&zpool, kzd, i) - 1;
            s = (cls & 1u) ? pool_in[rs] : pool_out[rs];
            d = (cls & 2u) ? pool_in[rd] : pool_out[rd];
        } else {
            s = (cls & 1u) ? inside_addr(&a, draw(ksp, i), draw(ksh, i)) : outside_addr(&a, draw(ksh, i));
            d = (cls & 2u) ? inside_addr(&a, draw(kdp, i), draw(kdh, i)) : outside_addr(&a, draw(kdh, i));
        }
        uint64_t t;
        if (g->ts_kind == 0) {
            t = g->t_lo + below(draw(kt, i), span);
        } else if (g->ts_kind == 1) {
            double q = ((double)i + 0.5) / (double)g->n_total;
            double base = floor(diurnal_inv(q, D, tp, knot));
            int64_t j = (int64_t)below(draw(kj, i), 2 * g->jitter + 1) - (int64_t)g->jitter;
            int64_t v = (int64_t)base + j;
            if (v < 0) v = 0;
            if (v > (int64_t)span - 1) v = (int64_t)span - 1;
            t = g->t_lo + (uint64_t)v;
        } else {
            uint64_t r = zipf_draw(&zts, kzt, i) - 1;
            uint64_t bin = (uint64_t)(((unsigned __int128)perm_a * r + perm_b) % g->zipf_bins);
            t = g->t_lo + bin * g->zipf_w + below(draw(kt2, i), g->zipf_w);
        }
        double u1 = ((double)(draw(kb1, i) >> 11) + 1.0) * 0x1.0p-53;   /* (0, 1] */
        double u2 = unit(draw(kb2, i));
        double z = sqrt(-2.0 * log(u1)) * cos(2.0 * GEN_PI * u2);
        double v = exp(g->bytes_mu + g->bytes_sigma * z);
        uint32_t b = v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
        if (ts) ts[ii] = t;
        if (src) src[ii] = s;
        if (dst) dst[ii] = d;
        if (bytes) bytes[ii] = b;
        if (intended_class) intended_class[ii] = (uint8_t)cls;
    }
    free(knot);
    free(pool_in);
    free(pool_out);
    return 0;
}

/* Uniform u64 words of a stream (slice sizes, windows and the like). */
void gen_u64(uint64_t seed, uint64_t stream, uint64_t first, uint64_t n, uint64_t *out) {
    uint64_t k = stream_key(seed, 1000 + stream);
    for (uint64_t i = 0; i < n; i++) out[i] = draw(k, first + i);
}

int gen_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
