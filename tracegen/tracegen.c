/*
 * tracegen.c - seeded synthetic memory-traffic traces.
 *
 * Input synthesis only: this file produces uint32 counter deltas (64-byte lines per
 * interval) and holds none of the control method's arithmetic.  Both the CPU oracle
 * and the CUDA replay path consume the buffers written here.
 *
 * Stream per trace: SplitMix64 seeds a xoshiro256** generator with
 * hash(seed, trace_id); the trace is a sequence of constant-demand phases.
 *   phase length  ~ geometric on {1, 2, ...} with mean m (success prob. 1/m)
 *   phase level   ~ U[level_lo, level_hi] GB/s
 *   per-interval  multiplicative noise exp(sigma * Z), Z ~ N(0,1) by Box-Muller
 *   delta         = clamp(llround(level * noise * dt * 1e9 / line_bytes), 0, 2^32 - 1)
 * Regime mixing (policy-sweep workload): the trace alternates regimes whose lengths are
 * geometric with mean regime_mean; each regime draws its phase mean from {m_a, m_b}
 * with probability 1/2 each.  A phase that would cross a regime boundary is cut there.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef struct {
    double mean_phase;      /* m (used when regime_mean <= 0) */
    double mean_phase_b;    /* second phase mean for regime mixing */
    double regime_mean;     /* > 0 enables regime mixing between mean_phase / mean_phase_b */
    double level_lo, level_hi; /* GB/s */
    double sigma;           /* lognormal noise sigma */
    double dt_s;            /* interval length, s */
    double line_bytes;      /* bytes per counted line */
} tg_params;

static uint64_t sm64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xs256;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xs_next(xs256 *g) {
    uint64_t *s = g->s;
    uint64_t r = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl64(s[3], 45);
    return r;
}

static void xs_seed(xs256 *g, uint64_t seed, uint64_t stream) {
    uint64_t x = seed ^ (0xd1b54a32d192ed03ULL * (stream + 1));
    for (int i = 0; i < 4; i++) g->s[i] = sm64_next(&x);
}

/* uniform in [0, 1) with 53 random bits */
static double xs_u01(xs256 *g) { return (double)(xs_next(g) >> 11) * 0x1.0p-53; }

/* geometric on {1, 2, ...} with the given mean (>= 1) */
static uint64_t xs_geom(xs256 *g, double mean) {
    if (mean <= 1.0) return 1;
    double p = 1.0 / mean;
    double u = 1.0 - xs_u01(g);              /* (0, 1] */
    double k = floor(log(u) / log1p(-p));
    if (k > 1e15) k = 1e15;
    return 1 + (uint64_t)k;
}

static double xs_normal(xs256 *g) {
    double u1 = 1.0 - xs_u01(g);             /* (0, 1] */
    double u2 = xs_u01(g);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Fill out[0..n) for one trace. */
void tg_trace(const tg_params *p, uint64_t seed, uint64_t trace_id, uint32_t *out, uint64_t n) {
    xs256 g;
    xs_seed(&g, seed, trace_id);
    const double scale = p->dt_s * 1e9 / p->line_bytes;
    uint64_t t = 0;
    uint64_t regime_left = 0;
    double cur_mean = p->mean_phase;
    while (t < n) {
        if (p->regime_mean > 0.0 && regime_left == 0) {
            regime_left = xs_geom(&g, p->regime_mean);
            cur_mean = (xs_u01(&g) < 0.5) ? p->mean_phase : p->mean_phase_b;
        }
        uint64_t len = xs_geom(&g, cur_mean);
        if (p->regime_mean > 0.0 && len > regime_left) len = regime_left;
        double level = p->level_lo + (p->level_hi - p->level_lo) * xs_u01(&g);
        for (uint64_t k = 0; k < len && t < n; k++, t++) {
            double v = level * exp(p->sigma * xs_normal(&g)) * scale;
            double r = nearbyint(v);
            if (!(r > 0.0)) r = 0.0;
            if (r > 4294967295.0) r = 4294967295.0;
            out[t] = (uint32_t)r;
        }
        if (p->regime_mean > 0.0) regime_left -= len;
    }
}

/* Many traces: trace i gets ids[i] (usually i) and is written at out + offsets[i]. */
void tg_traces(const tg_params *p, uint64_t seed, const uint64_t *ids, const uint64_t *lengths,
               const uint64_t *offsets, uint64_t n_traces, uint32_t *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < (int64_t)n_traces; i++)
        tg_trace(p, seed, ids[i], out + offsets[i], lengths[i]);
}

/* Lengths log-uniform in [lo, hi] (rounded to the nearest integer), one stream. */
void tg_lengths_loguniform(uint64_t seed, uint64_t n, double lo, double hi, uint64_t *out) {
    xs256 g;
    xs_seed(&g, seed, 0xffffffffULL);
    double a = log(lo), b = log(hi);
    for (uint64_t i = 0; i < n; i++) {
        double v = nearbyint(exp(a + (b - a) * xs_u01(&g)));
        if (v < lo) v = lo;
        if (v > hi) v = hi;
        out[i] = (uint64_t)v;
    }
}

/* Poisson arrivals / uniform stream ids / log-uniform request sizes (serving workload). */
void tg_requests(uint64_t seed, uint64_t n_req, double rate_per_s, uint64_t n_streams,
                 double size_lo, double size_hi, double *arrival_s, uint32_t *stream_id,
                 uint32_t *size) {
    xs256 g;
    xs_seed(&g, seed, 0xfffffffeULL);
    double t = 0.0, a = log(size_lo), b = log(size_hi);
    for (uint64_t i = 0; i < n_req; i++) {
        t += -log(1.0 - xs_u01(&g)) / rate_per_s;
        arrival_s[i] = t;
        stream_id[i] = (uint32_t)(xs_next(&g) % n_streams);
        double v = nearbyint(exp(a + (b - a) * xs_u01(&g)));
        if (v < size_lo) v = size_lo;
        if (v > size_hi) v = size_hi;
        size[i] = (uint32_t)v;
    }
}
