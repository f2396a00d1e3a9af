/*
 * Seeded synthetic input generators shared by the oracle tests, the GPU
 * parity tests and the benchmark.  This file holds no grouping arithmetic:
 * it only draws keys, values, timestamps and window sizes.
 *
 * Every draw is a pure function of (seed, stream, element index, attempt),
 * so the output does not depend on the number of host threads used.
 *
 * Random source: the SplitMix64 finaliser (Steele, Lea, Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014) applied to a
 * counter.  Zipf draws use rejection-inversion (Hormann and Derflinger,
 * "Rejection-inversion to generate variates from monotone discrete
 * distributions", ACM TOMACS 6(3), 1996).  Normal draws use Box-Muller.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t sm64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* one 64-bit draw for (seed, stream, index, attempt) */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t i, uint64_t j) {
    uint64_t base = sm64(seed ^ sm64(stream * 0xA24BAED4963EE407ull));
    return sm64(base ^ (i * 0xD1B54A32D192ED03ull + j * 0x8CB92BA72F3D8DD7ull));
}

/* uniform in [0, 1) with 53 random bits */
static inline double unif01(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }
/* uniform in (0, 1] */
static inline double unif01_open0(uint64_t r) { return (double)((r >> 11) + 1) * 0x1.0p-53; }

/* ---------------- threading ---------------- */
typedef void (*range_fn)(void* ctx, uint64_t lo, uint64_t hi);
typedef struct { range_fn fn; void* ctx; uint64_t lo, hi; } job_t;
static void* run_job(void* p) { job_t* j = (job_t*)p; j->fn(j->ctx, j->lo, j->hi); return NULL; }

static void parallel_for(uint64_t n, int nthreads, range_fn fn, void* ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < 65536 || nthreads == 1) { fn(ctx, 0, n); return; }
    pthread_t th[256];
    job_t jobs[256];
    uint64_t chunk = (n + (uint64_t)nthreads - 1) / (uint64_t)nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t lo = (uint64_t)t * chunk, hi = lo + chunk;
        if (lo >= n) break;
        if (hi > n) hi = n;
        jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].lo = lo; jobs[t].hi = hi;
        if (pthread_create(&th[t], NULL, run_job, &jobs[t]) != 0) { fn(ctx, lo, hi); jobs[t].fn = NULL; }
        started = t + 1;
    }
    for (int t = 0; t < started; ++t) if (jobs[t].fn) pthread_join(th[t], NULL);
}

/* ---------------- uniform integers ---------------- */
typedef struct { uint64_t seed, stream, lo, span; void* out; int bytes; } unif_ctx;

static void unif_range(void* p, uint64_t a, uint64_t b) {
    unif_ctx* c = (unif_ctx*)p;
    for (uint64_t i = a; i < b; ++i) {
        uint64_t r = draw(c->seed, c->stream, i, 0);
        /* span == 0 means the full 64-bit range */
        uint64_t v = c->span ? c->lo + (uint64_t)(((__uint128_t)r * c->span) >> 64) : r;
        if (c->bytes == 8) ((uint64_t*)c->out)[i] = v;
        else ((uint32_t*)c->out)[i] = (uint32_t)v;
    }
}

/* out[i] = lo + floor(r_i * span / 2^64); span == 0 draws the whole u64 range. */
void sbhgen_uniform(uint64_t seed, uint64_t stream, uint64_t n, uint64_t lo, uint64_t span,
                    void* out, int bytes, int nthreads) {
    unif_ctx c = {seed, stream, lo, span, out, bytes};
    parallel_for(n, nthreads, unif_range, &c);
}

/* ---------------- Zipf by rejection-inversion ---------------- */
typedef struct {
    double s, n, hx1, hn, sconst;
} zipf_t;

/* expm1(t)/t and log1p(t)/t with their limits at t = 0 */
static double hlp_expm1_over(double t) { return fabs(t) > 1e-8 ? expm1(t) / t : 1.0 + t * 0.5 + t * t / 6.0; }
static double hlp_log1p_over(double t) { return fabs(t) > 1e-8 ? log1p(t) / t : 1.0 - t * 0.5 + t * t / 3.0; }

static double zh(const zipf_t* z, double x) { return exp(-z->s * log(x)); }           /* x^-s */
static double zH(const zipf_t* z, double x) {                                         /* integral of x^-s from 1 */
    double lx = log(x);
    return hlp_expm1_over((1.0 - z->s) * lx) * lx;
}
static double zHinv(const zipf_t* z, double u) {
    double t = u * (1.0 - z->s);
    if (t < -1.0) t = -1.0;
    return exp(hlp_log1p_over(t) * u);
}

static void zipf_init(zipf_t* z, double s, uint64_t n) {
    z->s = s; z->n = (double)n;
    z->hx1 = zH(z, 1.5) - 1.0;
    z->hn = zH(z, z->n + 0.5);
    z->sconst = 2.0 - zHinv(z, zH(z, 2.5) - zh(z, 2.0));
}

/* One Zipf(s) rank in [1, n] for element i; attempts use draw index j. */
static uint64_t zipf_draw(const zipf_t* z, uint64_t seed, uint64_t stream, uint64_t i) {
    for (uint64_t j = 0;; ++j) {
        double u = z->hn + unif01(draw(seed, stream, i, j)) * (z->hx1 - z->hn);
        double x = zHinv(z, u);
        double kd = floor(x + 0.5);
        if (kd < 1.0) kd = 1.0;
        if (kd > z->n) kd = z->n;
        if (kd - x <= z->sconst || u >= zH(z, kd + 0.5) - zh(z, kd)) return (uint64_t)kd;
    }
}

/* ---------------- lognormal ---------------- */
static double normal_draw(uint64_t seed, uint64_t stream, uint64_t i, uint64_t j) {
    double u1 = unif01_open0(draw(seed, stream, i, 2 * j));
    double u2 = unif01(draw(seed, stream, i, 2 * j + 1));
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

/* floor(exp(mu + sigma z)), redrawn until it is below 2^64 */
static uint64_t lognormal_u64(double mu, double sigma, uint64_t seed, uint64_t stream, uint64_t i) {
    for (uint64_t j = 0;; ++j) {
        double x = exp(mu + sigma * normal_draw(seed, stream, i, j));
        if (x < 18446744073709551616.0) return (uint64_t)x;
    }
}

/* ---------------- mixtures ---------------- */
typedef struct {
    uint64_t seed;
    double zipf_frac;
    zipf_t z;
    double mu, sigma;
    int hashed;  /* Zipf ranks passed through the bijection sm64 */
    uint64_t* out;
} mix_ctx;

enum { ST_SELECT = 11, ST_ZIPF = 12, ST_LOGN = 13 };

static void mix_range(void* p, uint64_t a, uint64_t b) {
    mix_ctx* c = (mix_ctx*)p;
    for (uint64_t i = a; i < b; ++i) {
        double sel = unif01(draw(c->seed, ST_SELECT, i, 0));
        if (sel < c->zipf_frac) {
            const uint64_t r = zipf_draw(&c->z, c->seed, ST_ZIPF, i);
            c->out[i] = c->hashed ? sm64(r) : r;
        } else {
            c->out[i] = lognormal_u64(c->mu, c->sigma, c->seed, ST_LOGN, i);
        }
    }
}

/* Mixture of Zipf(s) ranks over [1, zipf_n] (weight zipf_frac) and
 * floor(lognormal(mu, sigma)) below 2^64 (weight 1 - zipf_frac).  With hashed,
 * a Zipf rank r becomes sm64(r) (a bijection of the 64-bit words: the same
 * multiplicities, spread over the whole key range). */
void sbhgen_zipf_lognormal_mix(uint64_t seed, uint64_t n, double zipf_frac, double s, uint64_t zipf_n,
                               double mu, double sigma, uint64_t* out, int nthreads, int hashed) {
    mix_ctx c;
    c.seed = seed; c.zipf_frac = zipf_frac; c.mu = mu; c.sigma = sigma; c.out = out; c.hashed = hashed;
    zipf_init(&c.z, s, zipf_n);
    parallel_for(n, nthreads, mix_range, &c);
}

typedef struct { uint64_t seed, stream; zipf_t z; uint64_t* out; } zipf_ctx;
static void zipf_range(void* p, uint64_t a, uint64_t b) {
    zipf_ctx* c = (zipf_ctx*)p;
    for (uint64_t i = a; i < b; ++i) c->out[i] = zipf_draw(&c->z, c->seed, c->stream, i);
}

/* Zipf(s) ranks in [1, zipf_n]. */
void sbhgen_zipf(uint64_t seed, uint64_t stream, uint64_t n, double s, uint64_t zipf_n, uint64_t* out, int nthreads) {
    zipf_ctx c;
    c.seed = seed; c.stream = stream; c.out = out;
    zipf_init(&c.z, s, zipf_n);
    parallel_for(n, nthreads, zipf_range, &c);
}

/* Integer lognormal sizes: clamp(floor(exp(mu + sigma z)), lo, hi). */
void sbhgen_lognormal_sizes(uint64_t seed, uint64_t stream, uint64_t n, double mu, double sigma,
                            uint64_t lo, uint64_t hi, uint64_t* out) {
    for (uint64_t i = 0; i < n; ++i) {
        double x = floor(exp(mu + sigma * normal_draw(seed, stream, i, 0)));
        uint64_t v = x < (double)lo ? lo : (x > (double)hi ? hi : (uint64_t)x);
        out[i] = v;
    }
}

/* Raw draws, exported so the tests can check the generator's distributions. */
void sbhgen_unif01(uint64_t seed, uint64_t stream, uint64_t n, double* out) {
    for (uint64_t i = 0; i < n; ++i) out[i] = unif01(draw(seed, stream, i, 0));
}
