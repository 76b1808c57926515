/*
 * Seeded synthetic inputs for the HashGraph build/probe workloads.
 *
 * This file holds only random-number generation and the recipes that turn
 * random numbers into key and query arrays.  It contains none of the hash
 * table's arithmetic (no hashing of keys, no bucket computation, no
 * counting): both the CUDA path and the CPU oracle are fed from here and
 * neither shares anything else.
 *
 * Random source: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used in counter form so any
 * element can be generated independently and the arrays can be filled by
 * several threads with identical results:
 *     out(state, i) = mix(state + (i + 1) * 0x9E3779B97F4A7C15)
 * where mix is the SplitMix64 output function.  A per-purpose stream state is
 * stream(master, id) = mix(master ^ (id * 0x9E3779B97F4A7C15)).
 *
 * Floating point appears only in the Zipf table (sequential double sums of
 * 1/r) and in the uniform-to-rank comparison; the file is compiled with
 * -ffp-contract=off so x86-64 and aarch64 produce identical arrays.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#define HGW_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* i-th output (0-based) of the SplitMix64 sequence whose state starts at `state`. */
static inline uint64_t sm64_at(uint64_t state, uint64_t i) {
    return sm64_mix(state + (i + 1) * HGW_GAMMA);
}

uint64_t hgw_splitmix64_at(uint64_t state, uint64_t i) { return sm64_at(state, i); }

uint64_t hgw_stream(uint64_t master, uint64_t id) { return sm64_mix(master ^ (id * HGW_GAMMA)); }

/* Uniform integer in [0, range) from the high 32 bits of x (range <= 2^32). */
static inline uint64_t pick32(uint64_t x32, uint64_t range) { return (x32 * range) >> 32; }

/* ------------------------------------------------------------------ */
/* A tiny fork-join helper: splits [0, n) into contiguous chunks.      */
/* ------------------------------------------------------------------ */
typedef void (*hgw_body)(void* ctx, uint64_t lo, uint64_t hi);
typedef struct { hgw_body fn; void* ctx; uint64_t lo, hi; } hgw_job;

static void* hgw_run(void* p) {
    hgw_job* j = (hgw_job*)p;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static int g_threads = 0;
void hgw_set_threads(int t) { g_threads = t; }

static void parallel_for(uint64_t n, hgw_body fn, void* ctx) {
    int t = g_threads;
    if (t <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        t = (c > 0) ? (int)c : 1;
    }
    if (t > 64) t = 64;
    if (n < (1u << 16) || t == 1) { fn(ctx, 0, n); return; }
    pthread_t th[64];
    hgw_job jobs[64];
    uint64_t chunk = (n + (uint64_t)t - 1) / (uint64_t)t;
    int started = 0;
    for (int k = 0; k < t; ++k) {
        uint64_t lo = (uint64_t)k * chunk, hi = lo + chunk;
        if (lo >= n) break;
        if (hi > n) hi = n;
        jobs[k].fn = fn; jobs[k].ctx = ctx; jobs[k].lo = lo; jobs[k].hi = hi;
        if (pthread_create(&th[k], NULL, hgw_run, &jobs[k]) != 0) { fn(ctx, lo, hi); jobs[k].fn = NULL; }
        started = k + 1;
    }
    for (int k = 0; k < started; ++k)
        if (jobs[k].fn) pthread_join(th[k], NULL);
}

/* ------------------------------------------------------------------ */
/* Uniform keys.                                                        */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t state; void* out; } uni_ctx;

static void uni32_body(void* p, uint64_t lo, uint64_t hi) {
    uni_ctx* c = (uni_ctx*)p;
    uint32_t* o = (uint32_t*)c->out;
    for (uint64_t i = lo; i < hi; ++i) o[i] = (uint32_t)(sm64_at(c->state, i) >> 32);
}
static void uni64_body(void* p, uint64_t lo, uint64_t hi) {
    uni_ctx* c = (uni_ctx*)p;
    uint64_t* o = (uint64_t*)c->out;
    for (uint64_t i = lo; i < hi; ++i) o[i] = sm64_at(c->state, i);
}

/* out[i] = high 32 bits of the i-th SplitMix64 output. */
void hgw_uniform_u32(uint64_t state, uint64_t n, uint32_t* out) {
    uni_ctx c = {state, out};
    parallel_for(n, uni32_body, &c);
}
/* out[i] = the i-th SplitMix64 output. */
void hgw_uniform_u64(uint64_t state, uint64_t n, uint64_t* out) {
    uni_ctx c = {state, out};
    parallel_for(n, uni64_body, &c);
}

/* ------------------------------------------------------------------ */
/* Hit/miss query mix over a key array.                                 */
/*   slot i: x = out(sel, i); hit iff (x >> 32) < hit_threshold;        */
/*   hit  -> keys[pick32(x & 0xffffffff, n)]                            */
/*   miss -> fresh uniform value out(miss, i) (high 32 bits for u32).   */
/* A miss may equal a key by chance; counts stay exact regardless.     */
/* ------------------------------------------------------------------ */
typedef struct {
    const void* keys; uint64_t n; uint64_t sel, miss; uint64_t thr; void* out;
} mix_ctx;

static void mix32_body(void* p, uint64_t lo, uint64_t hi) {
    mix_ctx* c = (mix_ctx*)p;
    const uint32_t* k = (const uint32_t*)c->keys;
    uint32_t* o = (uint32_t*)c->out;
    for (uint64_t i = lo; i < hi; ++i) {
        uint64_t x = sm64_at(c->sel, i);
        if (c->n > 0 && (x >> 32) < c->thr) o[i] = k[pick32(x & 0xffffffffULL, c->n)];
        else o[i] = (uint32_t)(sm64_at(c->miss, i) >> 32);
    }
}
static void mix64_body(void* p, uint64_t lo, uint64_t hi) {
    mix_ctx* c = (mix_ctx*)p;
    const uint64_t* k = (const uint64_t*)c->keys;
    uint64_t* o = (uint64_t*)c->out;
    for (uint64_t i = lo; i < hi; ++i) {
        uint64_t x = sm64_at(c->sel, i);
        if (c->n > 0 && (x >> 32) < c->thr) o[i] = k[pick32(x & 0xffffffffULL, c->n)];
        else o[i] = sm64_at(c->miss, i);
    }
}

void hgw_probe_mix_u32(const uint32_t* keys, uint64_t n, uint64_t sel, uint64_t miss,
                       uint64_t hit_threshold, uint64_t q, uint32_t* out) {
    mix_ctx c = {keys, n, sel, miss, hit_threshold, out};
    parallel_for(q, mix32_body, &c);
}
void hgw_probe_mix_u64(const uint64_t* keys, uint64_t n, uint64_t sel, uint64_t miss,
                       uint64_t hit_threshold, uint64_t q, uint64_t* out) {
    mix_ctx c = {keys, n, sel, miss, hit_threshold, out};
    parallel_for(q, mix64_body, &c);
}

/* ------------------------------------------------------------------ */
/* Zipf(s = 1) over ranks 1..M by inverse CDF.                         */
/*   S[0] = 0, S[r] = S[r-1] + 1.0 / r  (sequential double additions)  */
/*   u = (x >> 11) * 2^-53 in [0, 1), t = u * S[M],                     */
/*   rank = smallest r in [1, M] with S[r] > t.                         */
/* A guide table G[g] = rank(u = g / 2^GB) narrows each search: rank is */
/* nondecreasing in u, so a sample in [g, g+1) / 2^GB lies between      */
/* G[g] and G[g+1].                                                     */
/* Rank -> 32-bit value: v = r * 0x9E3779B1 mod 2^32 (odd multiplier,   */
/* so distinct ranks give distinct values).                             */
/* ------------------------------------------------------------------ */
#define ZIPF_GUIDE_BITS 20

static uint64_t zipf_search(const double* S, uint64_t lo, uint64_t hi, double t) {
    /* smallest r in [lo, hi] with S[r] > t; caller guarantees S[hi] > t or hi == M */
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (S[mid] > t) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* S must hold M + 1 doubles; G must hold 2^ZIPF_GUIDE_BITS + 1 entries. */
void hgw_zipf_table(uint64_t M, double* S, uint32_t* G) {
    S[0] = 0.0;
    for (uint64_t r = 1; r <= M; ++r) S[r] = S[r - 1] + 1.0 / (double)r;
    const uint64_t ng = 1ULL << ZIPF_GUIDE_BITS;
    for (uint64_t g = 0; g <= ng; ++g) {
        double u = (double)g * (1.0 / (double)ng);
        double t = u * S[M];
        G[g] = (uint32_t)zipf_search(S, 1, M, t);
    }
}

uint64_t hgw_zipf_guide_size(void) { return (1ULL << ZIPF_GUIDE_BITS) + 1; }

static inline uint64_t zipf_rank(const double* S, const uint32_t* G, uint64_t M, uint64_t x) {
    uint64_t m53 = x >> 11;
    double u = (double)m53 * (1.0 / 9007199254740992.0);
    double t = u * S[M];
    uint64_t g = m53 >> (53 - ZIPF_GUIDE_BITS);
    uint64_t lo = G[g], hi = G[g + 1];
    if (lo < 1) lo = 1;
    if (hi > M) hi = M;
    return zipf_search(S, lo, hi, t);
}

static inline uint32_t rank_value(uint64_t r) { return (uint32_t)(r * 0x9E3779B1ULL); }

typedef struct { const double* S; const uint32_t* G; uint64_t M; uint64_t state; uint32_t* out; } zipf_ctx;

static void zipf_body(void* p, uint64_t lo, uint64_t hi) {
    zipf_ctx* c = (zipf_ctx*)p;
    for (uint64_t i = lo; i < hi; ++i)
        c->out[i] = rank_value(zipf_rank(c->S, c->G, c->M, sm64_at(c->state, i)));
}

/* out[i] = value of a Zipf(1) rank over 1..M drawn from out(state, i). */
void hgw_zipf_values_u32(const double* S, const uint32_t* G, uint64_t M, uint64_t state,
                         uint64_t n, uint32_t* out) {
    zipf_ctx c = {S, G, M, state, out};
    parallel_for(n, zipf_body, &c);
}

/* Rank of one draw (for tests of the sampler). */
uint64_t hgw_zipf_rank_of(const double* S, const uint32_t* G, uint64_t M, uint64_t x) {
    return zipf_rank(S, G, M, x);
}

uint32_t hgw_rank_value(uint64_t r) { return rank_value(r); }

/* Queries over a Zipf key set: slot i, x = out(sel, i):
 *   hit iff (x >> 32) < hit_threshold: rank uniform in [1, M] -> value (present);
 *   miss: rank uniform in [M + 1, 2^32 - 1] from out(miss, i) -> value (absent,
 *   because the rank-to-value map is a bijection of 32-bit integers). */
typedef struct { uint64_t M, sel, miss, thr; uint32_t* out; } zq_ctx;

static void zq_body(void* p, uint64_t lo, uint64_t hi) {
    zq_ctx* c = (zq_ctx*)p;
    const uint64_t miss_span = 0xFFFFFFFFULL - c->M; /* ranks M+1 .. 2^32-1 */
    for (uint64_t i = lo; i < hi; ++i) {
        uint64_t x = sm64_at(c->sel, i);
        uint64_t r;
        if ((x >> 32) < c->thr) r = 1 + pick32(x & 0xffffffffULL, c->M);
        else r = c->M + 1 + pick32(sm64_at(c->miss, i) >> 32, miss_span);
        c->out[i] = rank_value(r);
    }
}

void hgw_zipf_queries_u32(uint64_t M, uint64_t sel, uint64_t miss, uint64_t hit_threshold,
                          uint64_t q, uint32_t* out) {
    zq_ctx c = {M, sel, miss, hit_threshold, out};
    parallel_for(q, zq_body, &c);
}

/* Zipf-weighted queries: as above, but a hit's rank follows the keys' own
 * Zipf(1) law, drawn from out(rank, i), so hot values are queried in
 * proportion to their multiplicity. */
typedef struct { const double* S; const uint32_t* G; uint64_t M, sel, miss, rank, thr; uint32_t* out; } zwq_ctx;

static void zwq_body(void* p, uint64_t lo, uint64_t hi) {
    zwq_ctx* c = (zwq_ctx*)p;
    const uint64_t miss_span = 0xFFFFFFFFULL - c->M;
    for (uint64_t i = lo; i < hi; ++i) {
        uint64_t x = sm64_at(c->sel, i);
        uint64_t r;
        if ((x >> 32) < c->thr) r = zipf_rank(c->S, c->G, c->M, sm64_at(c->rank, i));
        else r = c->M + 1 + pick32(sm64_at(c->miss, i) >> 32, miss_span);
        c->out[i] = rank_value(r);
    }
}

void hgw_zipf_weighted_queries_u32(const double* S, const uint32_t* G, uint64_t M, uint64_t sel,
                                   uint64_t miss, uint64_t rank, uint64_t hit_threshold,
                                   uint64_t q, uint32_t* out) {
    zwq_ctx c = {S, G, M, sel, miss, rank, hit_threshold, out};
    parallel_for(q, zwq_body, &c);
}

/* ------------------------------------------------------------------ */
/* Key-value join probe relation with a repeated hot subset.            */
/*   D distinct probe keys: H hot keys (each placed `rep` times) then    */
/*   the singles; distinct key j: x = out(sel, j); hit iff top bit set: */
/*   keys[pick32(x & 0xffffffff, n)], else out(miss, j).                 */
/*   Slots 0 .. rep*H-1 hold hot key s / rep; slot s >= rep*H holds     */
/*   single key H + (s - rep*H).  Then a Fisher-Yates shuffle with       */
/*   j = pick32(out(shuf, s) >> 32, s + 1) for s = q-1 .. 1.              */
/* ------------------------------------------------------------------ */
void hgw_join_probe_u64(const uint64_t* keys, uint64_t n, uint64_t sel, uint64_t miss,
                        uint64_t shuf, uint64_t q, uint64_t hot, uint64_t rep, uint64_t* out) {
    const uint64_t hot_slots = hot * rep;
    for (uint64_t s = 0; s < q; ++s) {
        uint64_t j = (s < hot_slots) ? (s / rep) : (hot + (s - hot_slots));
        uint64_t x = sm64_at(sel, j);
        if (n > 0 && (x >> 63)) out[s] = keys[pick32(x & 0xffffffffULL, n)];
        else out[s] = sm64_at(miss, j);
    }
    for (uint64_t s = q; s-- > 1;) {
        uint64_t j = pick32(sm64_at(shuf, s) >> 32, s + 1);
        uint64_t tmp = out[s]; out[s] = out[j]; out[j] = tmp;
    }
}
