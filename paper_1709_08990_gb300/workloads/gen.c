/*
 * Seeded synthetic workloads for the Stream VByte codec.
 *
 * This file holds random-number generation and value distributions only: no
 * byte lengths, control bytes, offsets or prefix sums of the codec.  Both the
 * CUDA path's tests and the oracle's tests take their inputs from here, so
 * the two sides always see the same integers.
 *
 * Generator: counter-based SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014).  Word i of stream s under
 * seed S is the first output of a SplitMix64 generator whose state is
 * S*2^40 + s*2^32 + i, i.e. mix(S*2^40 + s*2^32 + i + gamma).  Streams
 * s < 256 and indexes i < 2^32 never collide.  Because every word is a pure
 * function of its counter, any thread count gives the same arrays.
 *
 * Distributions (the posting-list structure of the paper's Sec. 5: sorted
 * document identifiers, gaps that are small for long lists):
 *   uniform_lengths : byte length L ~ U{1..4}, value ~ U[2^(8(L-1)), 2^(8L)),
 *                     [0, 256) for L = 1;
 *   skewed_lengths  : P(L) = (.50, .30, .15, .05), value uniform as above;
 *   sorted_geometric: x_i = start + sum_{j<=i} g_j, g_j i.i.d. geometric on
 *                     {1, 2, ...} with mean `mean` (p = 1/mean);
 *   list_lengths    : log-uniform on [lo, hi], then scaled down (largest
 *                     common factor, floor, clamped at lo) until the total
 *                     is at most `cap`;
 *   posting_list    : sorted ids in [0, 2^31), geometric gaps of mean
 *                     2^31/(m+1); a list that would reach 2^31 is redrawn
 *                     from the next stream.
 */
#include <math.h>
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define GAMMA 0x9e3779b97f4a7c15ull

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

uint64_t svbgen_word(uint64_t seed, uint32_t stream, uint64_t i)
{
    uint64_t ctr = (seed << 40) + ((uint64_t)stream << 32) + i;
    return mix64(ctr + GAMMA);
}

/* Uniform integer in [0, range) by the multiply-high method. */
static inline uint64_t bounded(uint64_t r, uint64_t range)
{
    return (uint64_t)(((unsigned __int128)r * range) >> 64);
}

/* Uniform double in (0, 1] from the top 53 bits. */
static inline double unit_open0(uint64_t r)
{
    return (double)((r >> 11) + 1) * (1.0 / 9007199254740992.0);
}

/* Geometric on {1, 2, ...} with success probability p, by inversion. */
static inline uint64_t geometric(uint64_t r, double log1mp)
{
    double g = floor(log(unit_open0(r)) / log1mp);
    if (g > 4.0e18)
        g = 4.0e18;
    return 1 + (uint64_t)g;
}

static uint32_t value_of_length(uint64_t r, unsigned len)
{
    uint64_t lo = (len == 1) ? 0 : (1ull << (8 * (len - 1)));
    uint64_t hi = 1ull << (8 * len);
    return (uint32_t)(lo + bounded(r, hi - lo));
}

/* ------------------------------------------------------------------ */
/* A tiny parallel-for over index ranges.                              */

typedef void (*range_fn)(void *ctx, size_t begin, size_t end);

struct range_job {
    range_fn fn;
    void *ctx;
    size_t begin, end;
};

static void *range_thread(void *p)
{
    struct range_job *j = (struct range_job *)p;
    j->fn(j->ctx, j->begin, j->end);
    return NULL;
}

static int thread_count(int requested)
{
    if (requested > 0)
        return requested;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    if (c < 1)
        c = 1;
    if (c > 64)
        c = 64;
    return (int)c;
}

static void parallel_for(size_t n, int nthreads, range_fn fn, void *ctx)
{
    nthreads = thread_count(nthreads);
    if (n < 65536 || nthreads == 1) {
        fn(ctx, 0, n);
        return;
    }
    if ((size_t)nthreads > n)
        nthreads = (int)n;
    pthread_t tid[64];
    struct range_job job[64];
    size_t chunk = (n + nthreads - 1) / nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; t++) {
        size_t b = (size_t)t * chunk, e = b + chunk;
        if (b >= n)
            break;
        if (e > n)
            e = n;
        job[t].fn = fn;
        job[t].ctx = ctx;
        job[t].begin = b;
        job[t].end = e;
        if (pthread_create(&tid[t], NULL, range_thread, &job[t]) != 0) {
            fn(ctx, b, e); /* run inline if a thread cannot start */
            job[t].fn = NULL;
        }
        started = t + 1;
    }
    for (int t = 0; t < started; t++)
        if (job[t].fn)
            pthread_join(tid[t], NULL);
}

/* ------------------------------------------------------------------ */
/* Independent values with a chosen byte-length mix.                   */

struct lengths_ctx {
    uint64_t seed;
    uint32_t *out;
    int skewed;
};

static void lengths_range(void *p, size_t b, size_t e)
{
    struct lengths_ctx *c = (struct lengths_ctx *)p;
    for (size_t i = b; i < e; i++) {
        uint64_t r0 = svbgen_word(c->seed, 0, i);
        unsigned len;
        if (c->skewed) {
            uint64_t u = bounded(r0, 100); /* .50 / .30 / .15 / .05 */
            len = u < 50 ? 1 : u < 80 ? 2 : u < 95 ? 3 : 4;
        } else {
            len = 1 + (unsigned)bounded(r0, 4);
        }
        c->out[i] = value_of_length(svbgen_word(c->seed, 1, i), len);
    }
}

void svbgen_uniform_lengths(uint64_t seed, size_t n, uint32_t *out, int nthreads)
{
    struct lengths_ctx c = {seed, out, 0};
    parallel_for(n, nthreads, lengths_range, &c);
}

void svbgen_skewed_lengths(uint64_t seed, size_t n, uint32_t *out, int nthreads)
{
    struct lengths_ctx c = {seed, out, 1};
    parallel_for(n, nthreads, lengths_range, &c);
}

/* ------------------------------------------------------------------ */
/* Sorted arrays from geometric gaps.                                  */

struct geo_ctx {
    uint64_t seed;
    uint32_t *out;
    double log1mp;
};

static void gaps_range(void *p, size_t b, size_t e)
{
    struct geo_ctx *c = (struct geo_ctx *)p;
    for (size_t i = b; i < e; i++)
        c->out[i] = (uint32_t)geometric(svbgen_word(c->seed, 0, i), c->log1mp);
}

/* Gaps first (in parallel), then a running sum (serial, mod 2^32). */
void svbgen_sorted_geometric(uint64_t seed, size_t n, double mean, uint32_t start,
                             uint32_t *out, int nthreads)
{
    struct geo_ctx c = {seed, out, log1p(-1.0 / mean)};
    parallel_for(n, nthreads, gaps_range, &c);
    uint32_t run = start;
    for (size_t i = 0; i < n; i++) {
        run += out[i];
        out[i] = run;
    }
}

/* ------------------------------------------------------------------ */
/* Posting lists of uneven lengths.                                    */

static uint64_t scaled_total(const double *raw, size_t k, double s, uint32_t lo)
{
    uint64_t t = 0;
    for (size_t j = 0; j < k; j++) {
        double m = floor(raw[j] * s);
        t += m < lo ? lo : (uint64_t)m;
    }
    return t;
}

/* Returns the realised total. */
uint64_t svbgen_list_lengths(uint64_t seed, size_t k, uint32_t lo, uint32_t hi,
                             uint64_t cap, uint32_t *len)
{
    double *raw = (double *)malloc(k * sizeof(double));
    if (!raw)
        return 0;
    double llo = log((double)lo), lhi = log((double)hi);
    double sum = 0.0;
    for (size_t j = 0; j < k; j++) {
        double u = (double)(svbgen_word(seed, 0, j) >> 11) * (1.0 / 9007199254740992.0);
        double m = floor(exp(llo + u * (lhi - llo)));
        if (m < lo)
            m = lo;
        if (m > hi)
            m = hi;
        raw[j] = m;
        sum += m;
    }
    double s = 1.0;
    if (cap > 0 && sum > (double)cap) {
        /* Largest s in (0, cap/sum] whose floored, clamped total fits. */
        double a = 0.0, b = (double)cap / sum;
        if (scaled_total(raw, k, b, lo) <= cap) {
            s = b;
        } else {
            for (int it = 0; it < 200; it++) {
                double mid = 0.5 * (a + b);
                if (scaled_total(raw, k, mid, lo) <= cap)
                    a = mid;
                else
                    b = mid;
            }
            s = a;
        }
    }
    uint64_t total = 0;
    for (size_t j = 0; j < k; j++) {
        double m = floor(raw[j] * s);
        uint32_t v = m < lo ? lo : (uint32_t)m;
        len[j] = v;
        total += v;
    }
    free(raw);
    return total;
}

/* One sorted list of m ids below 2^31.  `first` is the list's position in the
 * concatenation of all lists (counter base); attempt a uses stream 1 + a. */
static int posting_list_one(uint64_t seed, uint64_t first, uint32_t m, uint32_t *out)
{
    double log1mp = log1p(-((double)m + 1.0) / 2147483648.0);
    for (uint32_t attempt = 0; attempt < 255; attempt++) {
        uint64_t run = 0;
        int ok = 1;
        for (uint32_t k = 0; k < m; k++) {
            run += geometric(svbgen_word(seed, 1 + attempt, first + k), log1mp);
            if (run >= 2147483648ull) {
                ok = 0;
                break;
            }
            out[k] = (uint32_t)run;
        }
        if (ok)
            return (int)attempt;
    }
    /* Never reached in practice: fall back to a dense run 0..m-1. */
    for (uint32_t k = 0; k < m; k++)
        out[k] = k;
    return 255;
}

struct lists_ctx {
    uint64_t seed;
    const uint32_t *len;
    const uint64_t *first; /* exclusive prefix of len */
    uint32_t *out;
};

static void lists_range(void *p, size_t b, size_t e)
{
    struct lists_ctx *c = (struct lists_ctx *)p;
    for (size_t j = b; j < e; j++)
        posting_list_one(c->seed, c->first[j], c->len[j], c->out + c->first[j]);
}

/* Lists are uneven (8 .. ~10^5 ids): thread t takes lists t, t+T, t+2T, ... */
struct lists_thread {
    struct lists_ctx *c;
    size_t t, T, k;
};

static void *lists_strided(void *p)
{
    struct lists_thread *a = (struct lists_thread *)p;
    for (size_t j = a->t; j < a->k; j += a->T)
        lists_range(a->c, j, j + 1);
    return NULL;
}

/* All k lists back to back into out (sum of len entries). */
void svbgen_posting_lists(uint64_t seed, size_t k, const uint32_t *len,
                          const uint64_t *first, uint32_t *out, int nthreads)
{
    struct lists_ctx c = {seed, len, first, out};
    nthreads = thread_count(nthreads);
    if (k < 64 || nthreads == 1) {
        lists_range(&c, 0, k);
        return;
    }
    pthread_t tid[64];
    struct lists_thread arg[64];
    int ok[64];
    for (int t = 0; t < nthreads; t++) {
        arg[t].c = &c;
        arg[t].t = (size_t)t;
        arg[t].T = (size_t)nthreads;
        arg[t].k = k;
        ok[t] = pthread_create(&tid[t], NULL, lists_strided, &arg[t]) == 0;
        if (!ok[t])
            lists_strided(&arg[t]);
    }
    for (int t = 0; t < nthreads; t++)
        if (ok[t])
            pthread_join(tid[t], NULL);
}

/* One fresh list, for the serving loop's encode requests. */
int svbgen_posting_list(uint64_t seed, uint64_t first, uint32_t m, uint32_t *out)
{
    return posting_list_one(seed, first, m, out);
}
