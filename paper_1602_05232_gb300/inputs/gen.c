/*
 * Seeded synthetic input generators for the incremental-connectivity streams.
 *
 * This file holds no connectivity arithmetic: it only produces vertex ids
 * (edges and query pairs) and random numbers. Both the CUDA path and the CPU
 * oracle consume exactly the bytes written here, so the same seed gives the
 * same stream on both sides.
 *
 * Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast Splittable
 * Pseudorandom Number Generators", OOPSLA 2014), evaluated at an arbitrary
 * position: the generator's state after i steps is key + i * GAMMA, and the
 * output is the published 64-bit finaliser of that state. Every draw is a pure
 * function of (seed, tag, counter), so a batch can be generated on its own and
 * multi-threaded generation is deterministic whatever the thread count.
 *
 * The stream model is the paper's (Section 1, "Model"): a graph stream is a
 * sequence of minibatches of edges on V = {0..n-1}; minibatches may differ in
 * size. Shapes follow the paper's workloads (Section 5.2, Table 1): uniform
 * random edges, R-MAT power-law edges and a mesh.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#define SM64_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* i-th output (i >= 0) of the SplitMix64 sequence whose initial state is key. */
static inline uint64_t sm64_at(uint64_t key, uint64_t i) {
    return sm64_mix(key + (i + 1) * SM64_GAMMA);
}

/* Independent stream key per (seed, tag). */
uint64_t gen_stream_key(uint64_t seed, uint64_t tag) {
    return sm64_mix(sm64_mix(seed) ^ sm64_mix(tag * SM64_GAMMA + 0x632BE59BD9B4E019ULL));
}

/* Uniform integer in [0, n) from the top 32 bits (multiply-shift; the bias is
 * at most n / 2^32, below 2^-15 for every n used here). n <= 2^32. */
static inline uint32_t below(uint64_t r, uint64_t n) {
    return (uint32_t)(((r >> 32) * n) >> 32);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double unit(uint64_t r) {
    return (double)(r >> 11) * (1.0 / 9007199254740992.0);
}

/* ---------------------------------------------------------------- threads */

typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);
typedef struct { range_fn fn; void* ctx; int64_t lo, hi; } range_job;

static void* range_thread(void* arg) {
    range_job* j = (range_job*)arg;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static int g_threads = 0;

void gen_set_threads(int t) { g_threads = t; }

static void parallel_for(int64_t count, range_fn fn, void* ctx) {
    int t = g_threads;
    if (t <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        t = c > 0 ? (int)c : 1;
        if (t > 64) t = 64;
    }
    if (count < (1 << 16) || t == 1) {
        fn(ctx, 0, count);
        return;
    }
    pthread_t th[64];
    range_job jobs[64];
    int64_t chunk = (count + t - 1) / t;
    int started = 0;
    for (int i = 0; i < t; i++) {
        int64_t lo = (int64_t)i * chunk, hi = lo + chunk;
        if (lo >= count) break;
        if (hi > count) hi = count;
        jobs[i].fn = fn; jobs[i].ctx = ctx; jobs[i].lo = lo; jobs[i].hi = hi;
        if (pthread_create(&th[i], NULL, range_thread, &jobs[i]) != 0) {
            fn(ctx, lo, hi);          /* could not start a thread: do it here */
            jobs[i].fn = NULL;
        }
        started = i + 1;
    }
    for (int i = 0; i < started; i++)
        if (jobs[i].fn) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------- uniform pairs */

typedef struct { uint64_t key; uint64_t n; int64_t offset; int32_t* out; } pairs_ctx;

static void pairs_range(void* vc, int64_t lo, int64_t hi) {
    pairs_ctx* c = (pairs_ctx*)vc;
    for (int64_t i = lo; i < hi; i++) {
        uint64_t ctr = (uint64_t)(c->offset + i) * 2;
        c->out[2 * i]     = (int32_t)below(sm64_at(c->key, ctr), c->n);
        c->out[2 * i + 1] = (int32_t)below(sm64_at(c->key, ctr + 1), c->n);
    }
}

/* k pairs (u, v), u and v i.i.d. uniform over [0, n), pair i drawn from
 * counters 2(offset+i) and 2(offset+i)+1. Self-pairs are kept. */
void gen_uniform_pairs(uint64_t seed, uint64_t tag, int64_t n, int64_t k,
                       int64_t offset, int32_t* out) {
    pairs_ctx c = { gen_stream_key(seed, tag), (uint64_t)n, offset, out };
    parallel_for(k, pairs_range, &c);
}

/* ------------------------------------------------------------------ R-MAT */

typedef struct {
    uint64_t key; int scale; double ta, tab, tabc;
    int64_t offset; const int32_t* perm; int32_t* out;
} rmat_ctx;

static void rmat_range(void* vc, int64_t lo, int64_t hi) {
    rmat_ctx* c = (rmat_ctx*)vc;
    const int s = c->scale;
    for (int64_t i = lo; i < hi; i++) {
        uint64_t base = (uint64_t)(c->offset + i) * (uint64_t)s;
        uint32_t u = 0, v = 0;
        for (int l = 0; l < s; l++) {
            double r = unit(sm64_at(c->key, base + (uint64_t)l));
            uint32_t bit = 1u << (s - 1 - l);
            if (r < c->ta) {
                /* quadrant a: top-left */
            } else if (r < c->tab) {
                v |= bit;               /* b: top-right */
            } else if (r < c->tabc) {
                u |= bit;               /* c: bottom-left */
            } else {
                u |= bit; v |= bit;     /* d: bottom-right */
            }
        }
        if (c->perm) { u = (uint32_t)c->perm[u]; v = (uint32_t)c->perm[v]; }
        c->out[2 * i] = (int32_t)u;
        c->out[2 * i + 1] = (int32_t)v;
    }
}

/* k R-MAT edges on 2^scale vertices (Chakrabarti, Zhan and Faloutsos, SDM
 * 2004): at each of the scale levels one quadrant is picked with
 * probabilities (a, b, c, 1-a-b-c), no noise; level l of edge i uses counter
 * (offset+i)*scale + l. perm (length 2^scale, or NULL) relabels the ids.
 * Self-loops and repeated edges are kept. */
void gen_rmat_edges(uint64_t seed, uint64_t tag, int scale, double a, double b,
                    double c, int64_t k, int64_t offset, const int32_t* perm,
                    int32_t* out) {
    rmat_ctx x = { gen_stream_key(seed, tag), scale, a, a + b, a + b + c,
                   offset, perm, out };
    parallel_for(k, rmat_range, &x);
}

/* ------------------------------------------------- permutations, shuffles */

/* Fisher-Yates (Durstenfeld) permutation of [0, n): for i = n-1 .. 1 swap
 * out[i] with out[j], j uniform in [0, i], drawn from counter n-1-i. */
void gen_permutation(uint64_t seed, uint64_t tag, int64_t n, int32_t* out) {
    uint64_t key = gen_stream_key(seed, tag);
    for (int64_t i = 0; i < n; i++) out[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; i--) {
        int64_t j = below(sm64_at(key, (uint64_t)(n - 1 - i)), (uint64_t)(i + 1));
        int32_t t = out[i]; out[i] = out[j]; out[j] = t;
    }
}

/* Fisher-Yates shuffle of k pairs in place (pairs move as units). */
void gen_shuffle_pairs(uint64_t seed, uint64_t tag, int64_t k, int32_t* pairs) {
    uint64_t key = gen_stream_key(seed, tag);
    int64_t* p = (int64_t*)pairs;   /* a pair is 8 bytes; the buffer is 8-aligned */
    for (int64_t i = k - 1; i > 0; i--) {
        int64_t j = below(sm64_at(key, (uint64_t)(k - 1 - i)), (uint64_t)(i + 1));
        int64_t t = p[i]; p[i] = p[j]; p[j] = t;
    }
}

/* 4-neighbour grid of rows x cols, id = r*cols + c. Edges in row-major order
 * of their lower endpoint: (v, v+1) if c+1 < cols, then (v, v+cols) if
 * r+1 < rows. Returns the number written: rows*(cols-1) + (rows-1)*cols. */
int64_t gen_grid_edges(int64_t rows, int64_t cols, int32_t* out) {
    int64_t e = 0;
    for (int64_t r = 0; r < rows; r++)
        for (int64_t c = 0; c < cols; c++) {
            int64_t v = r * cols + c;
            if (c + 1 < cols) { out[2 * e] = (int32_t)v; out[2 * e + 1] = (int32_t)(v + 1); e++; }
            if (r + 1 < rows) { out[2 * e] = (int32_t)v; out[2 * e + 1] = (int32_t)(v + cols); e++; }
        }
    return e;
}

/* 6-neighbour 3-D grid of a x b x c vertices, id = (i*b + j)*c + k. Edges in
 * id order of their lower endpoint: +k, then +j, then +i neighbours. Returns
 * the number written: a*b*(c-1) + a*(b-1)*c + (a-1)*b*c. */
int64_t gen_grid3d_edges(int64_t a, int64_t b, int64_t c, int32_t* out) {
    int64_t e = 0;
    for (int64_t i = 0; i < a; i++)
        for (int64_t j = 0; j < b; j++)
            for (int64_t k = 0; k < c; k++) {
                int64_t v = (i * b + j) * c + k;
                if (k + 1 < c) { out[2 * e] = (int32_t)v; out[2 * e + 1] = (int32_t)(v + 1); e++; }
                if (j + 1 < b) { out[2 * e] = (int32_t)v; out[2 * e + 1] = (int32_t)(v + c); e++; }
                if (i + 1 < a) { out[2 * e] = (int32_t)v; out[2 * e + 1] = (int32_t)(v + b * c); e++; }
            }
    return e;
}

/* ------------------------------------------------------ scalar draws */

/* count doubles uniform in [0, 1), draw i from counter offset+i. */
void gen_unit(uint64_t seed, uint64_t tag, int64_t count, int64_t offset, double* out) {
    uint64_t key = gen_stream_key(seed, tag);
    for (int64_t i = 0; i < count; i++) out[i] = unit(sm64_at(key, (uint64_t)(offset + i)));
}

/* count raw 64-bit draws, draw i from counter offset+i. */
void gen_u64(uint64_t seed, uint64_t tag, int64_t count, int64_t offset, uint64_t* out) {
    uint64_t key = gen_stream_key(seed, tag);
    for (int64_t i = 0; i < count; i++) out[i] = sm64_at(key, (uint64_t)(offset + i));
}
