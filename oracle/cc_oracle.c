/*
 * CPU oracle for bulk incremental connectivity -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library. It shares no code with the CUDA path.
 *
 * What it computes (Section 1, "Model"; Section 3): on V = {0..n-1} the graph
 * after minibatch t is G_t = (V, A_1 u ... u A_t). Bulk-Query answers, per
 * pair (u, v), whether u and v are connected in the edges seen so far. The
 * component label of v is the smallest vertex id connected to v. Both are
 * functions of the edge set alone.
 *
 * How: a plain sequential union-find, the paper's "UF (p.c.)" baseline
 * (Section 5.3, Table 2): edges are applied one at a time in array order.
 * find() walks to the root and then, in a second walk, points every node on
 * the path at that root (full path compression, Section 5.1 "Path
 * Compression"). union() links the root of lower rank under the root of
 * higher rank (union by rank, the variant Section 3 allows besides union by
 * size); on equal ranks the second root goes under the first, whose rank
 * grows by one.
 *
 * Readings where the paper is silent:
 *  - ids are 0..n-1 (Section 2 writes [n] = {0..n}, a typo against the
 *    length-n parent array of Section 3);
 *  - self-loops and repeated edges are legal and change nothing;
 *  - an endpoint outside [0, n) makes that edge (or query) an error: it is
 *    counted and skipped, and a skipped query answers 0;
 *  - query (u, u) answers 1.
 *
 * Pinned (tests/test_oracle_pins.py) against breadth-first search, scipy's
 * connected_components, closed forms (the paper's star minibatch, grids,
 * paths, matchings, the empty stream) and invariants.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct oracle_uf {
    int64_t n;
    int32_t* p;        /* parent; p[r] == r for a root */
    uint8_t* rank;     /* upper bound on the height of r's tree */
    int64_t unions;    /* successful unions so far */
    int64_t errors;    /* edges and queries skipped for an out-of-range id */
} oracle_uf;

oracle_uf* oracle_create(int64_t n) {
    if (n < 1 || n > INT32_MAX) return NULL;
    oracle_uf* u = (oracle_uf*)calloc(1, sizeof(oracle_uf));
    if (!u) return NULL;
    u->n = n;
    u->p = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    u->rank = (uint8_t*)calloc((size_t)n, 1);
    if (!u->p || !u->rank) {
        free(u->p); free(u->rank); free(u);
        return NULL;
    }
    for (int64_t v = 0; v < n; v++) u->p[v] = (int32_t)v;   /* G_0: n singletons */
    return u;
}

void oracle_destroy(oracle_uf* u) {
    if (!u) return;
    free(u->p); free(u->rank); free(u);
}

static int in_range(const oracle_uf* u, int64_t x) { return x >= 0 && x < u->n; }

/* Root of x's tree; afterwards every node on the walked path points at it. */
static int32_t find(oracle_uf* u, int32_t x) {
    int32_t r = x;
    while (u->p[r] != r) r = u->p[r];
    while (u->p[x] != r) {
        int32_t next = u->p[x];
        u->p[x] = r;
        x = next;
    }
    return r;
}

/* Apply k edges (flat u0,v0,u1,v1,...) in array order. Returns the number of
 * successful unions this call made. */
int64_t oracle_bulk_update(oracle_uf* u, const int32_t* edges, int64_t k) {
    int64_t made = 0;
    for (int64_t i = 0; i < k; i++) {
        int32_t a = edges[2 * i], b = edges[2 * i + 1];
        if (!in_range(u, a) || !in_range(u, b)) { u->errors++; continue; }
        int32_t ra = find(u, a), rb = find(u, b);
        if (ra == rb) continue;
        if (u->rank[ra] < u->rank[rb]) {
            u->p[ra] = rb;
        } else if (u->rank[ra] > u->rank[rb]) {
            u->p[rb] = ra;
        } else {
            u->p[rb] = ra;
            u->rank[ra]++;
        }
        made++;
    }
    u->unions += made;
    return made;
}

/* out[i] = 1 iff pairs[2i] and pairs[2i+1] are connected (Algorithm 1). */
void oracle_bulk_query(oracle_uf* u, const int32_t* pairs, int64_t k, uint8_t* out) {
    for (int64_t i = 0; i < k; i++) {
        int32_t a = pairs[2 * i], b = pairs[2 * i + 1];
        if (!in_range(u, a) || !in_range(u, b)) { u->errors++; out[i] = 0; continue; }
        out[i] = (uint8_t)(find(u, a) == find(u, b));
    }
}

/* out[v] = smallest vertex id in v's component. */
void oracle_labels(oracle_uf* u, int32_t* out) {
    const int64_t n = u->n;
    int32_t* mn = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    for (int64_t v = 0; v < n; v++) mn[v] = INT32_MAX;
    for (int64_t v = 0; v < n; v++) {
        int32_t r = find(u, (int32_t)v);
        if (v < mn[r]) mn[r] = (int32_t)v;
    }
    for (int64_t v = 0; v < n; v++) out[v] = mn[find(u, (int32_t)v)];
    free(mn);
}

/* Relabel and filter (Algorithm 2, the relabel step and the self-loop
 * filter), for the edges about to be added: every edge (u, v) becomes
 * (id(u), id(v)) where id is the component identifier before the minibatch,
 * canonicalised to the smallest vertex id of the component; pairs with
 * id(u) == id(v) are dropped. Writes the survivors (A'') to out, in edge
 * order, and returns how many. Out-of-range edges are skipped. Does not add
 * the edges. */
int64_t oracle_relabel(oracle_uf* u, const int32_t* edges, int64_t k, int32_t* out) {
    const int64_t n = u->n;
    int32_t* lab = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    oracle_labels(u, lab);
    int64_t m = 0;
    for (int64_t i = 0; i < k; i++) {
        int32_t a = edges[2 * i], b = edges[2 * i + 1];
        if (!in_range(u, a) || !in_range(u, b)) continue;
        if (lab[a] == lab[b]) continue;
        out[2 * m] = lab[a];
        out[2 * m + 1] = lab[b];
        m++;
    }
    free(lab);
    return m;
}

/* Bulk-Find (Algorithm 4) on a given forest, by what it leaves behind: every
 * node on a path from a query node to its root (the union of the traversal
 * paths of Phase I), other than the root, points at that root afterwards
 * (Phase II); nothing else changes, and res[i] is the root of S[i]. The same
 * forest results from serial finds with full path compression in any order,
 * which is the equivalence of Section 4.2. Walks stop where an earlier walk
 * already passed (a flow meeting a visited node stops). `parent_in` must be
 * acyclic; a walk longer than n steps returns -1. Returns the number of
 * traversed non-root nodes, i.e. |R_u| without R_0. */
int64_t oracle_bulk_find(int64_t n, const int32_t* parent_in, const int32_t* S, int64_t k,
                         int32_t* parent_out, int32_t* res) {
    uint8_t* seen = (uint8_t*)calloc((size_t)n, 1);
    memcpy(parent_out, parent_in, (size_t)n * sizeof(int32_t));
    int64_t traversed = 0;
    for (int64_t i = 0; i < k; i++) {
        int32_t r = S[i];
        for (int64_t steps = 0; parent_in[r] != r; steps++) {
            if (steps > n) { free(seen); return -1; }
            r = parent_in[r];
        }
        res[i] = r;
        for (int32_t x = S[i]; x != r && !seen[x]; x = parent_in[x]) {
            seen[x] = 1;
            parent_out[x] = r;
            traversed++;
        }
    }
    free(seen);
    return traversed;
}

int64_t oracle_n(const oracle_uf* u) { return u->n; }
int64_t oracle_unions(const oracle_uf* u) { return u->unions; }
int64_t oracle_errors(const oracle_uf* u) { return u->errors; }

/* Number of connected components: every successful union merges two. */
int64_t oracle_components(const oracle_uf* u) { return u->n - u->unions; }
