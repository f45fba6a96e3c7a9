/*
 * libcc -- bulk-parallel incremental graph connectivity on one GB300 (sm_103a).
 *
 * The data structure of Section 3 ("Simple Bulk-Parallel Data Structure"):
 * a union-find forest over the vertex set {0, ..., n-1}, kept in device
 * memory as one int32 parent array (parent[v] == v for a root). Two bulk
 * operations act on it (Section 1, "Model"):
 *
 *   Bulk-Update  folds a minibatch of edges into the forest (Algorithm 2);
 *   Bulk-Query   answers, for each vertex pair of a minibatch, whether the two
 *                are connected by the edges added so far (Algorithm 1).
 *
 * Link rule. Hooking always makes the root with the larger id a child of the
 * root with the smaller id, so parent[v] <= v holds for every v at all times
 * and the root of each tree is the smallest id in its component. Section 3
 * links by size; any rule that joins two distinct roots is correct for
 * connectivity (the correctness lemma of Section 3.2 needs only that), and
 * this one needs no sizes array and no locks.
 *
 * Conventions for every entry point:
 *  - Vertex ids are int32 in [0, n). An edge or a query pair is two int32s,
 *    stored flat as u0, v0, u1, v1, ... (8 bytes per pair). A pointer of 16-
 *    byte alignment gets 16-byte vector loads; 4-byte alignment is the minimum.
 *  - Array arguments are DEVICE-ACCESSIBLE pointers owned by the caller
 *    unless stated otherwise: device memory, or pinned host memory mapped for
 *    the device (see cc_device_can_read), which the kernels then read and
 *    write directly over the host link. They must stay valid until the
 *    handle's stream has executed the call (calls are asynchronous).
 *  - All work is enqueued in order on the handle's stream, so each bulk
 *    operation completes before the next one starts (the paper's ordering
 *    rule, Section 1). A handle must not be used from two host threads at once.
 *  - Argument errors are found on the host and returned at once, with no
 *    state change. Errors found by kernels (out-of-range ids, a broken forest)
 *    set a device status word; they are returned by the next cc_sync() (or
 *    any call that synchronises), which also clears the word.
 *  - No entry point aborts the process. cc_last_error_string() gives the text
 *    of the last failure on the calling thread.
 */
#ifndef LIBCC_CC_H
#define LIBCC_CC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cc_ctx cc_ctx;
/* Same object as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* cc_stream_t;

typedef enum {
    CC_OK = 0,
    CC_ERR_ARG = 1,      /* bad argument (null handle/pointer, bad size, misalignment) */
    CC_ERR_OOM = 2,      /* a device allocation failed */
    CC_ERR_CUDA = 3,     /* a CUDA runtime call or a launch failed */
    CC_ERR_RANGE = 4,    /* a kernel met a vertex id outside [0, n); see below */
    CC_ERR_CORRUPT = 5,  /* a kernel met parent[v] > v (only after a bad load) */
    CC_ERR_LABELS = 6,   /* cc_load_labels: the array is not a valid labelling */
    CC_ERR_UNSUPPORTED = 7
} cc_status;

/* Compression scopes for cc_compress and the automatic policy. */
typedef enum {
    CC_COMPRESS_ALL = 0,      /* every vertex points at its root afterwards */
    CC_COMPRESS_TOUCHED = 1   /* only the endpoints of a given edge array, and their paths */
} cc_compress_scope;

/* Tunables (cc_set_option / cc_get_option). */
typedef enum {
    CC_OPT_BLOCK = 0,            /* threads per block for the bulk kernels: 64..1024, multiple of 32 (default 256) */
    CC_OPT_EDGES_PER_THREAD = 1, /* edges (or pairs) per thread in update and query: 1, 2 or 4 (default 2) */
    CC_OPT_COMPRESS_EVERY = 2,   /* cc_bulk_update compresses after every c-th call; 0 = never (default 1) */
    CC_OPT_COMPRESS_SCOPE = 3,   /* scope of that automatic compression: a cc_compress_scope (default ALL) */
    CC_OPT_QUERY_HALVING = 4,    /* how Bulk-Query finds walk: 0 read-only, all walks of a thread in
                                    lockstep (default); 1 path halving, one pair after the other;
                                    2 path splitting, all walks in lockstep (1 and 2 write, which
                                    shortens paths for later operations) */
    CC_OPT_PROFILE = 5,          /* 1: time every kernel with CUDA events on the handle's stream */
    CC_OPT_UPDATE_VARIANT = 6,   /* Bulk-Update kernel: 0 per-edge walks, 1 lockstep walks of all
                                    endpoints of a thread, 2 = 1 on a persistent grid that prefetches
                                    the next edges, 3 = 2 that also has the next chunk's first
                                    parent reads in flight during this chunk's walks, 4 = two
                                    kernels: a filter pass that reads every edge's first parents
                                    and lists the edges whose parents differ (16 B each; the list,
                                    room for the largest minibatch so far, is allocated on first
                                    use and grown with one stream synchronisation), then a pass
                                    that walks and hooks only the listed edges; 5 = a persistent
                                    grid over tiles: every thread reads its edges' first parents,
                                    the open edges go to a list in shared memory, and the whole
                                    CTA walks and hooks that list while the next tile's reads are
                                    in flight (default 0) */
    CC_OPT_L2_PERSIST = 7,       /* 1: ask L2 to keep the forest resident: the Bulk-Update and
                                    Bulk-Query kernels are launched with an access-policy window
                                    over the forest (a per-launch attribute; the stream is not
                                    changed), and the process's persisting-L2 limit is raised to
                                    the forest size, capped by the device maximum. When the last
                                    handle with the option on leaves a device (set to 0, or
                                    destroyed), the limit found before is restored and all
                                    persisting lines are reset to normal
                                    (cudaCtxResetPersistingL2Cache). Default 0 */
    CC_OPT_SEG_BLOCK = 8,        /* batched form: threads per CTA of the persistent kernel (default 512) */
    CC_OPT_SEG_EDGES_PER_THREAD = 9, /* batched form: edges (pairs) per thread per step: 1, 2, 4 (default 1) */
    CC_OPT_SEG_SMEM_CAP = 10,    /* batched form: graphs of at most this many vertices are processed in
                                    shared memory (0..65536; default 65536; 0 = all in global memory) */
    CC_OPT_SEG_GRAPH = 11,       /* batched form: 1 = capture the submit (table copy, queue reset,
                                    kernel) once as a CUDA graph and replay it (default 1) */
    CC_OPT_SEG_MAX_CTAS = 12,    /* batched form: cap on persistent CTAs (0 = one full wave, default) */
    CC_OPT_UPDATE_SCHEDULE = 13, /* Bulk-Update schedule: 0 = one fused find + CAS-hook kernel
                                    (default); 1 = the paper's Algorithm 2 as written: relabel
                                    and drop self-loops, connected components of the relabelled
                                    edges (Shiloach-Vishkin rounds), then join each component's
                                    roots under its smallest root. Schedule 1 synchronises once
                                    per round. */
    CC_OPT_LINK = 14,            /* 0 = link by index: the larger root goes under the smaller
                                    (default; parent[v] <= v always, roots are component minima);
                                    1 = union by size (Section 3, Lemma 1: trees stay O(log n) high;
                                    needs CC_OPT_UPDATE_SCHEDULE = 1, whose join step is
                                    conflict-free). Settable only while the forest has no edges;
                                    not for segmented handles. */
    CC_OPT_BULK_FIND = 15,       /* 1: Bulk-Query, and the relabel step of CC_OPT_UPDATE_SCHEDULE = 1,
                                    find all their roots with ONE Bulk-Find (Algorithm 4), whose
                                    path compression is shared by the whole minibatch (Theorem 3).
                                    Synchronises once per tree level. Default 0 */
    CC_OPT_QUERY_VARIANT = 16,   /* Bulk-Query kernel: 0 = one chunk of pairs per thread (default),
                                    1 = a persistent grid that loads the next chunk's pairs while
                                    working on the current one, 2 = warp-cooperative: a warp takes
                                    chunks of pairs, each lane keeps two pairs in flight, and a
                                    ballot hands the next pair of the chunk to every slot whose
                                    walk has finished (read-only walks whatever
                                    CC_OPT_QUERY_HALVING says) */
    CC_OPT_PDL = 17,             /* programmatic dependent launch of the Bulk-Update and Bulk-Query
                                    kernels: 0 = off; 1 = each may become resident while the kernel
                                    before it on the stream drains, and waits for that kernel to
                                    complete before it reads anything (results unchanged; default);
                                    2 = as 1, but each thread's first pairs are read BEFORE that
                                    wait -- only for pair arrays that the kernel launched just
                                    before on the same stream does not write */
    CC_OPT_QUERY_PAIRS_PER_THREAD = 18, /* pairs per thread of the Bulk-Query kernel: 1, 2 or 4;
                                    0 = as CC_OPT_EDGES_PER_THREAD (default) */
    CC_OPT_HOOK = 19,            /* how the fused Bulk-Update links two roots: 0 = compare-and-swap on
                                    the larger root, retried from its new root on failure (default);
                                    1 = atomicMin on the larger root's parent word, and when that
                                    word was no longer the root's own id, a join of the displaced
                                    parent with the smaller root (cheaper when many edges of a
                                    minibatch hook onto one root); 2 = as 1 for the first
                                    Bulk-Update after cc_create or cc_reset (an empty forest,
                                    where hub vertices make that contention worst), as 0 after.
                                    Same answers and labels */
    CC_OPT_SV_GRAPH = 20,        /* CC_OPT_UPDATE_SCHEDULE = 1 only: 1 = its hooking rounds run as one
                                    CUDA graph whose while node repeats them on the device until a
                                    round hooks nothing, with no host round trip (default); the
                                    graph is built on the first such update and rebuilt when the A''
                                    buffer grows or the block size changes. 0 = the host reads a
                                    flag after every round. Same answers and labels */
    CC_OPT_EDGE_ORDER = 21,      /* 0 = Bulk-Update takes the edges in the caller's order (default);
                                    b in 6..9 = it first orders a minibatch of at least 4096 edges
                                    into 2^b buckets by the smaller endpoint's id (a counting sort
                                    into a scratch copy; the caller's array is not written), so
                                    that the update reads the forest in roughly address order. A
                                    minibatch is a set (Section 1), so the result is the same; on
                                    graphs whose ids have locality (meshes numbered row by row)
                                    the forest's lines are then fetched about once per minibatch
                                    instead of once per endpoint. The scratch (8 B per edge of the
                                    largest minibatch so far, plus 8 B per bucket) is allocated on
                                    first use and grown with one stream synchronisation. Counted
                                    as CC_K_ORDER launches (two per ordered minibatch; they return
                                    at once while CC_OPT_BIG_FILTER's bitmap is in use) */
    CC_OPT_HOOK_WARP = 22,       /* 1 = the fused Bulk-Update's lockstep variants (CC_OPT_UPDATE_VARIANT
                                    1..4) group the hooks of a warp by target root: one lane per
                                    distinct target writes it (compare-and-swap or atomicMin, per
                                    CC_OPT_HOOK), the others join their smaller root with the
                                    winner's, so a root that many edges of a minibatch hook onto
                                    sees one atomic per warp instead of one per edge. 0 = every
                                    lane hooks on its own (default). Same answers and labels */
    CC_OPT_BIG_FILTER = 23,      /* largest-component filter (the large-component skip of Afforest,
                                    Sutton, Ben-Nun and Barak, IPDPS 2018). 0 = off (default).
                                    s in 1..1024 = before every full compression pass (automatic,
                                    CC_OPT_COMPRESS_EVERY, or cc_compress with CC_COMPRESS_ALL) one
                                    CTA walks 1024 sampled vertices to their roots; if at least s of
                                    them reach one root R, that pass also writes a bitmap of n bits
                                    (bit v = v is in R's tree; 4 bytes per 32 vertices, allocated
                                    when the option is first set), else the filter stays off until
                                    the next pass. Trees only merge, so two vertices marked then
                                    stay connected: the fused Bulk-Query (CC_OPT_QUERY_VARIANT 0, 1)
                                    answers a pair of marked vertices with 1 without reading the
                                    forest, and the fused Bulk-Update drops an edge between marked
                                    vertices before its parent reads. While it is in use, the edge
                                    order (CC_OPT_EDGE_ORDER) of the fused update does nothing and
                                    the update reads the caller's edges; this is decided on the
                                    device, with no synchronisation. cc_reset, cc_load_labels and
                                    cc_load_forest turn it off until the next pass. Plain handles,
                                    default link rule; CC_ERR_UNSUPPORTED on a segmented handle.
                                    Same answers and labels. Pick launches count as CC_K_BIG_PICK */
    CC_OPT__COUNT = 24
} cc_option;

/* Kernel kinds reported by the launch counters and the profiler. */
typedef enum {
    CC_K_UPDATE = 0,
    CC_K_COMPRESS_ALL = 1,
    CC_K_COMPRESS_TOUCHED = 2,
    CC_K_QUERY = 3,
    CC_K_LABELS = 4,
    CC_K_RESET = 5,
    CC_K_LOAD = 6,
    CC_K_SEGMENTED = 7,
    CC_K_ORDER = 8,          /* the locality order of CC_OPT_EDGE_ORDER (count, scan, scatter) */
    CC_K_BIG_PICK = 9,       /* the root pick of CC_OPT_BIG_FILTER (one CTA, before a compression) */
    CC_K__COUNT = 10
} cc_kernel_kind;

/* ------------------------------------------------------------ lifetime */

/* Create a forest over n vertices, 1 <= n <= 2^31 - 1, on the current CUDA
 * device, starting as n singletons (the empty graph G_0 of Section 1). The
 * library allocates parent[n] (4n bytes) and a status word; both are freed by
 * cc_destroy. *out receives the handle (NULL on failure). Enqueues one kernel
 * on the legacy default stream and waits for it.
 * Errors: CC_ERR_ARG (n out of range, out NULL), CC_ERR_OOM, CC_ERR_CUDA. */
cc_status cc_create(int64_t n, cc_ctx** out);

/* Wait for the handle's stream and free everything. NULL is a no-op. */
cc_status cc_destroy(cc_ctx* ctx);

/* Bind the handle to a stream (a cudaStream_t of the handle's device). Work
 * already enqueued stays on the old stream; the caller orders the two. */
cc_status cc_set_stream(cc_ctx* ctx, cc_stream_t stream);

/* Wait for all work enqueued on the handle, then return and clear any error a
 * kernel recorded since the last sync: CC_ERR_RANGE if an edge or a query had
 * an endpoint outside [0, n) (that edge was skipped and that query answered 0;
 * the rest of the minibatch was applied), else CC_ERR_CORRUPT if a kernel met
 * a parent pointer to a larger id. */
cc_status cc_sync(cc_ctx* ctx);

/* Back to n singletons (G_0), asynchronously. Clears the union counter. */
cc_status cc_reset(cc_ctx* ctx);

/* ------------------------------------------------------- bulk operations */

/* Bulk-Update (Algorithm 2; Section 3.2): add the k edges at `edges`
 * (device, 2k int32, u0 v0 u1 v1 ...) to the graph. One fused kernel: per
 * edge, find both roots with path halving (Algorithm 2's relabel step, with
 * the walk shortening of Section 5.1), drop it if the roots agree (the self-
 * loop filter of Algorithm 2), else hook the larger root under the smaller
 * with a compare-and-swap, re-finding and retrying when another edge moved
 * that root first. This replaces Algorithm 2's connected-components step and
 * Parallel-Join (Algorithm 3): both only exist to join distinct roots without
 * conflicts. The order of edges inside a minibatch does not matter (Section
 * 2); self-loops and repeated edges are legal no-ops. k = 0 is a no-op. Then,
 * per CC_OPT_COMPRESS_EVERY / _SCOPE, one compression pass (cc_compress).
 * Errors: CC_ERR_ARG (k < 0, k > 2^31 - 1, edges NULL with k > 0); ids outside
 * [0, n) are reported by cc_sync as CC_ERR_RANGE. */
cc_status cc_bulk_update(cc_ctx* ctx, const int32_t* edges, int64_t k);

/* Bulk-Query (Algorithm 1; Section 3.1): out[i] = 1 if pairs[2i] and
 * pairs[2i+1] are connected by the edges added so far, else 0. `pairs`:
 * device, 2k int32; `out`: device, k bytes, written by the kernel. A pair
 * (u, u) answers 1. Finds are read-only unless CC_OPT_QUERY_HALVING is 1;
 * when the forest is known to be flat (right after a full compression, with
 * no update since) each answer is the equality of the two parents.
 * Errors: CC_ERR_ARG; ids outside [0, n) answer 0 and are reported by cc_sync. */
cc_status cc_bulk_query(cc_ctx* ctx, const int32_t* pairs, int64_t k, uint8_t* out);

/* Path compression as a separate pass (Section 5.1, "Path Compression":
 * after the root is found, the path is walked again and every node on it is
 * pointed at the root). CC_COMPRESS_ALL does this for every vertex, leaving
 * every tree of height at most one; CC_COMPRESS_TOUCHED does it for the 2k
 * endpoints of `edges` (device, 2k int32). Answers never depend on it. */
cc_status cc_compress(cc_ctx* ctx, int32_t scope, const int32_t* edges, int64_t k);

/* Component labels: out[v] = the smallest vertex id connected to v (device,
 * n int32). Under the link rule above this is v's root; computing it also
 * compresses the forest fully. */
cc_status cc_labels(cc_ctx* ctx, int32_t* out);

/* Replace the forest by a labelling (the inverse of cc_labels, for
 * checkpoint and resume; the whole state of the structure is the O(n) parent
 * array, Theorem 2). `labels` (device, n int32) must satisfy 0 <= labels[v]
 * <= v and labels[labels[v]] == labels[v]; any labelling of a graph by
 * minimum component ids does. Synchronises. On CC_ERR_LABELS the forest is
 * unchanged. */
cc_status cc_load_labels(cc_ctx* ctx, const int32_t* labels);

/* Copy the raw parent array (device, n int32) -- for invariant checks. */
cc_status cc_copy_parent(cc_ctx* ctx, int32_t* out);

/* Number of connected components (n minus the successful hooks since create
 * or reset). Synchronises; *out is a host int64. */
cc_status cc_components(cc_ctx* ctx, int64_t* out);

/* ---------------------------------------- batched form (many graphs) */

/* Many independent graphs in one handle (the batching pattern: uneven
 * minibatches, Section 1, over many small graphs). Graph g has n_per_graph[g]
 * vertices with LOCAL ids 0..n_g-1; it owns the slice [off_g, off_g + n_g)
 * of one forest, off_g = n_0 + ... + n_{g-1}. `n_per_graph` is a host array
 * of G values, each >= 1, summing to at most 2^31 - 1. On such a handle (G >
 * 1) the forest changes only through cc_submit and cc_reset, so no edge ever
 * joins two graphs: cc_bulk_update, touched compression and cc_load_labels
 * return CC_ERR_UNSUPPORTED. Bulk-Query, cc_labels and cc_components take
 * GLOBAL ids (off_g + local id); labels are global minimum ids. */
cc_status cc_create_segmented(int32_t G, const int64_t* n_per_graph, cc_ctx** out);

enum { CC_OP_UPDATE = 0, CC_OP_QUERY = 1 };

/* One bulk operation of the batched form. */
typedef struct {
    int32_t graph;        /* graph index in [0, G) (0 on a handle from cc_create) */
    int32_t kind;         /* CC_OP_UPDATE (Algorithm 2) or CC_OP_QUERY (Algorithm 1) */
    const int32_t* data;  /* device: 2k int32 local ids, u0 v0 u1 v1 ... (4-byte aligned) */
    int64_t k;            /* edges or pairs, 0 <= k <= 2^31 - 1 */
    uint8_t* out;         /* device: k answers (CC_OP_QUERY), else ignored */
} cc_op;

/* Run `nops` operations (host array) in ONE persistent kernel launch. The
 * operations of one graph run in their order in `ops`, each completing before
 * the next starts (Section 1); operations of different graphs are independent.
 * A CTA takes a whole graph (largest work first), loads its slice of the
 * forest into shared memory when it has at most CC_OPT_SEG_SMEM_CAP vertices,
 * runs its operations there with the same find/hook as the plain path, and
 * writes the slice back with every vertex pointing at its root. With
 * CC_OPT_SEG_GRAPH the table copy, the queue reset and the launch are
 * captured once as a CUDA graph and replayed on later calls. The library
 * copies `ops` into pinned staging memory, so `ops` may be reused on return;
 * the data/out arrays must stay valid until the stream reaches the call.
 * Errors: CC_ERR_ARG (bad graph, kind, k or pointer) before anything is
 * enqueued; out-of-range local ids are reported by cc_sync (CC_ERR_RANGE). */
cc_status cc_submit(cc_ctx* ctx, const cc_op* ops, int64_t nops);

/* ------------------------------------------------------- serving form */

/* A request loop over one forest. Requests are admitted in arrival order.
 * Updates take the next stream edges; queries are vertex pairs whose answers
 * must reflect exactly the updates that arrived before them (Section 1: each
 * bulk operation completes before the next one starts).
 *
 * Continuous batching: a worker thread takes the requests that have arrived
 * and cuts them into groups of consecutive same-kind requests:
 *  - A group of updates runs as ONE Bulk-Update launch. This is exact: G_t is
 *    the union of the edge sets, and union is commutative and associative.
 *  - A group of queries runs as ONE Bulk-Query launch.
 * The stages overlap on the device:
 *  - Request data is copied from host memory into a device staging ring on a
 *    copy stream while earlier groups compute. Updates and queries have a
 *    ring each, and requests whose host data follow one another (as in one
 *    caller buffer) and land next to each other in their ring share one
 *    copy, across the groups the worker forms at a time (up to 64), so the
 *    copies stay large when the groups are small.
 *  - Query answers go back on a second copy stream.
 *  - Groups compute in arrival order on one compute stream, so no query
 *    overlaps a later update.
 * A request is admitted when its footprint (8 bytes in, plus 1 byte out per
 * query pair) fits in the free part of its kind's ring; otherwise it waits for
 * earlier groups to finish. Latency runs from enqueue to the moment a completion
 * thread sees the event recorded after the group's last device operation. */
typedef struct cc_server cc_server;

typedef struct {
    int64_t ring_pairs;       /* staging capacity in pairs of EACH of the two device rings, one for
                                 update edges and one for query pairs (<= 0: 2^25, i.e. 256 MiB
                                 each, plus 32 MiB of query answers); also the largest k a
                                 request may have */
    int64_t max_group_pairs;  /* most pairs merged into one launch (<= 0: 2^22) */
    int32_t merge;            /* 1: merge consecutive same-kind requests (default); 0: one launch per request */
} cc_server_config;

typedef struct {
    int64_t requests, updates, queries;  /* enqueued so far */
    int64_t completed;
    int64_t groups;                      /* launches (groups) issued */
    int64_t edges, pairs;                /* total update edges and query pairs enqueued */
} cc_server_stats;

/* Start a server on `ctx` (a handle from cc_create). The server binds the
 * handle to its own compute stream until cc_server_destroy, and the caller
 * must not use the handle meanwhile. cfg may be NULL (defaults).
 * Memory: besides the device staging ring, the server keeps one host record
 * (about 64 bytes) per request it has ever been given, so that any ticket can
 * be waited on and cc_server_latencies can report every request. A service
 * that runs indefinitely bounds this by draining, destroying and re-creating
 * the server from time to time (the forest is untouched by that). */
cc_status cc_server_create(cc_ctx* ctx, const cc_server_config* cfg, cc_server** out);

/* Enqueue one request; returns at once with a ticket (0, 1, 2, ... in arrival
 * order). kind is CC_OP_UPDATE or CC_OP_QUERY. `data` is a HOST array of 2k
 * int32 (pinned memory lets copies overlap), read before the request
 * completes. `out` is a host array of k bytes (queries), written before
 * completion. Both stay owned by the caller and must stay valid until then.
 * Errors: CC_ERR_ARG if k exceeds the ring or an argument is bad;
 * CC_ERR_CUDA if the worker has failed. */
cc_status cc_server_enqueue(cc_server* s, int32_t kind, const int32_t* data, int64_t k,
                            uint8_t* out, uint64_t* ticket);

/* Enqueue n requests in array order, as n calls of cc_server_enqueue would,
 * but under one lock and with one wake-up of the worker: for callers that
 * receive requests in batches (a network front end draining a socket, a
 * replayed trace), where a call per request would cost more than the request.
 * Request i is (kinds[i], data[i], k[i], out[i]) with the meaning and
 * ownership of cc_server_enqueue; `out` may be NULL when no request is a
 * query, and out[i] is ignored for updates. Its ticket is *first_ticket + i.
 * All n are checked before any is accepted: on an argument error nothing is
 * enqueued (CC_ERR_ARG, naming the first bad index). */
cc_status cc_server_enqueue_many(cc_server* s, int64_t n, const int32_t* kinds,
                                 const int32_t* const* data, const int64_t* k, uint8_t* const* out,
                                 uint64_t* first_ticket);

/* Block until request `ticket` completes; *latency_s (may be NULL) receives
 * its enqueue-to-completion time in seconds. */
cc_status cc_server_wait(cc_server* s, uint64_t ticket, double* latency_s);

/* Block until every enqueued request has completed. */
cc_status cc_server_drain(cc_server* s);

cc_status cc_server_get_stats(cc_server* s, cc_server_stats* out);

/* Latencies in seconds of requests 0 .. n-1 in ticket order (host array of n
 * doubles; -1 for a request not yet complete); *written receives min(n,
 * requests). */
cc_status cc_server_latencies(cc_server* s, double* out, int64_t n, int64_t* written);

/* Drain, stop the worker, free the server's memory and streams, and give the
 * handle back (bound again to the stream it had before). */
cc_status cc_server_destroy(cc_server* s);

/* ----------------------------------------------------------- tunables */

cc_status cc_set_option(cc_ctx* ctx, int32_t option, int64_t value);
cc_status cc_get_option(const cc_ctx* ctx, int32_t option, int64_t* value);

/* Kernel launches made by the handle so far, per cc_kernel_kind (host array
 * of CC_K__COUNT uint64), and, when CC_OPT_PROFILE is on, the summed CUDA-
 * event duration of those launches in milliseconds (host array of CC_K__COUNT
 * doubles; NULL to skip). Synchronises when ms is not NULL; reading resets the
 * timing sums, not the counters. */
cc_status cc_kernel_stats(cc_ctx* ctx, uint64_t* launches, double* ms);

/* ------------------------------------------- allocation-free labelling */

/* The paper has no counterpart to this entry point: it exists for callers
 * that cannot allocate device memory. Examples are real-time loops that
 * cannot afford cudaMalloc's implicit synchronisation and unbounded latency,
 * and plugins whose host framework owns all device memory and offers them no
 * allocator.
 *
 * Computes labels[v] = the smallest vertex id connected to v in the graph of
 * the k edges at `edges` on vertices 0..n-1: one Bulk-Update of a fresh
 * forest, then a full compression. The working forest and status word live
 * in a static device array inside libcc of CC_STATIC_MAX_VERTICES vertices
 * (16 MiB); every GPU that loads libcc holds it until the process exits. No
 * call allocates.
 *
 * `edges` (device, 2k int32) and `labels` (device, n int32) are caller-owned.
 * `status` (device, one uint32, may be NULL) receives the kernels' status
 * bits: 1 = an id outside [0, n) was skipped. Asynchronous on `stream`.
 *
 * All calls share the static array and each call re-initialises it, so calls
 * whose work can overlap on the GPU (e.g. on two unordered streams) race and
 * give wrong labels: order them. The first call on each device (and the
 * first after that device's context was replaced, e.g. by cudaDeviceReset)
 * looks up the array's device address; make that first call before any
 * stream capture.
 *
 * Errors: CC_ERR_ARG if n < 1 or n > CC_STATIC_MAX_VERTICES, or for bad k or
 * pointers, with nothing enqueued; CC_ERR_CUDA if the lookup or a launch
 * fails. */
#define CC_STATIC_MAX_VERTICES (1 << 22)
cc_status cc_components_static(const int32_t* edges, int64_t k, int64_t n, int32_t* labels,
                               uint32_t* status, cc_stream_t stream);

/* Schedule 1 only (CC_OPT_UPDATE_SCHEDULE): for the last Bulk-Update, the
 * number of relabelled edges that were not self-loops (|A''| of Algorithm 2)
 * and the number of connected-components rounds it took. Host outputs. */
cc_status cc_schedule_stats(cc_ctx* ctx, int64_t* nonloop_edges, int32_t* rounds);

/* Schedule 1 only: copy the last Bulk-Update's A'' (pairs of distinct roots,
 * in no particular order) to `out` (device, 2*cap int32); *count receives
 * |A''| (the copy stops at cap pairs). Synchronises. */
cc_status cc_copy_nonloop(cc_ctx* ctx, int32_t* out, int64_t cap, int64_t* count);

/* Bulk-Find (Algorithm 4; Section 4): res[i] = the root of S[i] for k
 * vertices `S` (device, k int32; an id outside [0, n) gives -1 and is
 * reported by cc_sync), with path compression shared by all of them:
 * afterwards every vertex on a path from some S[i] to its root points at that
 * root, and no other parent changes. Phase I walks up from all of S at once,
 * merging flows that meet; the Response Distributor (hashing into 3|R_u|
 * buckets and a counting sort, Section 4.1) lets Phase II hand each root back
 * down the recorded paths. `res`: device, k int32. Synchronises once per
 * level. */
cc_status cc_bulk_find(cc_ctx* ctx, const int32_t* S, int64_t k, int32_t* res);

/* For the last Bulk-Find: the number of traversed non-root vertices
 * (|R_u| without R_0), and the number of Phase I and Phase II levels. */
cc_status cc_bulk_find_stats(cc_ctx* ctx, int64_t* traversed, int32_t* levels_up,
                             int32_t* levels_down);

/* Replace the forest by an arbitrary one (device, n int32) with
 * 0 <= parent[v] <= v for every v -- the invariant of the default link rule,
 * which also rules out cycles. Synchronises. CC_ERR_LABELS (forest unchanged)
 * if the array breaks it; CC_ERR_UNSUPPORTED under union by size or on a
 * segmented handle. */
cc_status cc_load_forest(cc_ctx* ctx, const int32_t* parent);

/* Height of the forest: *max_depth (host) = the longest path from a vertex
 * to its root, *mean_depth (host, may be NULL) = the mean over all vertices.
 * A diagnostic for the link rules (CC_OPT_LINK). Synchronises. */
cc_status cc_forest_depth(cc_ctx* ctx, int32_t* max_depth, double* mean_depth);

/* CC_OPT_BIG_FILTER: *root (host) = the root whose tree the bitmap marks, or
 * -1 while the filter is off; *members (host) = the vertices the last
 * compression pass marked (0 when *root is -1), counted by a kernel over the
 * bitmap at this call. A diagnostic. Synchronises.
 * Errors: CC_ERR_ARG (a NULL output), CC_ERR_CUDA. */
cc_status cc_big_filter_stats(cc_ctx* ctx, int32_t* root, int64_t* members);

/* *ok = 1 if kernels on the current device can read `p` directly: device or
 * managed memory, or host memory that is pinned and mapped into the device's
 * address space (on a Grace-Blackwell node the kernels then read it over
 * NVLink-C2C). Every array argument of the bulk entry points may be such
 * host memory; check it with this call first. *ok = 0 otherwise. */
cc_status cc_device_can_read(const void* p, int32_t* ok);

int64_t cc_num_vertices(const cc_ctx* ctx);
const char* cc_status_string(cc_status s);
const char* cc_last_error_string(void);

#ifdef __cplusplus
}
#endif
#endif /* LIBCC_CC_H */
