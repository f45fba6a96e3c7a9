// Internal declarations shared by the libcc translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "cc.h"

namespace cc {

// Bits of the device status word.
enum : unsigned {
    ST_RANGE = 1u,    // an edge or query endpoint was outside [0, n)
    ST_CORRUPT = 2u,  // parent[x] > x was seen (cannot happen through the API)
};

// Device-side bookkeeping of one handle (one small allocation).
struct DevState {
    unsigned status;            // ST_* bits, cleared by cc_sync
    unsigned labels_bad;        // set by the label validator
    unsigned long long unions;  // successful hooks since create / reset
    unsigned long long roots;   // roots counted by the label validator
    unsigned queue;             // work-queue counter of the batched form
    unsigned max_depth;         // forest height diagnostic
    unsigned long long sum_depth;
    int big_root;               // largest-component filter: the root R whose tree the bitmap
                                // marks, or -1 = no filter (set by the pick kernel)
    unsigned big_pad;
    unsigned long long big_members;  // set bits of the bitmap (launch_big_count, on demand)
};

struct Launch {
    int block;        // threads per block, multiple of 32
    int ept;          // edges (pairs) per thread: 1, 2 or 4
    int variant = 0;  // update kernel: 0 per-edge walks, 1 lockstep walks, 2 persistent + prefetch,
                      // 3 persistent + two-stage prefetch (edges two chunks ahead, parents one),
                      // 4 filter pass + live-edge pass (launch_update_split),
                      // 5 persistent tiles whose open edges the whole CTA walks from a shared-memory list
    int query_variant = 0;  // query kernel: 0 one chunk per thread, 1 persistent + prefetch
    const cudaAccessPolicyWindow* window = nullptr;  // L2 window over the forest, or none
    int pdl = 0;  // programmatic dependent launch: 0 off, 1 wait first, 2 first pairs before the wait
    int qept = 0; // pairs per thread of the query kernel (0 = ept)
    int minhook = 0;  // 1: Bulk-Update hooks with atomicMin + repair (hook_min) instead of CAS
    int warphook = 0; // 1: the hooks of a warp are grouped by target root (hook_warp); lockstep variants
    const unsigned* big = nullptr;  // largest-component bitmap (n bits), or none: pairs whose two
                                    // endpoints are marked are answered / dropped without walks
    const int* alt = nullptr;       // Bulk-Update on an ordered copy: the caller's edges, which the
                                    // update reads instead while the bitmap is in use (see BigArgs)
};

// What the fused Bulk-Update kernels take of the largest-component filter.
// While the bitmap marks a tree (big != null, DevState::big_root >= 0) most
// edges are dropped before their parent reads, and ordering them no longer
// pays: launch_order_edges given the same `big` then does nothing, and an
// update kernel given the ordered copy reads the caller's edges, `alt`,
// instead. Both decide from big_root, which only the pick kernel writes, and
// a full compression pass, launched without programmatic dependence, always
// follows the pick, so every later kernel reads its final value.
struct BigArgs {
    const unsigned* big = nullptr;
    const int* alt = nullptr;
};

// Alignment class of a pair array: 2 = 16-byte, 1 = 8-byte, 0 = 4-byte.
int pair_vec(const void* p);

// Sets the text returned by cc_last_error_string() and returns s.
cc_status record_error(cc_status s, const char* msg);

// The stream a handle is bound to, and its device.
cudaStream_t ctx_stream(const cc_ctx* c);
int ctx_device(const cc_ctx* c);
int32_t ctx_graphs(const cc_ctx* c);

cudaError_t launch_reset(int* parent, int64_t n, int block, cudaStream_t s);

cudaError_t launch_update(int* parent, int n, const int* edges, int64_t k, DevState* ds,
                          Launch cfg, cudaStream_t s);

// Bulk-Update as two kernels (update variant 4): a filter pass that reads the
// first parents of every edge and lists the edges whose parents differ as
// (u, v, parent[u], parent[v]) in live[] (room for k entries), then a pass
// that walks and hooks the listed edges. count[2]: list counters, both zero
// initially; sel alternates 0, 1, 0, ... between consecutive calls.
cudaError_t launch_update_split(int* parent, int n, const int* edges, int64_t k, DevState* ds, Launch cfg,
                                int4* live, unsigned* count, int sel, cudaStream_t s);

// mode: 0 read-only finds, 1 finds with path halving, 2 flat forest (parent
// equality decides), 3 lockstep finds with path splitting.
cudaError_t launch_query(int* parent, int n, const int* pairs, int64_t k, uint8_t* out,
                         DevState* ds, int mode, Launch cfg, cudaStream_t s);

// Full compression; also writes labels to `out` when it is not null. With
// `big` (n bits, rounded up to whole 32-bit words), bit v is set to whether v's
// root is ds->big_root (nothing is written while that is -1).
cudaError_t launch_compress_all(int* parent, int64_t n, int* out, DevState* ds, int block,
                                cudaStream_t s, unsigned* big = nullptr);

// The root of the largest tree, estimated from kBigSample vertices (read-only
// walks): ds->big_root = that root if at least min_share of the sample reached
// it, else -1. One CTA.
constexpr int kBigSample = 1024;
cudaError_t launch_big_pick(const int* parent, int64_t n, int min_share, DevState* ds, cudaStream_t s);
// ds->big_members += the set bits of words[0, nwords).
cudaError_t launch_big_count(const unsigned* words, int64_t nwords, DevState* ds, cudaStream_t s);

cudaError_t launch_compress_touched(int* parent, int n, const int* edges, int64_t k,
                                    DevState* ds, Launch cfg, cudaStream_t s);

// ---- locality order of a Bulk-Update's edges (CC_OPT_EDGE_ORDER) ----

// out (2k ints) = the k edges bucketed by (min endpoint) >> order_shift(n, b)
// into 2^b buckets (b <= 9). counters: order_counter_ints(b) ints, all zero
// before the first call; each call leaves them zero again. pdl as for the
// update kernel (programmatic dependent launch: 0 off, 1 wait first, 2 read
// the edges first). *kernels = the number of kernels launched. With `big`
// (see BigArgs), both kernels return at once while ds->big_root >= 0, and
// `out` is left unwritten.
int order_shift(int64_t n, int log_buckets);
int64_t order_counter_ints(int log_buckets);
cudaError_t launch_order_edges(const int* edges, int64_t k, int n, int log_buckets, int* counters,
                               int* out, int pdl, cudaStream_t s, int* kernels,
                               const unsigned* big = nullptr, const DevState* ds = nullptr);

// ---- batched form (segmented forests, one persistent kernel) ----

// One bulk operation of the batched form, as the kernel reads it.
struct SegOp {
    const int* data;  // 2k local ids
    uint8_t* out;     // k answers (queries)
    int64_t k;
    int32_t kind;     // CC_OP_UPDATE / CC_OP_QUERY
    int32_t pad;
};

// Per-submit tables in device memory: ops grouped by graph (list order kept
// within a graph), op_begin[G+1] delimiting each graph's ops, and the order in
// which CTAs claim the *nactive graphs that have work.
struct SegTables {
    const SegOp* ops;
    const int* op_begin;
    const int* order;
    const int* nactive;
};

struct SegLaunch {
    int block;     // threads per CTA
    int ept;       // edges (pairs) per thread per step: 1, 2 or 4
    int smem_cap;  // graphs of at most this many vertices run in shared memory (<= 65536)
    int max_ctas;  // cap on the persistent grid (0 = one wave of resident CTAs)
    int grid = 0;  // set by prepare_segmented
};

// Sets the kernel's shared-memory attribute and the persistent grid size.
// Call before launching or capturing.
cudaError_t prepare_segmented(SegLaunch& cfg);

cudaError_t launch_segmented(int* parent, const int64_t* seg_off, const SegTables& t,
                             unsigned* queue, DevState* ds, const SegLaunch& cfg, cudaStream_t s);

// ---- the paper's Bulk-Update schedule (Algorithm 2 as written) ----

cudaError_t launch_relabel(int* parent, int n, const int* edges, int64_t k, int* a2, unsigned* m2,
                           int* comp, DevState* ds, int block, cudaStream_t s);
cudaError_t launch_sv_round(const int* a2, const unsigned* m2, int* comp, unsigned* hooked,
                            int grid, int block, cudaStream_t s);
cudaError_t launch_join(const int* a2, const unsigned* m2, const int* comp, int* parent,
                        DevState* ds, int grid, int block, cudaStream_t s);

// The hooking rounds as one executable CUDA graph: a while node repeats
// {clear pc[1]; hook; jump; decide} on the device until a round hooks nothing.
// pc: [0] |A''| (set by the relabel step), [1] hooked flag, [2] rounds run
// (written by the graph). The graph holds these pointers and the launch shape;
// rebuild it when any of them changes.
cudaError_t build_sv_loop(const int* a2, unsigned* pc, int* comp, DevState* ds, int grid, int block,
                          cudaGraphExec_t* out);

// Union by size (the paper's schedule only) and the walks for forests that
// do not keep parent[v] <= v.
cudaError_t launch_relabel_generic(int* parent, int n, const int* edges, int64_t k, int* a2,
                                   unsigned* m2, int* comp, unsigned long long* best, DevState* ds,
                                   int block, cudaStream_t s);
cudaError_t launch_size_join(const int* a2, const unsigned* m2, const int* comp, int* parent,
                             int* size, unsigned long long* best, DevState* ds, int grid, int block,
                             cudaStream_t s);
cudaError_t launch_fill(int* a, int64_t n, int value, cudaStream_t s);
cudaError_t launch_size_count(const int* parent, int64_t n, int* size, DevState* ds, cudaStream_t s);
cudaError_t launch_query_generic(int* parent, int n, const int* pairs, int64_t k, uint8_t* out,
                                 DevState* ds, bool flat, int block, cudaStream_t s);
// Full compression; with labels_out also the minimum-id labels (uses minid_scratch, n ints).
cudaError_t launch_compress_generic(int* parent, int64_t n, int* labels_out, int* minid_scratch,
                                    DevState* ds, int block, cudaStream_t s);
cudaError_t launch_depth(const int* parent, int64_t n, unsigned* max_depth,
                         unsigned long long* sum_depth, DevState* ds, cudaStream_t s);

// ---- Bulk-Find (Algorithm 4) with the Response Distributor ----

struct BulkFindState {
    int* mark = nullptr;         // n entries: epoch stamp = visited in this call
    int epoch = 0;
    int* front[2] = {nullptr, nullptr};
    int* roots = nullptr;
    int* D[2] = {nullptr, nullptr};  // Phase II frontiers of (v, root) pairs
    int64_t cap_front = 0;           // entries of front/roots, pairs of D
    int* R = nullptr;                // R_u: (from, to) pairs
    int64_t cap_R = 0;
    int* sorted = nullptr;           // R_u sorted by bucket
    int64_t cap_R2 = 0;
    int* bucket = nullptr;           // rho + 1 bucket offsets
    int* cursor = nullptr;
    int64_t cap_bucket = 0;
    int* scan = nullptr;
    int64_t cap_scan = 0;
    int* work = nullptr;             // Phase II: bucket sizes, then their prefix sums
    int64_t cap_work = 0;
    int* res = nullptr;              // roots of the query endpoints (Bulk-Query)
    int64_t cap_res = 0;
    unsigned* count = nullptr;
    // statistics of the last call
    int64_t traversed = 0;           // |R_u| without R_0
    int32_t levels_up = 0, levels_down = 0;
    uint64_t launches = 0;           // kernels launched, cumulative
};

// res[i] = root of S[i] (-1 for an id outside [0, n)); every node on the
// paths from S to the roots points at its root afterwards. Synchronises once
// per level.
cudaError_t bulk_find(BulkFindState& b, int* parent, int n, const int* S, int64_t k, int* res,
                      DevState* ds, cudaStream_t s);
// Bulk-Query through one Bulk-Find over all 2k endpoints.
cudaError_t bulk_find_query(BulkFindState& b, int* parent, int n, const int* pairs, int64_t k,
                            uint8_t* out, DevState* ds, cudaStream_t s);
void bulk_find_free(BulkFindState& b);
// In-place exclusive scan of len ints; scratch needs scan_scratch_ints(len) ints.
int64_t scan_scratch_ints(int64_t len);
cudaError_t exclusive_scan(int* a, int64_t len, int* scratch, cudaStream_t s);

// A'' from the roots found by a Bulk-Find over the 2k endpoints (res): the
// pairs whose roots differ, with their component entries initialised.
cudaError_t launch_filter_roots(const int* res, int64_t k, int* a2, unsigned* m2, int* comp,
                                unsigned long long* best, int block, cudaStream_t s);

// Checks 0 <= p[v] <= v (and no more); counts roots.
cudaError_t launch_validate_forest(const int* p, int64_t n, DevState* ds, int block, cudaStream_t s);

// Checks 0 <= lab[v] <= v and lab[lab[v]] == lab[v]; counts roots.
cudaError_t launch_validate_labels(const int* lab, int64_t n, DevState* ds, int block,
                                   cudaStream_t s);

}  // namespace cc
