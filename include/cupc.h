/*
 * cupc: GB300-native sketch-based dynamic connectivity (arXiv 2509.14433).
 *
 * C-ABI of the CUDA library libcupc.so. Plain pointers and sizes only. All
 * compute runs in the library's sm_103a kernels on the caller's stream.
 *
 * The operations follow the paper's problem statements:
 *   - the stream model and the spanning-forest problem: App. A.1, Problem 1;
 *   - Connected(u,v) answered after any prefix of the stream: §2.1 and
 *     App. A.2, Problem 2;
 *   - vertex sketches (CameoSketch l0 samplers of the characteristic vectors
 *     f_u, O(log V) of them per vertex) and recovery by Boruvka rounds over
 *     XOR-merged sketches: App. A.1.1 (Theorem A.2, "The AGM Algorithm").
 *
 * Conventions shared by every call:
 *   - Status codes are returned; no C++ exception crosses the ABI.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Calls are
 *     stream-ordered and asynchronous unless stated otherwise. Caller-owned
 *     buffers must stay valid until the stream has reached the call.
 *   - Input/output pointers may be device memory or host memory (pinned or
 *     pageable). Host inputs are staged through a library-owned device
 *     buffer, in chunks, inside the call; host outputs are copied back and
 *     the call then synchronises the stream.
 *   - Edge (u,v), u != v, both < V, has the id u*V + v with u < v.
 *   - Errors found on the device (an invalid edge in a batch) are sticky:
 *     the batch and every later batch are dropped until cupc_sync reports
 *     and clears the error.
 *
 * Parameters and derived sizes (0 in cupc_params = default):
 *   lg = ceil(log2 V) (at least 1); rounds/layers L = lg + 2;
 *   columns C = 7; rows D = 2*lg; buckets per layer W = 1 + C*D;
 *   a bucket is two u64 words {alpha, gamma}; a vertex sketch is L*W
 *   buckets. The hash of index idx in column c of layer r is
 *   mix(idx ^ key[r*(C+1)+c]), its depth min(ctz(hash), D-1); the checksum
 *   is mix(idx ^ key[r*(C+1)+C]); key[j] = mix(seed + 0x9E3779B97F4A7C15 *
 *   (j+1)) and mix is the SplitMix64 finalizer.
 */
#ifndef CUPC_H
#define CUPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cupc_graph cupc_graph;  /* opaque; owns or borrows device memory */
typedef struct CUstream_st* cupc_stream; /* same type as cudaStream_t */

typedef enum {
  CUPC_OK = 0,
  CUPC_EINVAL = 1,      /* bad argument, or an invalid edge/pair found on the device */
  CUPC_ENOMEM = 2,      /* allocation failed or the workspace is too small */
  CUPC_EINCOMPLETE = 3, /* warning: recovery used all L rounds and some
                           component still sampled an edge or FAIL; labels and
                           forest are the partial result */
  CUPC_ECUDA = 4,       /* a CUDA runtime call failed */
  CUPC_ETIMEOUT = 5     /* a bounded device-side wait gave up */
} cupc_status;

typedef struct {
  uint32_t rounds;    /* L, sketch layers = Boruvka rounds (0: lg + 2) */
  uint32_t columns;   /* C, independent columns per l0 sampler (0: 7; max 31) */
  uint32_t rows;      /* D, rows per column (0: 2*lg; max 63) */
  uint32_t max_batch; /* edges staged per internal chunk (0: 1<<20); larger
                         batches are applied chunk by chunk, which is exact
                         because sketch addition is XOR */
} cupc_params;
/* Limits (else CUPC_EINVAL): W = 1 + C*D <= 256; L * P <= 1024 with P the
 * power of two >= C + 1 (the update kernel runs one thread per layer and
 * column, plus a checksum thread); 2 * max_batch < 2^32. */

/* Device bytes cupc_init needs for V vertices (sketches + scratch), so that
 * a caller (e.g. a PyTorch allocation) can own the memory. 0 on bad input. */
size_t cupc_workspace_bytes(uint32_t V, const cupc_params* params /* nullable */);

/* Create a graph on 2 <= V <= 2^21 vertices with no edges (the recovery packs
 * an edge id and a vertex id into one 64-bit key); hash keys derive from
 * `seed`. `workspace` (device, >= cupc_workspace_bytes, 256-byte aligned)
 * is borrowed for the graph's lifetime; NULL makes the library allocate.
 * The graph is zeroed on `stream` before the call returns.
 * Errors: CUPC_EINVAL (V out of range, params out of range, misaligned
 * workspace), CUPC_ENOMEM, CUPC_ECUDA. */
cupc_status cupc_init(uint32_t V, uint64_t seed, const cupc_params* params, void* workspace,
                      cupc_stream stream, cupc_graph** out);

/* Reset an existing graph to the empty graph (sketches zeroed), keeping
 * seed, parameters and memory. Stream-ordered. */
cupc_status cupc_reset(cupc_graph* g, cupc_stream stream);

/* Apply n edge updates (Problem 1's stream). edges: 2n u32, u0,v0,u1,v1...;
 * ops: n int8, +1 insert / -1 delete. Over F_2 both toggle the edge's
 * coordinate in f_u and f_v (App. A.1.1), so the caller must keep the stream
 * valid (insert only absent edges, delete only present ones) as Problem 1
 * requires. The whole batch is validated on the device first; any u == v,
 * u or v >= V, or op not +-1 drops the whole batch (sticky CUPC_EINVAL at
 * the next cupc_sync). n == 0 is a no-op. Marks the recovery stale.
 * edges and ops may be device or host memory. When both are host memory
 * and n <= max_batch, they are copied on an internal stream into one of two
 * staging buffers in turn, so that the copy overlaps the kernels of the
 * previous batch: the copy waits for its staging buffer, not for earlier
 * work on `stream`. So no earlier work on `stream` may still be writing
 * these host buffers, and they must stay unchanged until `stream` has
 * passed this call (as for cudaMemcpyAsync from pinned memory). Other host
 * inputs are copied on `stream`. */
cupc_status cupc_update_batch(cupc_graph* g, const uint32_t* edges, const int8_t* ops, size_t n,
                              cupc_stream stream);

/* Incremental labels (on != 0), off by default. After a complete recovery,
 * each update batch keeps the component labels exact without sketch work:
 * an insert that joins two components merges their labels and becomes an
 * edge of the kept spanning forest (the recovered forest plus these edges),
 * and a delete outside that forest changes nothing, so a query then skips
 * the Boruvka recovery. Deleting a kept forest edge makes the next query
 * recover from the fragments of the remaining forest (a warm start); a
 * batch may both merge components and delete edges, in any valid order
 * (an edge it inserts and then deletes again is found in the kept forest).
 * A reset, an import, a host batch staged in several chunks or a
 * cupc_batcher update clears the labels, and the next query recovers in
 * full. This relies on the stream
 * being valid (insert only absent edges, delete only present ones); with an
 * invalid stream the sketches toggle while the labels merge, and answers can
 * differ from a recovery's. cupc_spanning_forest always returns the forest
 * of a full recovery of the current sketches. Stream-ordered on `stream`. */
cupc_status cupc_set_incremental(cupc_graph* g, int on, cupc_stream stream);

/* Answer m Connected(u,v) queries (Problem 2): out[i] = 1 iff pairs[2i] and
 * pairs[2i+1] are in the same recovered component. Runs Boruvka recovery
 * first if an update happened since the last one. pairs: 2m u32; out: m u8.
 * A pair entry >= V sets the sticky CUPC_EINVAL and writes 0 for it. */
cupc_status cupc_query(cupc_graph* g, const uint32_t* pairs, size_t m, uint8_t* out, cupc_stream stream);

/* Spanning forest of the current graph (Problem 1): edge ids ascending into
 * edge_ids_out (cap >= V-1 always suffices); *n_out (host) receives the
 * count. Recovers first if stale. Synchronises `stream`. Returns the
 * recovery status (CUPC_OK or CUPC_EINCOMPLETE), CUPC_EINVAL if cap is too
 * small, or a pending sticky error. */
cupc_status cupc_spanning_forest(cupc_graph* g, uint64_t* edge_ids_out, size_t cap, size_t* n_out,
                                 cupc_stream stream);

/* Component label (minimum vertex id of the component) of every vertex
 * into labels_out (V u32). Recovers first if stale. */
cupc_status cupc_labels(cupc_graph* g, uint32_t* labels_out, cupc_stream stream);

/* Synchronise `stream`, then return and clear the sticky device error
 * (CUPC_EINVAL / CUPC_ETIMEOUT), else the last recovery's status. */
cupc_status cupc_sync(cupc_graph* g, cupc_stream stream);

/* Copy all sketches to dst (host or device) as [layer r][vertex w][bucket j]
 * x {alpha, gamma} u64, j = 0 deterministic bucket, j = 1 + c*D + d.
 * bytes must equal L*V*W*16. Synchronises `stream`. For parity checks and
 * checkpoints (the sketches are the whole state: import restores it). */
cupc_status cupc_export_sketches(cupc_graph* g, void* dst, size_t bytes, cupc_stream stream);
/* Overwrite all sketches from src (host or device, the export layout); the
 * next query recovers from them. Imported words need not come from a
 * stream, so until the next cupc_reset a recovery no longer assumes that
 * the XOR of all vertex sketches of a layer is zero (it samples the last
 * live component instead of taking it as ZERO); results stay those of the
 * recovery rules on whatever words were imported. Synchronises `stream`. */
cupc_status cupc_import_sketches(cupc_graph* g, const void* src, size_t bytes, cupc_stream stream);

/* Statistics of the last recovery, host array of 8 u64:
 * [0] rounds run, [1] FAIL samples, [2] checksum false positives,
 * [3] complete flag, [4] forest edges, [5] recoveries run so far,
 * [6] update batches applied, [7] sticky error bits. Synchronises. */
cupc_status cupc_stats(cupc_graph* g, uint64_t* out8, cupc_stream stream);

/* Per-round log of the last recovery (host arrays): live[r] = components
 * sampled in round r, ncand[r] = candidate entries logged in round r
 * (one per component that sampled a cut edge; the same edge may appear
 * twice), ids = the entries, round after round (unordered within a round),
 * cap = capacity of ids. *n_rounds receives the rounds run. Synchronises. */
cupc_status cupc_round_log(cupc_graph* g, uint32_t* live, uint32_t* ncand, uint64_t* ids, size_t cap,
                           uint32_t* n_rounds, cupc_stream stream);

/* Kernel timing with CUDA events recorded on the launching stream.
 * cupc_profile_enable(g, 1) starts recording around every library launch
 * (and clears earlier records); cupc_profile_read synchronises the graph's
 * last stream and returns, per kernel class k < n (0 validate, 1 group
 * = count+plan+scatter, 2 apply, 3 recover, 4 query, 5 forest sort), the
 * summed milliseconds ms[k] and the number of launches of the library's
 * kernels launches[k] since enabling. */
cupc_status cupc_profile_enable(cupc_graph* g, int on);
cupc_status cupc_profile_read(cupc_graph* g, double* ms, uint64_t* launches, size_t n);

/* ---- Batching (many batches, many graphs, few launches).
 *
 * cupc_update_batches: k consecutive batches of one graph stored back to
 * back (edges/ops as in cupc_update_batch, batch i = entries
 * [offsets[i], offsets[i+1]) of the arrays; offsets is a host array of k+1
 * non-decreasing values). Sketch addition is XOR (App. A.1.1), so applying
 * the concatenation equals applying the batches in order; they are applied
 * as one batch, in chunks of max_batch edges. The group is validated as one:
 * an invalid entry anywhere drops all k batches (sticky CUPC_EINVAL).
 *
 * cupc_batcher: applies one batch to each of k distinct graphs (k <= the
 * max_graphs given at creation) with five launches in all, whatever k is.
 * The launch sequence reads its arguments from a descriptor table in device
 * memory; with use_cuda_graph it is captured once per launch shape as a
 * CUDA graph and replayed, each call refreshing the table with one
 * host-to-device copy from pinned memory. edges[i]/ops[i] are device
 * pointers with n[i] <= that graph's max_batch entries. Results equal k
 * separate cupc_update_batch calls, including the per-graph sticky error on
 * an invalid batch; a graph with incremental labels drops them instead of
 * following the batch (its next query recovers in full). Calls on one batcher, and calls touching the same graph,
 * must be ordered on one stream. The batcher owns a small device table, two
 * pinned staging tables and the instantiated graphs. */
cupc_status cupc_update_batches(cupc_graph* g, const uint32_t* edges, const int8_t* ops, const uint64_t* offsets,
                                size_t k, cupc_stream stream);
typedef struct cupc_batcher cupc_batcher;
cupc_status cupc_batcher_create(uint32_t max_graphs, int use_cuda_graph, cupc_batcher** out);
cupc_status cupc_batcher_update(cupc_batcher* b, cupc_graph* const* graphs, const uint32_t* const* edges,
                                const int8_t* const* ops, const size_t* n, uint32_t k, cupc_stream stream);
void cupc_batcher_destroy(cupc_batcher* b);

/* ---- Serving: many resident graphs, interleaved requests (Problem 2).
 *
 * A server owns a device arena of mem_bytes in which graphs are made
 * resident (each takes cupc_workspace_bytes(V, {0,0,0,max_batch})), a pinned
 * pool of pinned_bytes for request payloads, query_streams CUDA streams and
 * one worker thread. cupc_server_open returns at once; the graph is admitted
 * when its workspace fits (graphs wait in arrival order; closing a graph
 * frees its space). Requests are copied at submission (host memory) and
 * return a ticket. The worker serves continuously: in each cycle the next
 * request of every resident graph with nothing in flight is started; a
 * graph's consecutive update requests are joined into one batch (up to
 * max_batch edges) and the batches of all such graphs go to the device in
 * one multi-graph launch sequence (cupc_batcher, CUDA-graph replay); queries
 * run on the query streams, overlapping with each other and with updates. A
 * graph has at most one request in flight, so each graph's requests complete
 * in submission order and give the same results as when it is served alone.
 * cupc_server_wait blocks up to timeout_ms for a ticket (CUPC_ETIMEOUT if it
 * is not done; the ticket stays valid) and returns its status (an invalid
 * batch reports CUPC_EINVAL on its own ticket) and latency, submission to
 * completion, in microseconds; a query's answers are in `out` by then.
 * CUPC_ENOMEM from a submission: the pinned pool is full (retry after
 * waiting) or the request can never fit. */
typedef struct cupc_server cupc_server;
typedef struct {
  size_t mem_bytes;        /* device arena for resident graphs: the admission cap */
  uint32_t max_graphs;     /* graphs open at once */
  uint32_t max_batch;      /* edges per joined update batch, pairs per query (0: 1<<20) */
  uint32_t query_streams;  /* queries in flight at once (0: 4) */
  size_t pinned_bytes;     /* pinned payload pool (0: 256 MB) */
} cupc_server_config;
cupc_status cupc_server_create(const cupc_server_config* cfg, cupc_server** out);
cupc_status cupc_server_open(cupc_server* s, uint32_t V, uint64_t seed, uint64_t* id);
cupc_status cupc_server_update(cupc_server* s, uint64_t id, const uint32_t* edges, const int8_t* ops, size_t n,
                               uint64_t* ticket);
cupc_status cupc_server_query(cupc_server* s, uint64_t id, const uint32_t* pairs, size_t m, uint8_t* out,
                              uint64_t* ticket);
cupc_status cupc_server_close(cupc_server* s, uint64_t id, uint64_t* ticket);
cupc_status cupc_server_wait(cupc_server* s, uint64_t ticket, uint32_t timeout_ms, double* latency_us);
/* Sketches of a resident graph with no pending request (export layout). */
cupc_status cupc_server_export(cupc_server* s, uint64_t id, void* dst, size_t bytes);
/* out8: [0] edges applied, [1] query pairs answered, [2] update launch
 * sequences, [3] update requests joined into them, [4] admissions, [5]
 * cycles that waited for memory, [6] resident graphs, [7] graphs waiting. */
cupc_status cupc_server_stats(cupc_server* s, uint64_t* out8);
void cupc_server_destroy(cupc_server* s);

/* Launch tunables of the update's apply kernel (results are identical for
 * every setting; only speed changes): item_records = endpoint records per
 * work item (64..512, 0 = 256), smem_rows = rows per column folded in shared
 * memory (1..min(D, 16), 0 = min(D, 8)); deeper rows go straight to HBM),
 * ctas_per_sm = resident CTAs per SM of the persistent grid (0 = as many as
 * fit). CUPC_EINVAL (previous settings kept) when out of range.
 * cupc_get_tuning: out4 = {item_records, smem_rows, ctas_per_sm, CTAs per SM
 * in use}. */
cupc_status cupc_set_tuning(cupc_graph* g, uint32_t item_records, uint32_t smem_rows, uint32_t ctas_per_sm);
cupc_status cupc_get_tuning(const cupc_graph* g, uint32_t* out4);
/* The same tunables for one batch-size bucket only: a chunk of n edges uses
 * bucket floor(log4 n) (5 for n < 4^6, 15 for n >= 4^15) if it was set,
 * else the graph's setting above, so that one graph can run small and large
 * batches each with its own setting. bucket in 5..15; all three tunables 0
 * clear the bucket. CUPC_EINVAL when out of range. */
cupc_status cupc_set_tuning_bucket(cupc_graph* g, uint32_t bucket, uint32_t item_records, uint32_t smem_rows,
                                   uint32_t ctas_per_sm);
/* Write-back of a vertex whose records form a single work item, for one
 * batch-size bucket (5..15, as above): CUPC_WRITEBACK_AUTO = load-and-store
 * when the chunk averages fewer than 32 endpoint records per vertex, else
 * XOR atomics (the default); CUPC_WRITEBACK_LOAD_STORE and
 * CUPC_WRITEBACK_ATOMIC force one. Vertices split over several items always
 * write back by atomics. Results are identical for every mode.
 * CUPC_EINVAL when bucket or mode is out of range. */
enum { CUPC_WRITEBACK_AUTO = 0, CUPC_WRITEBACK_LOAD_STORE = 1, CUPC_WRITEBACK_ATOMIC = 2 };
cupc_status cupc_set_writeback_bucket(cupc_graph* g, uint32_t bucket, uint32_t mode);

/* Derived parameters of a graph: out4 = {L, C, D, W}. */
cupc_status cupc_get_params(const cupc_graph* g, uint32_t* out4);

void cupc_destroy(cupc_graph* g);
const char* cupc_status_string(cupc_status s);

/* The architecture the library's kernels were built for, as the CUDA
 * runtime of the current device reports it for the update kernel:
 * binary (SASS) and PTX versions, major*10 + minor (103 for sm_103a).
 * Needs a device; returns CUPC_ECUDA when the runtime cannot load the
 * kernel image for it, CUPC_EINVAL for null outputs. */
cupc_status cupc_build_info(int* binary_version, int* ptx_version);

/* Self-test of failure detection on the device: every wait a library kernel
 * makes on other CTAs is bounded. This launches `ctas` (2..64) co-resident
 * CTAs that meet at a grid barrier, of which CTA `absent_cta` (-1: none)
 * never arrives; the waiting CTAs give up after limit_us microseconds
 * (1..1e6), record the timeout and return. Synchronises `stream`. Returns
 * CUPC_ETIMEOUT when the wait ran out, CUPC_OK when every CTA arrived; the
 * CUDA context stays usable either way. */
cupc_status cupc_selftest_wait_timeout(uint32_t ctas, uint32_t limit_us, int absent_cta, cupc_stream stream);

/* ---- Parallel cutset (§3.1, Lemma 3.1): tree sketches of a dynamic forest.
 *
 * A cupc_cutset keeps, for a forest F of link/cut operations over the
 * vertices of graph g, the sketch of every tree of F: the XOR of its
 * vertices' sketches in g (all L layers), i.e. the sketch of the tree's cut
 * (App. A.1.1: internal edges cancel). The forest is held as Euler tours in
 * search trees on the host; every tree node has an aggregate sketch in
 * device memory. A link or cut changes O(log V) aggregates; the sketch
 * additions it needs are logged and the batch's log is replayed in one
 * launch with one GPU thread per sketch word, each following the whole log
 * for its word (§3.1's parallel execution of the logged additions).
 *
 * The cutset reads g's vertex sketches: after changing them (any update of
 * g), REFRESH every vertex whose sketch changed. g must outlive the cutset.
 * Device memory: 3*V aggregate sketches (3*V*L*W*16 bytes) plus the log. Not
 * thread-safe; calls are ordered on `stream` and return after the replay
 * has been enqueued and its log copied (they synchronise `stream`). */
typedef struct cupc_cutset cupc_cutset;
enum { CUPC_CUTSET_LINK = 1, CUPC_CUTSET_CUT = 2, CUPC_CUTSET_REFRESH = 3 };
/* A cutset over g whose forest has no edge (every vertex its own tree). */
cupc_status cupc_cutset_create(cupc_graph* g, cupc_stream stream, cupc_cutset** out);
/* Apply n operations in order; ops (host) holds n triples {kind, u, v}:
 * LINK adds forest edge (u,v) (u and v must be in different trees), CUT
 * removes forest edge (u,v) (it must be in F), REFRESH (v ignored) recomputes
 * the aggregates over vertex u after its sketch in g changed. The first
 * invalid operation stops the batch: *applied (nullable) = the operations
 * applied before it, whose additions are replayed, and CUPC_EINVAL is
 * returned. */
cupc_status cupc_cutset_apply(cupc_cutset* c, const uint32_t* ops, size_t n, size_t* applied, cupc_stream stream);
/* *out = 1 if u and v are in one tree of F. Host only. */
cupc_status cupc_cutset_connected(const cupc_cutset* c, uint32_t u, uint32_t v, int* out);
/* The sketch of w's tree: L*W*16 bytes written to dst (device or host), laid
 * out [layer][bucket]{alpha, gamma} as one vertex of cupc_export_sketches. */
cupc_status cupc_cutset_tree_sketch(const cupc_cutset* c, uint32_t w, void* dst, cupc_stream stream);
/* Query of the cutset (Lemma 3.1; §2.1): sample layer r of w's tree sketch:
 * *result = 0 ZERO (no edge leaves the tree), 1 GOOD (*edge = u*V+v of an
 * edge with one endpoint in the tree, w.h.p.), 2 FAIL; same rule as the
 * recovery's sample. Synchronises `stream`. */
cupc_status cupc_cutset_query(const cupc_cutset* c, uint32_t w, uint32_t r, uint32_t* result, uint64_t* edge,
                              cupc_stream stream);
/* out4 = {sketch additions replayed, replay launches, links, cuts}. */
cupc_status cupc_cutset_stats(const cupc_cutset* c, uint64_t* out4);
void cupc_cutset_destroy(cupc_cutset* c);

/* ---- Update without any device allocation (the paper has no counterpart).
 *
 * For callers that cannot call cudaMalloc at all: code whose device memory
 * is owned entirely by another allocator (a framework's caching pool or a
 * fixed arena), or a latency-critical path that must not pay an allocation's
 * implicit device synchronisation. cupc_init allocates (or borrows) a
 * workspace; this call instead applies n edge updates (same rules as
 * cupc_update_batch, default parameters for V) to a sketch buffer the caller
 * owns, `sketch`, laid out exactly as cupc_export_sketches writes it
 * (L*V*W*16 bytes, device memory, zero = the empty graph), hashed with
 * `seed`. sketch (16-byte aligned), edges and ops must be device (or
 * managed) memory: anything else returns CUPC_EINVAL before any launch.
 * Its scratch is one static device array of CUPC_STATIC_SCRATCH_BYTES
 * (about 3.5 MB) in the library, held by every GPU that loads the library
 * until the process exits, so it accepts at most CUPC_STATIC_MAX_V vertices
 * and CUPC_STATIC_MAX_EDGES edges per call and returns CUPC_EINVAL beyond
 * that, before any work. The first call on a device sets up that device
 * (looks up the array's device address and the kernel's launch shape) with
 * the device current; make that first call before any stream capture. A
 * set-up that fails returns CUPC_ECUDA and is tried again by the next call.
 * Every call on a device shares the one array
 * and clears what must start at zero; calls whose work overlaps on the GPU
 * (other streams, other host threads) race on it, so order them. An invalid
 * edge drops the whole batch; status_out (nullable, device or host) receives
 * the error bits of this call (0 = applied, 1 = dropped), stream-ordered. */
#define CUPC_STATIC_MAX_V 65536u
#define CUPC_STATIC_MAX_EDGES 65536u
#define CUPC_STATIC_SCRATCH_BYTES 3494656u
cupc_status cupc_update_sketch_static(void* sketch, uint32_t V, uint64_t seed, const uint32_t* edges,
                                      const int8_t* ops, size_t n, uint32_t* status_out, cupc_stream stream);

#ifdef __cplusplus
}
#endif
#endif
