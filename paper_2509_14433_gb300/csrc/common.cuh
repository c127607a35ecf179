// Device helpers and graph state shared by the CUDA sources of libcupc.
//
// Sketch layout in HBM (layer-major): bucket (r, w, j) of layer r, vertex w,
// bucket j lives at sketch[(r * V + w) * W + j], 16 bytes {alpha, gamma}.
// j = 0 is the deterministic bucket, j = 1 + c*D + d is row d of column c
// (App. A.1.1, Theorem A.2: one bucket per column per update).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <vector>
#include <stdint.h>

#include "cupc.h"

namespace cupc {

constexpr uint32_t kErrInval = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr uint32_t kErrQuery = 4u;  // a query pair out of range (does not drop updates)
constexpr uint64_t kNone = ~0ull;
constexpr uint32_t kNoneU32 = 0xFFFFFFFFu;
// Most vertices: an edge id (< V^2) and a vertex id share one 64-bit key in
// the recovery's hook.
constexpr uint32_t kMaxVertices = 1u << 21;

// Rows per column that the update kernel folds in shared memory; deeper rows
// (probability 2^-kSmemRows per index) are XORed straight into HBM.
constexpr uint32_t kSmemRows = 8;      // default (the autotuner's usual pick on GB300)
constexpr uint32_t kSmemRowsMax = 16;
// Records (endpoint incidences) per update work item.
constexpr uint32_t kItemRecords = 512;  // maximum
constexpr uint32_t kDefaultItemRecords = 256;
constexpr uint32_t kMinItemRecords = 64;
// The update groups a batch through per-CTA shared histograms when
// V <= kPrivMaxV (8 bytes per vertex of shared memory) and one CTA per
// kPrivPerVertex * V endpoint records (at most one per SM) gives at least
// kPrivMinCtas CTAs. Measured on GB300 (group time per batch): V = 16384,
// 2^20 edges 77 -> 45 us; V = 4096, 2^20 edges 133 -> 36 us; one CTA per
// 2V records was slower, and too few CTAs lose to the global atomics.
constexpr uint32_t kPrivMaxV = 24576;
constexpr uint32_t kPrivPerVertex = 1;
constexpr uint32_t kPrivMinCtas = 48;
// Most vertex slices of the update's plan kernels.
constexpr uint32_t kPlanSlices = 1024;
// Most CTAs of the single-graph apply kernel (its direct-path items number
// at most 2 per CTA + 1 beyond one per 64 direct records).
constexpr uint32_t kPlanGridCap = 8192;
// Below this many endpoint records per vertex on average in a batch, the
// apply kernel writes a single-item vertex back by load and store; at or
// above it, by XOR atomics. GB300, uniform batches, ms per launch
// (load-store / atomics): V = 2^17 and 2^18, 2^20, 2^22 edges: 1.03 / 1.25,
// 1.47 / 1.62, 2.84 / 2.29; V = 16384 and 2^16, 2^18, 2^20 edges: 0.14 /
// 0.18, 0.21 / 0.21, 0.48 / 0.41.
constexpr uint32_t kExclRecords = 32;
// Records an apply CTA stages per pass: idx and the checksums G_r(idx) of
// every layer of kStage records sit in shared memory.
constexpr uint32_t kStage = 64;
// Dynamic shared memory of an apply CTA for graphs of at most L layers:
// rows x threads fold rows, two buffers of kStage staged records, the L
// checksums of one pass, the L layer checksum keys and two buffers of the
// records' vertices (direct path).
inline size_t apply_smem_bytes(uint32_t rows, uint32_t threads, uint32_t L) {
  return (size_t)rows * threads * 16 + (size_t)kStage * 8 * (2 + L) + (size_t)L * 8 + (size_t)kStage * 2 * 4;
}
// Key words of a graph: L*(C+1) (column multipliers and layer checksum
// keys) + 3*L*C (the other multiply-add-shift words of every column).
constexpr size_t key_words(uint32_t L, uint32_t C) { return (size_t)L * (C + 1) + (size_t)3 * L * C; }
// Output bits of one multiply-add-shift stage for indices below V^2:
// 65 - 2*ceil(log2 V) (strong universality with 64-bit words).
inline uint32_t hash_bits(uint32_t V) {
  uint32_t lg = 0;
  while (((uint64_t)1 << lg) < (uint64_t)V) lg++;
  if (lg < 1) lg = 1;
  return 65 - 2 * lg;
}
// Threads of the recovery kernel and members per reduction work item.
constexpr uint32_t kRecThreads = 256;
constexpr uint32_t kRecSpan = 8;  // also the largest "small" component
// Members per CTA tile when reducing big components.
constexpr uint32_t kRecTile = 64;
constexpr uint32_t kWarpBuckets = 8;  // buckets per lane in the recovery: W <= 256
// Crossing candidates at or below which a recovery hook finishes in one CTA
// (shared memory) instead of across the grid.
constexpr uint32_t kSmallHook = 1024;
// One-cluster recovery (recover_small.cu): graphs of at most kClMaxV
// vertices keep their per-vertex recovery state in one CTA's shared memory
// (26 bytes a vertex); kClThreads threads per CTA. Measured on GB300 (one
// recovery after 100 toggles, ER graphs): V = 1024 55 us vs 118 us for the
// grid-wide kernel, V = 2048 74 vs 128, V = 4096 117-148 vs 150-179 (1024
// threads per CTA; 512 gave 56, 81 and 139-167 us). With 512 threads the
// grid-wide kernel was faster from V = 6144 on (186 vs 157 us): the
// cluster's 16 SMs run out of issue and memory bandwidth.
constexpr uint32_t kClMaxV = 4096;
constexpr uint32_t kClThreads = 1024;
// Bounded device-side waits give up after this long.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Device-side counters of one graph (u32 slots of `gc`).
enum : uint32_t {
  GC_ERR = 0,        // sticky error bits (kErrInval drops update batches)
  GC_NITEMS = 1,     // update work items of the current chunk
  GC_NEXT_ITEM = 2,  // dynamic scheduler cursor of the apply kernel
  GC_NFOREST = 3,
  GC_NZ = 4,         // non-ZERO samples this round
  GC_ACTIVE = 5,     // MSF: candidates still crossing two trees (even hook steps)
  GC_NMEMBERS = 6,   // live members this round
  GC_NFAIL = 7,
  GC_NFP = 8,
  GC_ROUNDS = 9,
  GC_COMPLETE = 10,
  GC_LOGLEN = 11,
  GC_ACTIVE_ODD = 12,  // MSF: same count for odd hook steps
  GC_BAR_COUNT = 13,
  GC_RECOVERIES = 15,
  GC_BATCHES = 16,   // update chunks applied
  GC_NBIG = 17,      // members of big components this round
  GC_NDIRECT = 18,   // direct-path records of the current chunk
  GC_NLIVE = 19,     // live components of the next recovery round
  GC_REC_DIRTY = 20, // a recovery gave up at a barrier: its scratch may be non-zero
  GC_LABELS_VALID = 21,  // incremental mode: labels hold the current graph's components
  GC_FOREST_SORTED = 22, // forest_sorted holds the last recovery's forest
  GC_BATCH_DEL = 24,     // the current batch deletes an edge (incremental mode)
  GC_WARM = 25,          // incremental mode: forest edges were deleted: warm-start recovery
  GC_NSORTED = 26,       // length of forest_sorted
  GC_NFADD = 27,         // incremental mode: merge edges recorded in fadd since the last recovery
  GC_BATCH_MERGE = 28,   // the current batch merged two components (incremental mode)
  GC_SLOTS = 32
};

// SplitMix64 output finalizer (Steele, Lea, Flood, OOPSLA 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_cg(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ uint64_t ld_cg(const uint64_t* p) {
  return (uint64_t)__ldcg((const unsigned long long*)p);
}
__device__ __forceinline__ uint8_t ld_cg(const uint8_t* p) {
  return (uint8_t)__ldcg((const unsigned char*)p);
}

}  // namespace cupc

// Host-side state of one graph. Device arrays are carved from one workspace.
struct cupc_graph {
  uint32_t V, L, C, D, W, P, R;  // P: lanes per layer in the update kernel
  uint32_t ell;                  // bits of one column-hash stage (hash_bits(V))
  bool long_depth;               // ell < D-1 or D-1 > 32: depths may need the slow path
  uint64_t seed;
  uint32_t max_batch, max_pairs;
  void* ws;
  size_t ws_bytes;
  bool owns_ws;
  bool dirty;
  bool inc;           // incremental labels (cupc_set_incremental)
  bool forest_stale;  // an update since the last full recovery
  bool sort_pending;  // incremental mode: a recovery ran; the next update sorts its forest first
  bool imported;      // words from cupc_import_sketches since the last reset:
                      // the XOR of all vertex sketches need not be zero
  int device, sms;
  int apply_threads, apply_smem, apply_grid;
  uint32_t item_records, apply_cps;  // tunables: records per work item, CTAs per SM (0 = max)
  // optional per-batch-size settings: bucket floor(log4 edges) (at least 5)
  struct ApplyTune {
    bool set;
    uint32_t item_records, R, cps;
    int smem, grid;
  } tune_b[16];
  uint32_t wb_b[16];  // write-back mode per bucket (CUPC_WRITEBACK_*)
  int rec_grid;
  int rec_cluster;  // CTAs of the one-cluster recovery (0: the grid-wide kernel)
  // sketches and keys
  ulonglong2* sketch;  // L*V*W
  uint64_t* keys;      // key_words(L, C)
  uint32_t* gc;        // GC_SLOTS device counters
  // update scratch
  uint32_t* cnt;       // V
  uint32_t* cursor;    // V
  uint64_t* rec;       // 2*max_batch
  uint32_t* recw;      // 2*max_batch: vertex of each direct-path record
  uint4* items;        // 4*max_batch/kMinItemRecords + min(V, 2*max_batch) + 1
  uint4* part;         // kPlanSlices per-slice totals of the plan
  uint32_t* stage_edges;  // 2*max_batch (host-input staging slot 0)
  int8_t* stage_ops;      // max_batch
  uint32_t* stage_edges1;  // 2*max_batch (slot 1)
  int8_t* stage_ops1;      // max_batch
  // host inputs of cupc_update_batch are copied on copy_stream into the two
  // slots in turn: slot_ready[k] after a copy, slot_free[k] after the last
  // kernel (on the caller's stream) that reads slot k
  cudaStream_t copy_stream;
  cudaEvent_t slot_ready[2], slot_free[2];
  int next_slot;
  uint32_t* stage_pairs;  // 2*max_pairs
  uint8_t* stage_out;     // max_pairs
  // recovery state
  uint32_t* label;   // V
  uint32_t* parent;  // V
  uint32_t* minv;    // V
  uint32_t* rcnt;    // V
  uint32_t* roff;    // V
  uint32_t* perm;    // V: members of small components, grouped
  uint32_t* permb;   // V: members of big components, grouped
  uint32_t* pcount;  // V: spans of a component reduced so far
  uint8_t* final_;   // V
  uint8_t* merged;   // V
  uint64_t* best;    // V
  uint64_t* best2;   // V
  ulonglong2* cand;  // V: {candidate edge, endpoint labels}
  uint64_t* forest;  // V
  uint64_t* forest_sorted;  // V
  ulonglong2* acc;   // V*W (partial component sums)
  uint64_t* log_ids; // L*V
  uint32_t* log_live;   // L
  uint32_t* log_ncand;  // L
  ulonglong2* hlist;    // kSmallHook: crossing candidates of a hook step (recovery)
  uint32_t* ipar;       // V: union-find over labels for incremental inserts
  uint8_t* fdead;       // V: forest_sorted[i] was deleted since the last recovery
  // incremental mode: the inserts that merged two components since the last
  // recovery (forest edges the stream added), and a hash table of their ids
  uint64_t* fadd;       // V
  uint8_t* fadd_dead;   // V: fadd[j] was deleted since
  uint64_t* ftab;       // 2^ftab_bits ids (0 = empty slot; no edge has id 0)
  uint32_t* ftab_pos;   // 2^ftab_bits: the fadd index of ftab's id
  uint32_t ftab_bits;
  cupc_status last_recovery;
  // profiling: (kernel class, start, stop, launches) per recorded launch group
  struct ProfRec {
    int cls;
    cudaEvent_t a, b;
    int launches;
  };
  bool prof_on;
  std::vector<ProfRec> prof;
  double prof_ms[8];
  uint64_t prof_launches[8];
  cudaStream_t last_stream;
};

namespace cupc {
enum ProfClass { PC_VALIDATE = 0, PC_GROUP = 1, PC_APPLY = 2, PC_RECOVER = 3, PC_QUERY = 4, PC_SORT = 5, PC_N = 8 };
// Record an event pair around a launch group when profiling is on.
struct ProfScope {
  cupc_graph* g;
  cudaStream_t s;
  int cls, launches;
  cudaEvent_t a = nullptr;
  ProfScope(cupc_graph* g_, cudaStream_t s_, int cls_, int launches_) : g(g_), s(s_), cls(cls_), launches(launches_) {
    g->last_stream = s;
    if (g->prof_on && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, s);
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    cudaEventRecord(b, s);
    g->prof.push_back({cls, a, b, launches});
  }
};
}  // namespace cupc

namespace cupc {
// Launchers (defined in update.cu / recover.cu); all stream-ordered.
cudaError_t launch_keys(cupc_graph* g, cudaStream_t s);
// validate_ops: also validate this chunk (a batch of one chunk), else the
// caller has validated the whole batch first.
cudaError_t launch_update_chunk(cupc_graph* g, const uint32_t* edges, size_t n, cudaStream_t s,
                                const int8_t* validate_ops = nullptr);
cudaError_t launch_validate(cupc_graph* g, const uint32_t* edges, const int8_t* ops, size_t n, cudaStream_t s);
cudaError_t setup_update(cupc_graph* g);
cudaError_t configure_apply(cupc_graph* g);
cudaError_t apply_config(const cupc_graph* g, uint32_t item_records, uint32_t R, uint32_t cps, int* smem, int* grid);
// Tuning bucket of a batch of n edges: floor(log4 n), at least 5, at most 15.
inline uint32_t tune_bucket(size_t n) {
  uint32_t b = 5;
  while (b < 15 && ((size_t)1 << (2 * (b + 1))) <= n) b++;
  return b;
}
cudaError_t raise_apply_smem_limit(int bytes);
cudaError_t setup_recover(cupc_graph* g);
cudaError_t launch_recover(cupc_graph* g, cudaStream_t s, bool force = false);
cudaError_t launch_query(cupc_graph* g, const uint32_t* pairs, size_t m, uint8_t* out, cudaStream_t s);
cudaError_t launch_forest_sort(cupc_graph* g, cudaStream_t s);
cudaError_t launch_incremental(cupc_graph* g, const uint32_t* edges, const int8_t* ops, size_t n, cudaStream_t s);
}  // namespace cupc
