// Batching: update batches of many graphs in one launch per stage.
//
// A cupc_batcher applies one batch to each of k graphs (App. A.1.1: every
// update touches every sketch of both endpoints; graphs are independent)
// with five launches in all, whatever k is: validate, count, plan, scatter
// and apply each cover every graph. Their arguments live in a descriptor
// table in device memory (one InstDesc per graph, prefix offsets of edges
// and work items), so the launch sequence is fixed for a batcher and is
// captured once as a CUDA graph and replayed; each call only refreshes the
// table with one host-to-device copy (double-buffered pinned staging).
// The apply kernel is persistent: CTAs pull work items from one counter
// across all graphs and fold them with the same per-item code as the
// single-graph kernel (apply_item). Results are identical to k separate
// cupc_update_batch calls.
#include <string.h>

#include <new>
#include <vector>

#include "update_dev.cuh"

namespace cupc {

struct alignas(16) InstDesc {
  const uint32_t* edges;
  const int8_t* ops;
  ulonglong2* sketch;
  const uint64_t* keys;
  uint32_t* cnt;
  uint32_t* cursor;
  uint64_t* rec;
  uint32_t* recw;
  uint4* items;
  uint32_t* gc;
  uint64_t edge_base;  // first edge of this graph in the launch's edge space
  uint32_t n, V, L, C, D, W, P, R, item_records;
  uint32_t item_base;  // first work item of this graph (set by k_plan_m)
  uint32_t nitems;     // set by k_plan_m
  uint32_t nd;         // direct-path records (set by k_plan_m)
  uint32_t ell;        // bits of one column-hash stage
  uint32_t long_depth; // depths may need the slow path
  uint32_t pad[1];
};

struct alignas(16) BatchHead {
  uint32_t k;            // graphs in this launch
  uint32_t total_items;  // set by k_plan_m
  uint32_t next_item;    // apply scheduler
  uint32_t plans_done;   // k_plan_m completion count
  uint64_t total_edges;
  uint64_t pad[5];
};

static_assert(sizeof(BatchHead) == 64, "head size");
static_assert(sizeof(InstDesc) % 16 == 0, "descriptor alignment");

__device__ __forceinline__ const InstDesc* descs_of(const BatchHead* h) {
  return reinterpret_cast<const InstDesc*>(h + 1);
}

// Graph holding global edge i: the last j with edge_base <= i.
__device__ __forceinline__ uint32_t inst_of_edge(const InstDesc* d, uint32_t k, uint64_t i) {
  uint32_t lo = 0, hi = k;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (d[mid].edge_base <= i)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t inst_of_item(const InstDesc* d, uint32_t k, uint32_t it) {
  uint32_t lo = 0, hi = k;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (ld_cg(&d[mid].item_base) <= it)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__global__ void k_validate_m(const BatchHead* __restrict__ h) {
  const InstDesc* d = descs_of(h);
  const uint32_t k = h->k;
  const uint64_t total = h->total_edges;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
    const InstDesc& g = d[inst_of_edge(d, k, i)];
    const uint64_t j = i - g.edge_base;
    const uint32_t u = g.edges[2 * j], v = g.edges[2 * j + 1];
    const int8_t op = g.ops[j];
    if ((u >= g.V) | (v >= g.V) | (u == v) | ((op != 1) & (op != -1))) atomicOr(&g.gc[GC_ERR], kErrInval);
  }
}

__global__ void k_count_m(const BatchHead* __restrict__ h) {
  const InstDesc* d = descs_of(h);
  const uint32_t k = h->k;
  const uint64_t total = h->total_edges;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
    const InstDesc& g = d[inst_of_edge(d, k, i)];
    if (ld_cg(&g.gc[GC_ERR]) & kErrInval) continue;
    const uint64_t j = i - g.edge_base;
    atomicAdd(&g.cnt[g.edges[2 * j]], 1u);
    atomicAdd(&g.cnt[g.edges[2 * j + 1]], 1u);
  }
}

// One CTA per graph: cursors and work items (plan_vertices); the last CTA
// to finish lays the graphs' work items end to end.
__global__ void __launch_bounds__(1024) k_plan_m(BatchHead* __restrict__ h) {
  __shared__ bool s_last;
  InstDesc* d = const_cast<InstDesc*>(descs_of(h));
  const uint32_t k = h->k, b = blockIdx.x;
  if (b >= k) return;
  InstDesc& g = d[b];
  uint32_t nitems = 0, nd = 0;
  const bool dropped = (ld_cg(&g.gc[GC_ERR]) & kErrInval) != 0;
  if (!dropped && g.n > 0) nitems = plan_vertices(g.cnt, g.cursor, g.items, g.V, g.item_records, &nd);
  if (threadIdx.x == 0) {
    g.nitems = nitems;
    g.nd = nd;
    if (!dropped && g.n > 0) g.gc[GC_BATCHES] += 1;
    __threadfence();
    s_last = atomicAdd(&h->plans_done, 1u) == k - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    uint32_t run = 0;
    for (uint32_t j = 0; j < k; j++) {
      d[j].item_base = run;
      run += ld_cg(&d[j].nitems);
    }
    h->total_items = run;
    h->next_item = 0;
  }
}

__global__ void k_scatter_m(const BatchHead* __restrict__ h) {
  const InstDesc* d = descs_of(h);
  const uint32_t k = h->k;
  const uint64_t total = h->total_edges;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
    const InstDesc& g = d[inst_of_edge(d, k, i)];
    if (ld_cg(&g.gc[GC_ERR]) & kErrInval) continue;
    const uint64_t j = i - g.edge_base;
    const uint32_t u = g.edges[2 * j], v = g.edges[2 * j + 1];
    const uint64_t idx = (uint64_t)min(u, v) * g.V + max(u, v);
    const uint32_t pu = atomicAdd(&g.cursor[u], 1u), pv = atomicAdd(&g.cursor[v], 1u);
    g.rec[pu] = idx;
    g.rec[pv] = idx;
    const uint32_t nd = ld_cg(&g.nd);
    if (pu < nd) g.recw[pu] = u;
    if (pv < nd) g.recw[pv] = v;
  }
}

// Persistent CTAs pull work items of all graphs from one counter. The lane
// layout follows the graph of the current item (recomputed when it changes);
// rows stay zero between items, so CTAs move freely between graphs.
__global__ void k_apply_m(BatchHead* __restrict__ h, uint32_t rmax, uint32_t lmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ApplySmem m = apply_smem(smem_raw, rmax, lmax);
  __shared__ uint32_t s_item;
  const InstDesc* d = descs_of(h);
  const uint32_t k = h->k;
  // CTA b starts with item b (CTAs beyond the items leave at once); the
  // counter hands out the rest, counting from the grid size
  const uint32_t total = ld_cg(&h->total_items);
  if (blockIdx.x >= total) return;
  ulonglong2* my_rows = m.rows + threadIdx.x;
  const uint32_t rs = blockDim.x;
  for (uint32_t r = 0; r < rmax; r++) my_rows[r * rs] = make_ulonglong2(0, 0);
  uint32_t cur = kNoneU32;
  ApplyLane l{};
  for (uint32_t it = blockIdx.x; it < total;) {
    const uint32_t j = inst_of_item(d, k, it);
    const InstDesc& g = d[j];
    if (j != cur) {
      cur = j;
      l = apply_lane(g.keys, g.L, g.C, g.D, g.P, g.R, g.ell);
      __syncthreads();  // every thread is done with the previous graph's keys
      load_kchk(m, g.keys, g.L, g.C);
      __syncthreads();
    }
    const uint4 item = g.items[it - ld_cg(&g.item_base)];
    if (item.x == kDirectItem) {
      if (g.long_depth)
        apply_direct<true>(l, g.sketch, g.V, g.W, g.rec + item.y, g.recw + item.y, item.z - item.y, g.L, m);
      else
        apply_direct<false>(l, g.sketch, g.V, g.W, g.rec + item.y, g.recw + item.y, item.z - item.y, g.L, m);
    } else {
      ulonglong2* gb = g.sketch + ((size_t)l.layer * g.V + item.x) * g.W + l.jbase;
      if (g.long_depth)
        apply_item<true>(l, gb, g.rec + item.y, item.z - item.y, item.w != 0, g.L, g.R, m, my_rows, rs);
      else
        apply_item<false>(l, gb, g.rec + item.y, item.z - item.y, item.w != 0, g.L, g.R, m, my_rows, rs);
    }
    // both item paths end with __syncthreads: every thread has read s_item
    if (threadIdx.x == 0) s_item = gridDim.x + atomicAdd(&h->next_item, 1u);
    __syncthreads();
    it = s_item;
  }
}

}  // namespace cupc

using namespace cupc;

struct cupc_batcher {
  uint32_t max_graphs;
  int sms;
  bool use_graph;
  size_t table_bytes;
  BatchHead* dtab;
  BatchHead* htab[2];
  cudaEvent_t used[2];
  int cur;
  cudaStream_t cap_stream;
  struct Exec {
    uint32_t threads, rmax, lmax;
    int apply_grid, apply_smem;
    cudaGraphExec_t exec[2];
  };
  std::vector<Exec> execs;
};

namespace {

bool is_dev(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cudaError_t enqueue(cupc_batcher* b, int slot, const cupc_batcher::Exec& x, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(b->dtab, b->htab[slot], b->table_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const int grid = b->sms * 8;
  k_validate_m<<<grid, 256, 0, s>>>(b->dtab);
  k_count_m<<<grid, 256, 0, s>>>(b->dtab);
  k_plan_m<<<b->max_graphs, 1024, 0, s>>>(b->dtab);
  k_scatter_m<<<grid, 256, 0, s>>>(b->dtab);
  k_apply_m<<<x.apply_grid, x.threads, x.apply_smem, s>>>(b->dtab, x.rmax, x.lmax);
  return cudaGetLastError();
}

cudaError_t get_exec(cupc_batcher* b, uint32_t threads, uint32_t rmax, uint32_t lmax, cupc_batcher::Exec** out) {
  for (auto& x : b->execs)
    if (x.threads == threads && x.rmax == rmax && x.lmax == lmax) {
      *out = &x;
      return cudaSuccess;
    }
  cupc_batcher::Exec x{};
  x.threads = threads;
  x.rmax = rmax;
  x.lmax = lmax;
  x.apply_smem = (int)apply_smem_bytes(rmax, threads, lmax);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_apply_m);
  if (e != cudaSuccess) return e;
  if (fa.maxDynamicSharedSizeBytes < x.apply_smem) {
    e = cudaFuncSetAttribute(k_apply_m, cudaFuncAttributeMaxDynamicSharedMemorySize, x.apply_smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_m, (int)threads, x.apply_smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  x.apply_grid = per_sm * b->sms;
  if (b->use_graph) {
    for (int slot = 0; slot < 2; slot++) {
      cudaGraph_t graph;
      e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return e;
      cudaError_t e2 = enqueue(b, slot, x, b->cap_stream);
      e = cudaStreamEndCapture(b->cap_stream, &graph);
      if (e2 != cudaSuccess) return e2;
      if (e != cudaSuccess) return e;
      e = cudaGraphInstantiate(&x.exec[slot], graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return e;
    }
  }
  b->execs.push_back(x);
  *out = &b->execs.back();
  return cudaSuccess;
}

}  // namespace

extern "C" {

cupc_status cupc_batcher_create(uint32_t max_graphs, int use_cuda_graph, cupc_batcher** out) {
  if (!out || max_graphs == 0 || max_graphs > 4096) return CUPC_EINVAL;
  *out = nullptr;
  cupc_batcher* b = new (std::nothrow) cupc_batcher();
  if (!b) return CUPC_ENOMEM;
  b->max_graphs = max_graphs;
  b->use_graph = use_cuda_graph != 0;
  b->table_bytes = sizeof(BatchHead) + (size_t)max_graphs * sizeof(InstDesc);
  int dev = 0;
  bool ok = cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaMalloc((void**)&b->dtab, b->table_bytes) == cudaSuccess &&
            cudaMallocHost((void**)&b->htab[0], b->table_bytes) == cudaSuccess &&
            cudaMallocHost((void**)&b->htab[1], b->table_bytes) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->used[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->used[1], cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cupc_batcher_destroy(b);
    return CUPC_ENOMEM;
  }
  *out = b;
  return CUPC_OK;
}

cupc_status cupc_batcher_update(cupc_batcher* b, cupc_graph* const* graphs, const uint32_t* const* edges,
                                const int8_t* const* ops, const size_t* n, uint32_t k, cupc_stream stream) {
  if (!b || (k && (!graphs || !edges || !ops || !n)) || k > b->max_graphs) return CUPC_EINVAL;
  if (k == 0) return CUPC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  for (uint32_t i = 0; i < k; i++) {
    if (!graphs[i] || n[i] > graphs[i]->max_batch) return CUPC_EINVAL;
    if (n[i] && (!is_dev(edges[i]) || !is_dev(ops[i]))) return CUPC_EINVAL;
    for (uint32_t j = 0; j < i; j++)
      if (graphs[j] == graphs[i]) return CUPC_EINVAL;
  }
  const int slot = b->cur;
  if (cudaEventSynchronize(b->used[slot]) != cudaSuccess) return CUPC_ECUDA;
  BatchHead* h = b->htab[slot];
  memset(h, 0, sizeof(BatchHead) + (size_t)k * sizeof(InstDesc));
  InstDesc* d = reinterpret_cast<InstDesc*>(h + 1);
  uint64_t base = 0;
  uint32_t threads = 32, rmax = 1, lmax = 1;
  for (uint32_t i = 0; i < k; i++) {
    cupc_graph* g = graphs[i];
    InstDesc& x = d[i];
    x.edges = edges[i];
    x.ops = ops[i];
    x.sketch = g->sketch;
    x.keys = g->keys;
    x.cnt = g->cnt;
    x.cursor = g->cursor;
    x.rec = g->rec;
    x.recw = g->recw;
    x.items = g->items;
    x.gc = g->gc;
    x.edge_base = base;
    x.n = (uint32_t)n[i];
    x.V = g->V;
    x.L = g->L;
    x.C = g->C;
    x.D = g->D;
    x.W = g->W;
    x.P = g->P;
    x.R = g->R;
    x.item_records = g->item_records;
    x.ell = g->ell;
    x.long_depth = g->long_depth ? 1u : 0u;
    base += n[i];
    if ((uint32_t)g->apply_threads > threads) threads = (uint32_t)g->apply_threads;
    if (g->R > rmax) rmax = g->R;
    if (g->L > lmax) lmax = g->L;
  }
  h->k = k;
  h->total_edges = base;
  cupc_batcher::Exec* x = nullptr;
  if (get_exec(b, threads, rmax, lmax, &x) != cudaSuccess) {
    cudaGetLastError();
    return CUPC_ECUDA;
  }
  cudaError_t e = b->use_graph ? cudaGraphLaunch(x->exec[slot], s) : enqueue(b, slot, *x, s);
  if (e != cudaSuccess) return CUPC_ECUDA;
  if (cudaEventRecord(b->used[slot], s) != cudaSuccess) return CUPC_ECUDA;
  b->cur ^= 1;
  // like cupc_update_batch: the next query recovers; the batcher does not
  // follow incremental labels, so a graph in that mode drops them
  for (uint32_t i = 0; i < k; i++) {
    if (!n[i]) continue;
    graphs[i]->dirty = true;
    graphs[i]->forest_stale = true;
    if (graphs[i]->inc && cudaMemsetAsync(graphs[i]->gc + GC_LABELS_VALID, 0, sizeof(uint32_t), s) != cudaSuccess)
      return CUPC_ECUDA;
  }
  return CUPC_OK;
}

void cupc_batcher_destroy(cupc_batcher* b) {
  if (!b) return;
  for (int i = 0; i < 2; i++) {
    if (b->used[i]) cudaEventSynchronize(b->used[i]);
  }
  for (auto& x : b->execs)
    for (int i = 0; i < 2; i++)
      if (x.exec[i]) cudaGraphExecDestroy(x.exec[i]);
  if (b->dtab) cudaFree(b->dtab);
  for (int i = 0; i < 2; i++) {
    if (b->htab[i]) cudaFreeHost(b->htab[i]);
    if (b->used[i]) cudaEventDestroy(b->used[i]);
  }
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

cupc_status cupc_update_batches(cupc_graph* g, const uint32_t* edges, const int8_t* ops, const uint64_t* offsets,
                                size_t k, cupc_stream stream) {
  if (!g || (k && !offsets)) return CUPC_EINVAL;
  if (k == 0) return CUPC_OK;
  for (size_t i = 0; i < k; i++)
    if (offsets[i + 1] < offsets[i]) return CUPC_EINVAL;
  // consecutive batches stored back to back are one batch: sketch addition
  // is XOR, so applying their concatenation equals applying them in order
  const uint64_t first = offsets[0], total = offsets[k] - offsets[0];
  return cupc_update_batch(g, edges + 2 * first, ops + first, total, stream);
}

}  // extern "C"
