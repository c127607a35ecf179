// Batched edge updates into the vertex sketches (App. A.1.1, "The AGM
// Algorithm": an update of edge (u,v) updates every sketch of u and of v;
// Theorem A.2: CameoSketch touches one bucket per column per update).
//
// One chunk of <= max_batch edges goes through five stream-ordered kernels
// (a batch is validated whole by k_validate first, or, when it is one chunk
// that k_count_priv counts, inside k_count_priv):
//   k_count   per-vertex record counts (2 records per edge, one per
//             endpoint); k_count_priv for dense batches on small graphs,
//             through per-CTA shared histograms
//   k_plan_count / k_plan_write
//             exclusive scan over vertex slices -> per-vertex cursors and
//             work items: at most item_records records of one vertex, or
//             16..64 records of vertices with at most 2 (the direct path)
//   k_scatter endpoint records (the edge index u*V+v) grouped by vertex
//             (k_scatter_priv with k_count_priv)
//   k_apply   persistent CTAs, CTA b starting on item b; the CTA stages
//             the item's records 64 at a time with their checksum of every
//             layer (one SplitMix64 per record and layer), then thread
//             (layer r, slot s) takes the multiply-add-shift depth of each
//             record in column s of layer r (slot C owns the deterministic
//             bucket), folds it into shared-memory rows, and finally
//             read-modify-writes only the touched buckets of that vertex in
//             HBM with 16-byte accesses; direct items XOR each bucket
//             straight into HBM.
// XOR is associative and commutative, so the result is bit-identical to
// applying the updates one by one in stream order.
#include "update_dev.cuh"

namespace cupc {

__global__ void k_keys(uint64_t seed, uint64_t* keys, uint32_t n) {
  const uint64_t phi = 0x9E3779B97F4A7C15ull;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    keys[j] = mix64(seed + phi * (uint64_t)(j + 1));
}

cudaError_t launch_keys(cupc_graph* g, cudaStream_t s) {
  k_keys<<<1, 256, 0, s>>>(g->seed, g->keys, (uint32_t)key_words(g->L, g->C));
  return cudaGetLastError();
}

// Problem 1's stream: ((u,v), Delta) with u != v in V and Delta = +-1.
__global__ void k_validate(const uint32_t* __restrict__ edges, const int8_t* __restrict__ ops, size_t n,
                           uint32_t V, uint32_t* gc) {
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t u = edges[2 * i], v = edges[2 * i + 1];
    int8_t op = ops[i];
    bad |= (u >= V) | (v >= V) | (u == v) | ((op != 1) & (op != -1));
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&gc[GC_ERR], kErrInval);
}

cudaError_t launch_validate(cupc_graph* g, const uint32_t* edges, const int8_t* ops, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)g->sms * 8);
  ProfScope ps(g, s, PC_VALIDATE, 1);
  k_validate<<<grid, 256, 0, s>>>(edges, ops, n, g->V, g->gc);
  return cudaGetLastError();
}

__global__ void k_count(const uint32_t* __restrict__ edges, size_t n, uint32_t* cnt, const uint32_t* gc) {
  if (ld_cg(&gc[GC_ERR]) & kErrInval) return;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    atomicAdd(&cnt[edges[2 * i]], 1u);
    atomicAdd(&cnt[edges[2 * i + 1]], 1u);
  }
}

// Dense batches on small graphs (V <= kPrivMaxV, at least kPrivPerVertex
// records per vertex on average): each CTA takes a contiguous slice of the
// batch and counts its endpoints in a shared histogram of all V vertices, so
// the global counters see one atomic per (CTA, vertex) instead of one per
// record.
// With ops (a batch of one chunk) it also validates the batch as k_validate
// does, saving that pass; counts of an invalid batch are cleared by
// k_plan_write.
__global__ void __launch_bounds__(1024) k_count_priv(const uint32_t* __restrict__ edges,
                                                     const int8_t* __restrict__ ops, size_t n, uint32_t V,
                                                     uint32_t* cnt, uint32_t* gc) {
  extern __shared__ uint32_t s_h[];  // V
  if (ld_cg(&gc[GC_ERR]) & kErrInval) return;
  for (uint32_t w = threadIdx.x; w < V; w += blockDim.x) s_h[w] = 0;
  __syncthreads();
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x, lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  bool bad = false;
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const uint32_t u = edges[2 * i], v = edges[2 * i + 1];
    if (ops) {
      const int8_t op = ops[i];
      bad |= (u >= V) | (v >= V) | (u == v) | ((op != 1) & (op != -1));
    }
    if (u < V && v < V) {
      atomicAdd(&s_h[u], 1u);
      atomicAdd(&s_h[v], 1u);
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&gc[GC_ERR], kErrInval);
  __syncthreads();
  for (uint32_t w = threadIdx.x; w < V; w += blockDim.x) {
    const uint32_t c = s_h[w];
    if (c) atomicAdd(&cnt[w], c);
  }
}

// ... and groups them: the CTA counts its slice again, reserves one range of
// each of its vertices' segments (one atomic per vertex), then places each
// record at the range start + its rank in shared memory. Records of a vertex
// land in a different order than with k_scatter; XOR does not see order.
__global__ void __launch_bounds__(1024) k_scatter_priv(const uint32_t* __restrict__ edges, size_t n, uint32_t V,
                                                       uint32_t* cursor, uint64_t* __restrict__ rec,
                                                       uint32_t* __restrict__ recw, const uint32_t* gc) {
  extern __shared__ uint32_t s_h[];  // V counts, then V range starts
  uint32_t* s_base = s_h + V;
  if (ld_cg(&gc[GC_ERR]) & kErrInval) return;
  const uint32_t nd = ld_cg(&gc[GC_NDIRECT]);
  for (uint32_t w = threadIdx.x; w < V; w += blockDim.x) s_h[w] = 0;
  __syncthreads();
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x, lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    atomicAdd(&s_h[edges[2 * i]], 1u);
    atomicAdd(&s_h[edges[2 * i + 1]], 1u);
  }
  __syncthreads();
  for (uint32_t w = threadIdx.x; w < V; w += blockDim.x) {
    const uint32_t c = s_h[w];
    if (c) s_base[w] = atomicAdd(&cursor[w], c);
    s_h[w] = 0;
  }
  __syncthreads();
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const uint32_t u = edges[2 * i], v = edges[2 * i + 1];
    const uint64_t idx = (uint64_t)min(u, v) * V + max(u, v);
    const uint32_t pu = s_base[u] + atomicAdd(&s_h[u], 1u), pv = s_base[v] + atomicAdd(&s_h[v], 1u);
    rec[pu] = idx;
    rec[pv] = idx;
    if (pu < nd) recw[pu] = u;
    if (pv < nd) recw[pv] = v;
  }
}

// ---- incremental labels (cupc_set_incremental). After a complete
// recovery the labels are the components of the graph; with a valid stream
// (inserts of absent edges, deletes of present ones) an insert can only
// merge two components, and deleting an edge outside a spanning forest of
// the graph cannot split one. So a batch keeps the labels exact by merging
// the endpoint labels of its inserts (union-find over labels, the larger
// root under the smaller, so a root is its component's minimum vertex id,
// the label a recovery gives). Each insert whose link succeeds joins two
// components: it becomes a forest edge (fadd, with a hash table of ids), so
// the recovered forest plus these edges stays a spanning forest of the
// graph. A deleted forest edge of either kind is marked (fdead, fadd_dead)
// and sets GC_WARM: the next recovery starts from the fragments of the
// remaining forest. In a batch that both merges and deletes, an edge the
// batch inserts (a merge) and then deletes is found by a second lookup pass
// (k_incr_dead) once all of the batch's merges are recorded.
__device__ __forceinline__ uint32_t inc_find(uint32_t* par, uint32_t x, uint32_t V) {
  for (uint32_t k = 0; k < V; k++) {  // a path is shorter than V
    const uint32_t y = ld_cg(&par[x]);
    if (y == x) break;
    const uint32_t z = ld_cg(&par[y]);
    if (z != y) par[x] = z;  // halving: only ever to an ancestor
    x = y;
  }
  return x;
}

// Home slot of an edge id in the merge-edge table (Fibonacci hashing).
__device__ __forceinline__ uint32_t ftab_home(uint64_t id, uint32_t bits) {
  return (uint32_t)((id * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

struct IncArgs {
  const uint32_t* label;
  uint32_t* ipar;
  const uint64_t* forest_sorted;
  uint8_t* fdead;
  uint64_t* fadd;
  uint8_t* fadd_dead;
  unsigned long long* ftab;
  uint32_t* ftab_pos;
  uint32_t ftab_bits, V;
  uint32_t* gc;
};

__global__ void k_incr(const uint32_t* __restrict__ edges, const int8_t* __restrict__ ops, size_t n, IncArgs a) {
  uint32_t* gc = a.gc;
  if ((ld_cg(&gc[GC_ERR]) & kErrInval) || !ld_cg(&gc[GC_LABELS_VALID])) return;
  const uint32_t V = a.V, nf = ld_cg(&gc[GC_NSORTED]), nadd = ld_cg(&gc[GC_NFADD]);
  const uint32_t mask = (1u << a.ftab_bits) - 1u;
  bool del = false, merged = false, cut = false, warm = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t u = edges[2 * i], v = edges[2 * i + 1];
    const uint64_t id = (uint64_t)min(u, v) * V + max(u, v);
    if (ops[i] < 0) {
      del = true;
      uint32_t lo = 0, hi = nf;  // first recovered forest id >= id
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a.forest_sorted[mid] < id)
          lo = mid + 1;
        else
          hi = mid;
      }
      if (lo < nf && a.forest_sorted[lo] == id) {
        a.fdead[lo] = 1;
        warm = true;
      } else if (nadd) {  // a forest edge added by a merge?
        uint32_t sl = ftab_home(id, a.ftab_bits);
        for (uint32_t k = 0; k <= mask; k++, sl = (sl + 1) & mask) {
          const unsigned long long key = ld_cg((const uint64_t*)&a.ftab[sl]);
          if (key == 0ull) break;
          if (key == (unsigned long long)id) {
            const uint32_t j = ld_cg(&a.ftab_pos[sl]);
            if (j < V) a.fadd_dead[j] = 1;
            warm = true;
            break;
          }
        }
      }
    } else {
      uint32_t x = a.label[u], y = a.label[v];
      for (uint32_t k = 0; k < (1u << 20); k++) {  // bounded retries; giving up clears the labels
        x = inc_find(a.ipar, x, V);
        y = inc_find(a.ipar, y, V);
        if (x == y) break;
        if (x > y) {
          const uint32_t t = x;
          x = y;
          y = t;
        }
        if (atomicCAS(&a.ipar[y], y, x) == y) {
          merged = true;
          // this insert joined two components: record it as a forest edge
          const uint32_t j = atomicAdd(&gc[GC_NFADD], 1u);
          bool placed = false;
          if (j < V) {
            a.fadd[j] = id;
            a.fadd_dead[j] = 0;
            uint32_t sl = ftab_home(id, a.ftab_bits);
            for (uint32_t q = 0; q <= mask; q++, sl = (sl + 1) & mask) {
              const unsigned long long prev = atomicCAS(&a.ftab[sl], 0ull, (unsigned long long)id);
              if (prev == 0ull || prev == (unsigned long long)id) {
                a.ftab_pos[sl] = j;
                placed = true;
                break;
              }
            }
          }
          if (!placed) cut = true;  // cannot happen with a valid stream
          break;
        }
        if (k + 1 == (1u << 20)) cut = true;
      }
    }
  }
  if (__any_sync(0xffffffffu, cut) && (threadIdx.x & 31) == 0) gc[GC_LABELS_VALID] = 0;
  if (__any_sync(0xffffffffu, del) && (threadIdx.x & 31) == 0) gc[GC_BATCH_DEL] = 1;
  if (__any_sync(0xffffffffu, merged) && (threadIdx.x & 31) == 0) gc[GC_BATCH_MERGE] = 1;
  if (__any_sync(0xffffffffu, warm) && (threadIdx.x & 31) == 0) gc[GC_WARM] = 1;
}

// A batch that both merges and deletes: k_incr looked each delete up in the
// merge edges recorded before the batch, so an edge this batch inserted (and
// recorded as a merge) and then deleted again, in stream order, is looked up
// again here, once every merge of the batch is in the table.
__global__ void k_incr_dead(const uint32_t* __restrict__ edges, const int8_t* __restrict__ ops, size_t n,
                            IncArgs a) {
  uint32_t* gc = a.gc;
  if ((ld_cg(&gc[GC_ERR]) & kErrInval) || !ld_cg(&gc[GC_LABELS_VALID]) || !ld_cg(&gc[GC_BATCH_MERGE]) ||
      !ld_cg(&gc[GC_BATCH_DEL]))
    return;
  const uint32_t V = a.V, mask = (1u << a.ftab_bits) - 1u;
  bool warm = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (ops[i] >= 0) continue;
    const uint32_t u = edges[2 * i], v = edges[2 * i + 1];
    const uint64_t id = (uint64_t)min(u, v) * V + max(u, v);
    uint32_t sl = ftab_home(id, a.ftab_bits);
    for (uint32_t k = 0; k <= mask; k++, sl = (sl + 1) & mask) {
      const unsigned long long key = ld_cg((const uint64_t*)&a.ftab[sl]);
      if (key == 0ull) break;
      if (key == (unsigned long long)id) {
        const uint32_t j = ld_cg(&a.ftab_pos[sl]);
        if (j < V) a.fadd_dead[j] = 1;
        warm = true;
        break;
      }
    }
  }
  if (__any_sync(0xffffffffu, warm) && (threadIdx.x & 31) == 0) gc[GC_WARM] = 1;
}

// Labels after the merges: every vertex takes its label's root. Merges are
// exact whatever else the batch did: a delete can only split components,
// and one that removed a forest edge has set GC_WARM, so the next query
// recovers from the fragments of the remaining forest.
__global__ void k_incr_finish(uint32_t* label, uint32_t* ipar, uint32_t V, uint32_t* gc) {
  if (!ld_cg(&gc[GC_LABELS_VALID]) || !ld_cg(&gc[GC_BATCH_MERGE])) return;
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < V; w += gridDim.x * blockDim.x)
    label[w] = inc_find(ipar, label[w], V);
}

cudaError_t launch_incremental(cupc_graph* g, const uint32_t* edges, const int8_t* ops, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (g->sort_pending) {  // the forest of the last recovery, which this batch's deletes look up
    cudaError_t e = launch_forest_sort(g, s);
    if (e != cudaSuccess) return e;
    g->sort_pending = false;
  }
  cudaError_t e = cudaMemsetAsync(g->gc + GC_BATCH_DEL, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->gc + GC_BATCH_MERGE, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  IncArgs a;
  a.label = g->label;
  a.ipar = g->ipar;
  a.forest_sorted = g->forest_sorted;
  a.fdead = g->fdead;
  a.fadd = g->fadd;
  a.fadd_dead = g->fadd_dead;
  a.ftab = (unsigned long long*)g->ftab;
  a.ftab_pos = g->ftab_pos;
  a.ftab_bits = g->ftab_bits;
  a.V = g->V;
  a.gc = g->gc;
  const int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)g->sms * 8);
  k_incr<<<grid, 256, 0, s>>>(edges, ops, n, a);
  k_incr_dead<<<grid, 256, 0, s>>>(edges, ops, n, a);
  k_incr_finish<<<(int)std::min<size_t>((g->V + 255) / 256, (size_t)g->sms * 4), 256, 0, s>>>(g->label, g->ipar,
                                                                                                g->V, g->gc);
  return cudaGetLastError();
}

// Work plan of one chunk over many CTAs, in two launches that never wait on
// one another. The vertices are cut into slices of 256 * vpt; slice b is
// planned by CTA b. Kinds of vertices and the layout of records and items
// are those of plan_vertices: direct-path vertices (<= kDirectMax records)
// first in rec, then fold vertices, whose records are cut into items of
// item_records; direct items of kDirectItemRecords follow the fold items.
//
// k_plan_count: per-slice totals {fold records, direct records, fold items}.
__global__ void __launch_bounds__(256) k_plan_count(const uint32_t* __restrict__ cnt, uint32_t V, uint32_t vpt,
                                                    uint32_t item_records, uint4* part, const uint32_t* gc) {
  __shared__ uint32_t sw[3][32];
  if (ld_cg(&gc[GC_ERR]) & kErrInval) return;
  const uint32_t lo = blockIdx.x * blockDim.x * vpt, hi = min(V, lo + blockDim.x * vpt);
  uint32_t v[3] = {0, 0, 0};
  for (uint32_t w = lo + threadIdx.x; w < hi; w += blockDim.x) {
    const uint32_t c = cnt[w];
    if (c > kDirectMax) {
      v[0] += c;
      v[2] += (c + item_records - 1) / item_records;
    } else {
      v[1] += c;
    }
  }
  uint32_t e[3], t[3];
  block_scan3(v, e, t, sw);
  if (threadIdx.x == 0) part[blockIdx.x] = make_uint4(t[0], t[1], t[2], 0u);
}

// k_plan_write: CTA b adds up the totals of slices < b (its offsets) and of
// all slices (direct records nd, fold items), then scans its slice 256
// vertices at a time, writing cursors and fold items; every CTA writes a
// share of the direct items. Resets cnt for the next chunk.
__global__ void __launch_bounds__(256) k_plan_write(uint32_t* cnt, uint32_t* cursor, uint4* items, uint32_t V,
                                                    uint32_t vpt, uint32_t item_records, const uint4* __restrict__ part,
                                                    uint32_t apply_ctas, uint32_t* gc) {
  __shared__ uint32_t sw[3][32];
  const uint32_t nb = gridDim.x, b = blockIdx.x;
  if (ld_cg(&gc[GC_ERR]) & kErrInval) {  // a dropped batch may have counted: start clean
    const uint32_t lo = b * blockDim.x * vpt, hi = min(V, lo + blockDim.x * vpt);
    for (uint32_t w = lo + threadIdx.x; w < hi; w += blockDim.x) cnt[w] = 0;
    return;
  }
  // offsets of this slice and the grand totals
  uint32_t before[3] = {0, 0, 0}, all[3] = {0, 0, 0};
  for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
    const uint4 p = part[j];
    all[0] += p.x;
    all[1] += p.y;
    all[2] += p.z;
    if (j < b) {
      before[0] += p.x;
      before[1] += p.y;
      before[2] += p.z;
    }
  }
  uint32_t e[3], tb[3], ta[3];
  block_scan3(before, e, tb, sw);
  block_scan3(all, e, ta, sw);
  const uint32_t nd = ta[1], nfold = ta[2];
  uint32_t carry[3] = {nd + tb[0], tb[1], tb[2]};  // next fold record, direct record, fold item
  const uint32_t lo = b * blockDim.x * vpt, hi = min(V, lo + blockDim.x * vpt);
  for (uint32_t base = lo; base < hi; base += blockDim.x) {
    const uint32_t w = base + threadIdx.x;
    const uint32_t c = w < hi ? cnt[w] : 0;
    const bool fold = c > kDirectMax;
    const uint32_t ni = fold ? (c + item_records - 1) / item_records : 0;
    const uint32_t v[3] = {fold ? c : 0, fold ? 0 : c, ni};
    uint32_t t[3];
    block_scan3(v, e, t, sw);
    if (w < hi) {
      cnt[w] = 0;
      if (fold) {
        const uint32_t pf = carry[0] + e[0], pi = carry[2] + e[2];
        cursor[w] = pf;
        for (uint32_t q = 0; q < ni; q++) {
          const uint32_t bg = pf + q * item_records;
          items[pi + q] = make_uint4(w, bg, min(pf + c, bg + item_records), ni == 1 ? 1u : 0u);
        }
      } else {
        cursor[w] = carry[1] + e[1];
      }
    }
#pragma unroll
    for (int k = 0; k < 3; k++) carry[k] += t[k];
  }
  // direct items: about two per apply CTA, of kDirectItemMin..kDirectItemRecords
  // records (so at most max(2 * apply_ctas + 1, nd / kDirectItemRecords + 1))
  const uint32_t dsz = min(kDirectItemRecords, max(kDirectItemMin, (nd + 2 * apply_ctas - 1) / (2 * apply_ctas)));
  const uint32_t ndi = (nd + dsz - 1) / dsz;
  for (uint32_t q = b * blockDim.x + threadIdx.x; q < ndi; q += nb * blockDim.x)
    items[nfold + q] = make_uint4(kDirectItem, q * dsz, min(nd, (q + 1) * dsz), 0u);
  if (b == 0 && threadIdx.x == 0) {
    gc[GC_NITEMS] = nfold + ndi;
    gc[GC_NDIRECT] = nd;
    gc[GC_NEXT_ITEM] = 0;
    gc[GC_BATCHES] += 1;
  }
}

// Slice width of the plan kernels: at most kPlanSlices slices.
uint32_t plan_vpt(uint32_t V) {
  const uint32_t per = 256u * kPlanSlices;
  return std::max(1u, (V + per - 1) / per);
}

__global__ void k_scatter(const uint32_t* __restrict__ edges, size_t n, uint32_t V, uint32_t* cursor,
                          uint64_t* __restrict__ rec, uint32_t* __restrict__ recw, const uint32_t* gc) {
  if (ld_cg(&gc[GC_ERR]) & kErrInval) return;
  const uint32_t nd = ld_cg(&gc[GC_NDIRECT]);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t u = edges[2 * i], v = edges[2 * i + 1];
    uint32_t a = min(u, v), b = max(u, v);
    uint64_t idx = (uint64_t)a * V + b;
    const uint32_t pu = atomicAdd(&cursor[u], 1u), pv = atomicAdd(&cursor[v], 1u);
    rec[pu] = idx;
    rec[pv] = idx;
    if (pu < nd) recw[pu] = u;
    if (pv < nd) recw[pv] = v;
  }
}

// Fold the records of one work item into the sketches of its vertex (see
// apply_item); persistent CTAs pull work items from a counter. kExcl: a
// vertex with a single item writes back by load and store, else every
// write-back is by XOR atomics (the launch picks by records per vertex).
template <bool kLong, bool kExcl>
__global__ void k_apply(ulonglong2* __restrict__ sketch, const uint64_t* __restrict__ keys,
                        const uint64_t* __restrict__ rec, const uint32_t* __restrict__ recw,
                        const uint4* __restrict__ items, uint32_t* gc, uint32_t V, uint32_t L, uint32_t C,
                        uint32_t D, uint32_t W, uint32_t P, uint32_t R, uint32_t ell) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ApplySmem m = apply_smem(smem_raw, R, L);
  __shared__ uint32_t s_item;

  if (ld_cg(&gc[GC_ERR]) & kErrInval) return;
  // CTA b starts with item b; CTAs beyond the items leave before touching
  // the item counter (a small batch would otherwise have every CTA of the
  // grid queue on one address); a CTA that finishes takes the next item
  // from the counter, which counts from the grid size
  const uint32_t nitems = ld_cg(&gc[GC_NITEMS]);
  if (blockIdx.x >= nitems) return;
  const ApplyLane l = apply_lane(keys, L, C, D, P, R, ell);
  load_kchk(m, keys, L, C);
  ulonglong2* my_rows = m.rows + threadIdx.x;
  const uint32_t rs = blockDim.x;
  for (uint32_t d = 0; d < R; d++) my_rows[d * rs] = make_ulonglong2(0, 0);
  __syncthreads();

  for (uint32_t it = blockIdx.x; it < nitems;) {
    const uint4 item = items[it];
    if (item.x == kDirectItem) {
      apply_direct<kLong>(l, sketch, V, W, rec + item.y, recw + item.y, item.z - item.y, L, m);
    } else {
      ulonglong2* gb = sketch + ((size_t)l.layer * V + item.x) * W + l.jbase;
      apply_item<kLong>(l, gb, rec + item.y, item.z - item.y, kExcl && item.w != 0, L, R, m, my_rows, rs);
    }
    // both item paths end with __syncthreads: every thread has read s_item
    if (threadIdx.x == 0) s_item = gridDim.x + atomicAdd(&gc[GC_NEXT_ITEM], 1u);
    __syncthreads();
    it = s_item;
  }
}

// The dynamic shared-memory limit of k_apply is process-wide: only ever
// raise it, so that a graph created later never shrinks it below what an
// earlier graph's launches need.
cudaError_t raise_apply_smem_limit(int bytes) {
  const void* fns[4] = {(const void*)k_apply<false, false>, (const void*)k_apply<true, false>,
                        (const void*)k_apply<false, true>, (const void*)k_apply<true, true>};
  for (const void* f : fns) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    if (fa.maxDynamicSharedSizeBytes >= bytes) continue;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t setup_update(cupc_graph* g) {
  // the shared histograms of the dense-batch grouping (fixed maximum sizes)
  cudaError_t e = cudaFuncSetAttribute(k_count_priv, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * kPrivMaxV);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_scatter_priv, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * kPrivMaxV);
  if (e != cudaSuccess) return e;
  g->P = 1;
  while (g->P < g->C + 1) g->P <<= 1;
  g->R = g->D < kSmemRows ? g->D : kSmemRows;
  g->ell = hash_bits(g->V);
  g->long_depth = g->ell < g->D - 1 || g->D - 1 > 32;
  g->item_records = kDefaultItemRecords;
  g->apply_cps = 0;
  g->apply_threads = (int)(((g->L * g->P) + 31) / 32 * 32);
  return configure_apply(g);
}

// Shared memory and persistent grid of k_apply for the given tunables.
cudaError_t apply_config(const cupc_graph* g, uint32_t item_records, uint32_t R, uint32_t cps, int* smem, int* grid) {
  *smem = (int)apply_smem_bytes(R, (uint32_t)g->apply_threads, g->L);
  cudaError_t e = raise_apply_smem_limit(*smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm,
                                                    g->long_depth ? k_apply<true, false> : k_apply<false, false>,
                                                    g->apply_threads, *smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (cps && (int)cps < per_sm) per_sm = (int)cps;
  *grid = per_sm * g->sms;
  return cudaSuccess;
}

// ... and for the graph's default tunables.
cudaError_t configure_apply(cupc_graph* g) {
  return apply_config(g, g->item_records, g->R, g->apply_cps, &g->apply_smem, &g->apply_grid);
}

cudaError_t launch_update_chunk(cupc_graph* g, const uint32_t* edges, size_t n, cudaStream_t s,
                                const int8_t* validate_ops) {
  if (n == 0) return cudaSuccess;
  // the setting of this batch size's bucket, else the graph's default
  uint32_t ir = g->item_records, R = g->R;
  int smem = g->apply_smem, grid_max = g->apply_grid;
  const cupc_graph::ApplyTune& t = g->tune_b[tune_bucket(n)];
  if (t.set) {
    ir = t.item_records;
    R = t.R;
    smem = t.smem;
    grid_max = t.grid;
  }
  const int agrid = (int)std::min<size_t>(std::min<size_t>((size_t)grid_max, 2 * n), kPlanGridCap);
  int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)g->sms * 8);
  // dense batch on a small graph: group through shared histograms (and
  // validate there); else validate in a pass of its own
  const int pgrid = (int)std::min<size_t>((size_t)g->sms, 2 * n / ((size_t)kPrivPerVertex * g->V));
  const bool priv = g->V <= kPrivMaxV && pgrid >= (int)kPrivMinCtas;
  if (!priv && validate_ops) {
    cudaError_t e = launch_validate(g, edges, validate_ops, n, s);
    if (e != cudaSuccess) return e;
  }
  {
    ProfScope ps(g, s, PC_GROUP, 4);
    if (priv)
      k_count_priv<<<pgrid, 1024, 4 * g->V, s>>>(edges, validate_ops, n, g->V, g->cnt, g->gc);
    else
      k_count<<<grid, 256, 0, s>>>(edges, n, g->cnt, g->gc);
    const uint32_t vpt = plan_vpt(g->V), nb = (g->V + 256 * vpt - 1) / (256 * vpt);
    k_plan_count<<<nb, 256, 0, s>>>(g->cnt, g->V, vpt, ir, g->part, g->gc);
    k_plan_write<<<nb, 256, 0, s>>>(g->cnt, g->cursor, g->items, g->V, vpt, ir, g->part, (uint32_t)agrid, g->gc);
    if (priv)
      k_scatter_priv<<<pgrid, 1024, 8 * g->V, s>>>(edges, n, g->V, g->cursor, g->rec, g->recw, g->gc);
    else
      k_scatter<<<grid, 256, 0, s>>>(edges, n, g->V, g->cursor, g->rec, g->recw, g->gc);
  }
  ProfScope ps(g, s, PC_APPLY, 1);
  // the bucket's write-back mode; by default load-then-store for a vertex's
  // single item when the chunk averages fewer than kExclRecords endpoint
  // records per vertex (most touched rows then hold one or two records)
  const uint32_t wb = g->wb_b[tune_bucket(n)];
  const bool excl = wb == CUPC_WRITEBACK_AUTO ? 2 * n < (size_t)kExclRecords * g->V : wb == CUPC_WRITEBACK_LOAD_STORE;
  auto kern = g->long_depth ? (excl ? k_apply<true, true> : k_apply<true, false>)
                            : (excl ? k_apply<false, true> : k_apply<false, false>);
  kern<<<agrid, g->apply_threads, smem, s>>>(g->sketch, g->keys, g->rec, g->recw, g->items, g->gc, g->V, g->L, g->C,
                                              g->D, g->W, g->P, R, g->ell);
  return cudaGetLastError();
}

}  // namespace cupc

extern "C" cupc_status cupc_build_info(int* binary_version, int* ptx_version) {
  if (!binary_version || !ptx_version) return CUPC_EINVAL;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, (const void*)cupc::k_apply<false, false>) != cudaSuccess) {
    cudaGetLastError();
    return CUPC_ECUDA;
  }
  *binary_version = fa.binaryVersion;
  *ptx_version = fa.ptxVersion;
  return CUPC_OK;
}
