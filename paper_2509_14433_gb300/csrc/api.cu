// C-ABI of libcupc (declared in include/cupc.h): argument checks, workspace
// layout, host-buffer staging and the order of the device work. No compute
// happens here; every step of the path runs in the kernels of update.cu and
// recover.cu.
#include <stdlib.h>
#include <string.h>

#include <new>

#include "common.cuh"

using namespace cupc;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

uint32_t ceil_log2(uint32_t V) {
  uint32_t lg = 0;
  while (((uint64_t)1 << lg) < (uint64_t)V) lg++;
  return lg < 1 ? 1 : lg;
}

struct Dims {
  uint32_t V, L, C, D, W, max_batch, max_pairs;
  bool ok;
};

Dims derive(uint32_t V, const cupc_params* p) {
  Dims d{};
  d.ok = false;
  if (V < 2 || V > kMaxVertices) return d;
  uint32_t lg = ceil_log2(V);
  d.V = V;
  d.L = (p && p->rounds) ? p->rounds : lg + 2;
  d.C = (p && p->columns) ? p->columns : 7;
  d.D = (p && p->rows) ? p->rows : 2 * lg;
  d.max_batch = (p && p->max_batch) ? p->max_batch : (1u << 20);
  d.max_pairs = d.max_batch;
  if (d.C > 31 || d.D > 63 || d.D < 1 || d.L < 1 || d.L > 64) return d;
  d.W = 1 + d.C * d.D;
  if (d.W > 32 * kWarpBuckets) return d;
  uint32_t P = 1;  // apply threads per layer: the columns and the checksum lane
  while (P < d.C + 1) P <<= 1;
  if (d.L * P > 1024) return d;  // one apply CTA holds every (layer, lane)
  // the edge index u*V+v must fit the 64-bit bucket word; record offsets are u32
  if ((uint64_t)d.max_batch * 2 >= 0xFFFFFFFFull) return d;
  d.ok = true;
  return d;
}

// Byte offsets of every device array inside the workspace.
struct Layout {
  size_t sketch, keys, gc, cnt, cursor, rec, recw, items, part, stage_edges, stage_ops, stage_edges1, stage_ops1,
      label, parent, minv, rcnt, roff,
      perm, permb, pcount, final_, merged, best, best2, cand, forest, forest_sorted, acc, log_ids, log_live,
      log_ncand, hlist, ipar, fdead, fadd, fadd_dead, ftab, ftab_pos, total;
};

// Slots of the incremental merge-edge table: at least 2V, a power of two.
uint32_t ftab_bits(uint32_t V) {
  const uint32_t b = ceil_log2(V) + 1;
  return b < 6 ? 6 : b;
}

Layout layout(const Dims& d) {
  Layout l{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  const size_t V = d.V, B = d.max_batch;
  const size_t nitems = 4 * B / kMinItemRecords + (V < 2 * B ? V : 2 * B) + 2 * kPlanGridCap + 1;
  l.sketch = take((size_t)d.L * V * d.W * sizeof(ulonglong2));
  l.keys = take(key_words(d.L, d.C) * sizeof(uint64_t));
  l.gc = take(GC_SLOTS * sizeof(uint32_t));
  l.cnt = take(V * 4);
  l.cursor = take(V * 4);
  l.rec = take(2 * B * 8);
  l.recw = take(2 * B * 4);
  l.items = take(nitems * sizeof(uint4));
  l.part = take(kPlanSlices * sizeof(uint4));
  l.stage_edges = take(2 * B * 4);
  l.stage_ops = take(B);
  l.stage_edges1 = take(2 * B * 4);
  l.stage_ops1 = take(B);
  l.label = take(V * 4);
  l.parent = take(V * 4);
  l.minv = take(V * 4);
  l.rcnt = take(V * 4);
  l.roff = take(V * 4);
  l.perm = take(V * 4);
  l.permb = take(V * 4);
  l.pcount = take(V * 4);
  l.final_ = take(V);
  l.merged = take(V);
  l.best = take(V * 8);
  l.best2 = take(V * 8);
  l.cand = take(V * 16);
  l.forest = take(V * 8);
  l.forest_sorted = take(V * 8);
  l.acc = take(V * d.W * sizeof(ulonglong2));
  l.log_ids = take((size_t)d.L * V * 8);
  l.log_live = take(d.L * 4);
  l.log_ncand = take(d.L * 4);
  l.hlist = take(kSmallHook * sizeof(ulonglong2));
  l.ipar = take(V * 4);
  l.fdead = take(V);
  l.fadd = take(V * 8);
  l.fadd_dead = take(V);
  const size_t T = (size_t)1 << ftab_bits(d.V);
  l.ftab = take(T * 8);
  l.ftab_pos = take(T * 4);
  l.total = off;
  return l;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cupc_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return CUPC_OK;
  if (e == cudaErrorMemoryAllocation) return CUPC_ENOMEM;
  return CUPC_ECUDA;
}

#define CUPC_TRY(x)                        \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return from_cuda(e_); \
  } while (0)

// Incremental mode sorts the forest of a recovery before the next update
// batch, whose deletes look it up (k_incr): the sort stays off the query's
// path. The recovery returns at once while the labels are valid, and the
// sort while the forest is sorted.
cupc_status recover_if_dirty(cupc_graph* g, cudaStream_t s) {
  if (!g->dirty) return CUPC_OK;
  CUPC_TRY(launch_recover(g, s));
  if (g->inc) g->sort_pending = true;
  g->dirty = false;
  return CUPC_OK;
}

// Updates invalidate the forest; in incremental mode a change the labels
// cannot follow (a reset, imported sketches) clears them.
cupc_status mark_updated(cupc_graph* g, cudaStream_t s, bool labels_kept) {
  g->dirty = true;
  g->forest_stale = true;
  if (g->inc && !labels_kept) CUPC_TRY(cudaMemsetAsync(g->gc + GC_LABELS_VALID, 0, sizeof(uint32_t), s));
  return CUPC_OK;
}

}  // namespace

extern "C" {

size_t cupc_workspace_bytes(uint32_t V, const cupc_params* params) {
  Dims d = derive(V, params);
  if (!d.ok) return 0;
  return layout(d).total;
}

cupc_status cupc_init(uint32_t V, uint64_t seed, const cupc_params* params, void* workspace, cupc_stream stream,
                      cupc_graph** out) {
  if (!out) return CUPC_EINVAL;
  *out = nullptr;
  Dims d = derive(V, params);
  if (!d.ok) return CUPC_EINVAL;
  if (workspace && ((uintptr_t)workspace % kAlign)) return CUPC_EINVAL;
  Layout l = layout(d);
  cupc_graph* g = new (std::nothrow) cupc_graph();
  if (!g) return CUPC_ENOMEM;
  g->V = d.V;
  g->L = d.L;
  g->C = d.C;
  g->D = d.D;
  g->W = d.W;
  g->seed = seed;
  g->max_batch = d.max_batch;
  g->max_pairs = d.max_pairs;
  g->ws_bytes = l.total;
  g->owns_ws = workspace == nullptr;
  g->last_recovery = CUPC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  auto fail = [&](cupc_status st) {
    if (g->owns_ws && g->ws) cudaFree(g->ws);
    delete g;
    return st;
  };
  if (cudaGetDevice(&g->device) != cudaSuccess) return fail(CUPC_ECUDA);
  if (cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess)
    return fail(CUPC_ECUDA);
  if (g->owns_ws) {
    cudaError_t e = cudaMalloc(&g->ws, l.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(e == cudaErrorMemoryAllocation ? CUPC_ENOMEM : CUPC_ECUDA);
    }
  } else {
    g->ws = workspace;
  }
  char* b = (char*)g->ws;
  g->sketch = (ulonglong2*)(b + l.sketch);
  g->keys = (uint64_t*)(b + l.keys);
  g->gc = (uint32_t*)(b + l.gc);
  g->cnt = (uint32_t*)(b + l.cnt);
  g->cursor = (uint32_t*)(b + l.cursor);
  g->rec = (uint64_t*)(b + l.rec);
  g->recw = (uint32_t*)(b + l.recw);
  g->items = (uint4*)(b + l.items);
  g->part = (uint4*)(b + l.part);
  g->stage_edges = (uint32_t*)(b + l.stage_edges);
  g->stage_ops = (int8_t*)(b + l.stage_ops);
  g->stage_edges1 = (uint32_t*)(b + l.stage_edges1);
  g->stage_ops1 = (int8_t*)(b + l.stage_ops1);
  g->stage_pairs = g->stage_edges;
  g->stage_out = (uint8_t*)g->stage_ops;
  g->label = (uint32_t*)(b + l.label);
  g->parent = (uint32_t*)(b + l.parent);
  g->minv = (uint32_t*)(b + l.minv);
  g->rcnt = (uint32_t*)(b + l.rcnt);
  g->roff = (uint32_t*)(b + l.roff);
  g->perm = (uint32_t*)(b + l.perm);
  g->permb = (uint32_t*)(b + l.permb);
  g->pcount = (uint32_t*)(b + l.pcount);
  g->final_ = (uint8_t*)(b + l.final_);
  g->merged = (uint8_t*)(b + l.merged);
  g->best = (uint64_t*)(b + l.best);
  g->best2 = (uint64_t*)(b + l.best2);
  g->cand = (ulonglong2*)(b + l.cand);
  g->forest = (uint64_t*)(b + l.forest);
  g->forest_sorted = (uint64_t*)(b + l.forest_sorted);
  g->acc = (ulonglong2*)(b + l.acc);
  g->log_ids = (uint64_t*)(b + l.log_ids);
  g->log_live = (uint32_t*)(b + l.log_live);
  g->log_ncand = (uint32_t*)(b + l.log_ncand);
  g->hlist = (ulonglong2*)(b + l.hlist);
  g->ipar = (uint32_t*)(b + l.ipar);
  g->fdead = (uint8_t*)(b + l.fdead);
  g->fadd = (uint64_t*)(b + l.fadd);
  g->fadd_dead = (uint8_t*)(b + l.fadd_dead);
  g->ftab = (uint64_t*)(b + l.ftab);
  g->ftab_pos = (uint32_t*)(b + l.ftab_pos);
  g->ftab_bits = ftab_bits(d.V);
  if (setup_update(g) != cudaSuccess || setup_recover(g) != cudaSuccess) {
    cudaGetLastError();
    return fail(CUPC_ECUDA);
  }
  if (cudaMemsetAsync(g->ws, 0, l.total, s) != cudaSuccess || launch_keys(g, s) != cudaSuccess) {
    cudaGetLastError();
    return fail(CUPC_ECUDA);
  }
  // the empty graph: every vertex its own component, recovery exact
  g->dirty = true;
  g->forest_stale = true;
  *out = g;
  return CUPC_OK;
}

cupc_status cupc_reset(cupc_graph* g, cupc_stream stream) {
  if (!g) return CUPC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CUPC_TRY(cudaMemsetAsync(g->sketch, 0, (size_t)g->L * g->V * g->W * sizeof(ulonglong2), s));
  g->imported = false;
  return mark_updated(g, s, false);
}

// The copy stream and slot events of host-input staging, made on first use.
cudaError_t ensure_copy_stream(cupc_graph* g) {
  if (g->copy_stream) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; k++) {
    e = cudaEventCreateWithFlags(&g->slot_ready[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->slot_free[k], cudaEventDisableTiming);
  }
  return e;
}

// After the last kernel on s that reads staging slot k: a later copy into
// slot k on the copy stream waits for this point.
cudaError_t mark_slot_free(cupc_graph* g, int k, cudaStream_t s) {
  cudaError_t e = ensure_copy_stream(g);  // so that a first async copy sees this use
  return e == cudaSuccess ? cudaEventRecord(g->slot_free[k], s) : e;
}

cupc_status cupc_update_batch(cupc_graph* g, const uint32_t* edges, const int8_t* ops, size_t n,
                              cupc_stream stream) {
  if (!g) return CUPC_EINVAL;
  if (n == 0) return CUPC_OK;
  if (!edges || !ops) return CUPC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t B = g->max_batch;
  const bool dev_e = is_device_ptr(edges), dev_o = is_device_ptr(ops);
  if (dev_e && dev_o) {
    if (n <= B) {
      CUPC_TRY(launch_update_chunk(g, edges, n, s, ops));  // validated on the way
    } else {
      CUPC_TRY(launch_validate(g, edges, ops, n, s));
      for (size_t i = 0; i < n; i += B) CUPC_TRY(launch_update_chunk(g, edges + 2 * i, (n - i < B ? n - i : B), s));
    }
    if (g->inc) CUPC_TRY(launch_incremental(g, edges, ops, n, s));
    return mark_updated(g, s, true);
  } else if (!dev_e && !dev_o && n <= B) {
    // host input, one chunk: copy on the graph's copy stream into the
    // staging slot not used last, so that the copy overlaps the kernels of
    // the previous batch; the copy waits only for its slot to be free
    CUPC_TRY(ensure_copy_stream(g));
    const int k = g->next_slot;
    g->next_slot ^= 1;
    uint32_t* se = k ? g->stage_edges1 : g->stage_edges;
    int8_t* so = k ? g->stage_ops1 : g->stage_ops;
    CUPC_TRY(cudaStreamWaitEvent(g->copy_stream, g->slot_free[k], 0));
    CUPC_TRY(cudaMemcpyAsync(se, edges, 2 * n * sizeof(uint32_t), cudaMemcpyHostToDevice, g->copy_stream));
    CUPC_TRY(cudaMemcpyAsync(so, ops, n, cudaMemcpyHostToDevice, g->copy_stream));
    CUPC_TRY(cudaEventRecord(g->slot_ready[k], g->copy_stream));
    CUPC_TRY(cudaStreamWaitEvent(s, g->slot_ready[k], 0));
    CUPC_TRY(launch_update_chunk(g, se, n, s, so));
    if (g->inc) CUPC_TRY(launch_incremental(g, se, so, n, s));
    CUPC_TRY(mark_slot_free(g, k, s));
    return mark_updated(g, s, true);
  } else {
    // a host input mixed with a device one, or several chunks: stage in
    // slot 0 on the caller's stream; a multi-chunk batch is validated in
    // a first pass so that a bad entry drops the whole batch
    auto stage = [&](size_t i, size_t k) -> cudaError_t {
      cudaError_t e = cudaMemcpyAsync(g->stage_edges, edges + 2 * i, 2 * k * sizeof(uint32_t),
                                      dev_e ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return e;
      return cudaMemcpyAsync(g->stage_ops, ops + i, k, dev_o ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             s);
    };
    if (n <= B) {
      CUPC_TRY(stage(0, n));
      CUPC_TRY(launch_update_chunk(g, g->stage_edges, n, s, g->stage_ops));
    } else {
      for (size_t i = 0; i < n; i += B) {
        size_t k = n - i < B ? n - i : B;
        CUPC_TRY(stage(i, k));
        CUPC_TRY(launch_validate(g, g->stage_edges, g->stage_ops, k, s));
      }
      for (size_t i = 0; i < n; i += B) {
        size_t k = n - i < B ? n - i : B;
        CUPC_TRY(stage(i, k));
        CUPC_TRY(launch_update_chunk(g, g->stage_edges, k, s));
      }
    }
    CUPC_TRY(mark_slot_free(g, 0, s));
    // staged chunk by chunk: the labels are not followed (cleared)
    return mark_updated(g, s, false);
  }
}

cupc_status cupc_query(cupc_graph* g, const uint32_t* pairs, size_t m, uint8_t* out, cupc_stream stream) {
  if (!g) return CUPC_EINVAL;
  if (m == 0) return CUPC_OK;
  if (!pairs || !out) return CUPC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cupc_status st = recover_if_dirty(g, s);
  if (st != CUPC_OK) return st;
  const bool dev_p = is_device_ptr(pairs), dev_out = is_device_ptr(out);
  if (dev_p && dev_out) {
    CUPC_TRY(launch_query(g, pairs, m, out, s));
    return CUPC_OK;
  }
  const size_t B = g->max_pairs;
  for (size_t i = 0; i < m; i += B) {
    size_t k = m - i < B ? m - i : B;
    const uint32_t* p = pairs + 2 * i;
    if (!dev_p) {
      CUPC_TRY(cudaMemcpyAsync(g->stage_pairs, p, 2 * k * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
      p = g->stage_pairs;
    }
    uint8_t* o = dev_out ? out + i : g->stage_out;
    CUPC_TRY(launch_query(g, p, k, o, s));
    if (!dev_out) CUPC_TRY(cudaMemcpyAsync(out + i, g->stage_out, k, cudaMemcpyDeviceToHost, s));
  }
  CUPC_TRY(mark_slot_free(g, 0, s));  // the query staging is update slot 0
  if (!dev_out) CUPC_TRY(cudaStreamSynchronize(s));
  return CUPC_OK;
}

cupc_status cupc_sync(cupc_graph* g, cupc_stream stream) {
  if (!g) return CUPC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CUPC_TRY(cudaStreamSynchronize(s));
  uint32_t h[GC_SLOTS];
  CUPC_TRY(cudaMemcpy(h, g->gc, sizeof(h), cudaMemcpyDeviceToHost));
  if (h[GC_ERR]) {
    uint32_t zero = 0;
    CUPC_TRY(cudaMemcpy(g->gc + GC_ERR, &zero, sizeof(zero), cudaMemcpyHostToDevice));
    if (h[GC_ERR] & kErrTimeout) return CUPC_ETIMEOUT;
    return CUPC_EINVAL;
  }
  g->last_recovery = (h[GC_RECOVERIES] == 0 || h[GC_COMPLETE]) ? CUPC_OK : CUPC_EINCOMPLETE;
  return g->last_recovery;
}

cupc_status cupc_spanning_forest(cupc_graph* g, uint64_t* edge_ids_out, size_t cap, size_t* n_out,
                                 cupc_stream stream) {
  if (!g || !n_out) return CUPC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (g->inc && g->forest_stale) {  // labels may be incremental: the forest needs a recovery
    CUPC_TRY(launch_recover(g, s, true));
    g->dirty = false;
  } else {
    cupc_status st = recover_if_dirty(g, s);
    if (st != CUPC_OK) return st;
  }
  g->forest_stale = false;
  CUPC_TRY(launch_forest_sort(g, s));
  uint32_t h[GC_SLOTS];
  CUPC_TRY(cudaMemcpyAsync(h, g->gc, sizeof(h), cudaMemcpyDeviceToHost, s));
  CUPC_TRY(cudaStreamSynchronize(s));
  *n_out = h[GC_NFOREST];
  if (h[GC_ERR] & (kErrTimeout | kErrInval)) return cupc_sync(g, stream);
  if (cap < h[GC_NFOREST] || (!edge_ids_out && h[GC_NFOREST])) return CUPC_EINVAL;
  if (h[GC_NFOREST]) {
    CUPC_TRY(cudaMemcpyAsync(edge_ids_out, g->forest_sorted, h[GC_NFOREST] * sizeof(uint64_t), cudaMemcpyDefault,
                             s));
    CUPC_TRY(cudaStreamSynchronize(s));
  }
  g->last_recovery = (h[GC_RECOVERIES] == 0 || h[GC_COMPLETE]) ? CUPC_OK : CUPC_EINCOMPLETE;
  return g->last_recovery;
}

cupc_status cupc_labels(cupc_graph* g, uint32_t* labels_out, cupc_stream stream) {
  if (!g || !labels_out) return CUPC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cupc_status st = recover_if_dirty(g, s);
  if (st != CUPC_OK) return st;
  CUPC_TRY(cudaMemcpyAsync(labels_out, g->label, (size_t)g->V * 4, cudaMemcpyDefault, s));
  if (!is_device_ptr(labels_out)) CUPC_TRY(cudaStreamSynchronize(s));
  return CUPC_OK;
}

cupc_status cupc_export_sketches(cupc_graph* g, void* dst, size_t bytes, cupc_stream stream) {
  if (!g || !dst) return CUPC_EINVAL;
  size_t want = (size_t)g->L * g->V * g->W * sizeof(ulonglong2);
  if (bytes != want) return CUPC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CUPC_TRY(cudaMemcpyAsync(dst, g->sketch, want, cudaMemcpyDefault, s));
  CUPC_TRY(cudaStreamSynchronize(s));
  return CUPC_OK;
}

cupc_status cupc_import_sketches(cupc_graph* g, const void* src, size_t bytes, cupc_stream stream) {
  if (!g || !src) return CUPC_EINVAL;
  size_t want = (size_t)g->L * g->V * g->W * sizeof(ulonglong2);
  if (bytes != want) return CUPC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CUPC_TRY(cudaMemcpyAsync(g->sketch, src, want, cudaMemcpyDefault, s));
  g->imported = true;
  const cupc_status st = mark_updated(g, s, false);
  if (st != CUPC_OK) return st;
  CUPC_TRY(cudaStreamSynchronize(s));
  return CUPC_OK;
}

cupc_status cupc_set_incremental(cupc_graph* g, int on, cupc_stream stream) {
  if (!g) return CUPC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  g->inc = on != 0;
  // labels become incremental after the next complete recovery
  CUPC_TRY(cudaMemsetAsync(g->gc + GC_LABELS_VALID, 0, sizeof(uint32_t), s));
  g->dirty = true;
  return CUPC_OK;
}

cupc_status cupc_stats(cupc_graph* g, uint64_t* out8, cupc_stream stream) {
  if (!g || !out8) return CUPC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t h[GC_SLOTS];
  CUPC_TRY(cudaMemcpyAsync(h, g->gc, sizeof(h), cudaMemcpyDeviceToHost, s));
  CUPC_TRY(cudaStreamSynchronize(s));
  out8[0] = h[GC_ROUNDS];
  out8[1] = h[GC_NFAIL];
  out8[2] = h[GC_NFP];
  out8[3] = h[GC_COMPLETE];
  out8[4] = h[GC_NFOREST];
  out8[5] = h[GC_RECOVERIES];
  out8[6] = h[GC_BATCHES];
  out8[7] = h[GC_ERR];
  return CUPC_OK;
}

cupc_status cupc_round_log(cupc_graph* g, uint32_t* live, uint32_t* ncand, uint64_t* ids, size_t cap,
                           uint32_t* n_rounds, cupc_stream stream) {
  if (!g || !live || !ncand || !n_rounds) return CUPC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t h[GC_SLOTS];
  CUPC_TRY(cudaMemcpyAsync(h, g->gc, sizeof(h), cudaMemcpyDeviceToHost, s));
  CUPC_TRY(cudaStreamSynchronize(s));
  *n_rounds = h[GC_ROUNDS];
  if (cap < h[GC_LOGLEN] || (!ids && h[GC_LOGLEN])) return CUPC_EINVAL;
  CUPC_TRY(cudaMemcpy(live, g->log_live, g->L * 4, cudaMemcpyDeviceToHost));
  CUPC_TRY(cudaMemcpy(ncand, g->log_ncand, g->L * 4, cudaMemcpyDeviceToHost));
  if (h[GC_LOGLEN]) CUPC_TRY(cudaMemcpy(ids, g->log_ids, h[GC_LOGLEN] * 8, cudaMemcpyDeviceToHost));
  return CUPC_OK;
}

static void prof_drain(cupc_graph* g) {
  for (auto& r : g->prof) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      g->prof_ms[r.cls] += ms;
      g->prof_launches[r.cls] += (uint64_t)r.launches;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g->prof.clear();
  cudaGetLastError();
}

cupc_status cupc_profile_enable(cupc_graph* g, int on) {
  if (!g) return CUPC_EINVAL;
  prof_drain(g);
  for (int k = 0; k < PC_N; k++) {
    g->prof_ms[k] = 0.0;
    g->prof_launches[k] = 0;
  }
  g->prof_on = on != 0;
  return CUPC_OK;
}

cupc_status cupc_profile_read(cupc_graph* g, double* ms, uint64_t* launches, size_t n) {
  if (!g || !ms || !launches) return CUPC_EINVAL;
  prof_drain(g);
  for (size_t k = 0; k < n; k++) {
    ms[k] = k < (size_t)PC_N ? g->prof_ms[k] : 0.0;
    launches[k] = k < (size_t)PC_N ? g->prof_launches[k] : 0;
  }
  return CUPC_OK;
}

cupc_status cupc_set_tuning(cupc_graph* g, uint32_t item_records, uint32_t smem_rows, uint32_t ctas_per_sm) {
  if (!g) return CUPC_EINVAL;
  if (item_records == 0) item_records = kDefaultItemRecords;
  if (smem_rows == 0) smem_rows = g->D < kSmemRows ? g->D : kSmemRows;
  if (item_records < kMinItemRecords || item_records > kItemRecords || smem_rows > kSmemRowsMax || smem_rows > g->D)
    return CUPC_EINVAL;
  const uint32_t old_items = g->item_records, old_rows = g->R, old_cps = g->apply_cps;
  g->item_records = item_records;
  g->R = smem_rows;
  g->apply_cps = ctas_per_sm;
  if (configure_apply(g) != cudaSuccess) {
    cudaGetLastError();
    g->item_records = old_items;
    g->R = old_rows;
    g->apply_cps = old_cps;
    configure_apply(g);
    return CUPC_EINVAL;
  }
  return CUPC_OK;
}

cupc_status cupc_set_tuning_bucket(cupc_graph* g, uint32_t bucket, uint32_t item_records, uint32_t smem_rows,
                                   uint32_t ctas_per_sm) {
  if (!g || bucket < 5 || bucket > 15) return CUPC_EINVAL;
  cupc_graph::ApplyTune& t = g->tune_b[bucket];
  if (item_records == 0 && smem_rows == 0 && ctas_per_sm == 0) {  // back to the default
    t.set = false;
    return CUPC_OK;
  }
  if (item_records == 0) item_records = kDefaultItemRecords;
  if (smem_rows == 0) smem_rows = g->D < kSmemRows ? g->D : kSmemRows;
  if (item_records < kMinItemRecords || item_records > kItemRecords || smem_rows > kSmemRowsMax || smem_rows > g->D)
    return CUPC_EINVAL;
  int smem = 0, grid = 0;
  if (apply_config(g, item_records, smem_rows, ctas_per_sm, &smem, &grid) != cudaSuccess) {
    cudaGetLastError();
    return CUPC_EINVAL;
  }
  t = cupc_graph::ApplyTune{true, item_records, smem_rows, ctas_per_sm, smem, grid};
  return CUPC_OK;
}

cupc_status cupc_set_writeback_bucket(cupc_graph* g, uint32_t bucket, uint32_t mode) {
  if (!g || bucket < 5 || bucket > 15 || mode > CUPC_WRITEBACK_ATOMIC) return CUPC_EINVAL;
  g->wb_b[bucket] = mode;
  return CUPC_OK;
}

cupc_status cupc_get_tuning(const cupc_graph* g, uint32_t* out4) {
  if (!g || !out4) return CUPC_EINVAL;
  out4[0] = g->item_records;
  out4[1] = g->R;
  out4[2] = g->apply_cps;
  out4[3] = (uint32_t)(g->apply_grid / (g->sms ? g->sms : 1));
  return CUPC_OK;
}

cupc_status cupc_get_params(const cupc_graph* g, uint32_t* out4) {
  if (!g || !out4) return CUPC_EINVAL;
  out4[0] = g->L;
  out4[1] = g->C;
  out4[2] = g->D;
  out4[3] = g->W;
  return CUPC_OK;
}

void cupc_destroy(cupc_graph* g) {
  if (!g) return;
  prof_drain(g);
  if (g->copy_stream) {  // released once their pending work completes
    for (int k = 0; k < 2; k++) {
      cudaEventDestroy(g->slot_ready[k]);
      cudaEventDestroy(g->slot_free[k]);
    }
    cudaStreamDestroy(g->copy_stream);
  }
  if (g->owns_ws && g->ws) {
    cudaDeviceSynchronize();
    cudaFree(g->ws);
  }
  delete g;
}

const char* cupc_status_string(cupc_status s) {
  switch (s) {
    case CUPC_OK: return "CUPC_OK";
    case CUPC_EINVAL: return "CUPC_EINVAL: invalid argument or invalid edge/pair";
    case CUPC_ENOMEM: return "CUPC_ENOMEM: out of device memory or workspace too small";
    case CUPC_EINCOMPLETE: return "CUPC_EINCOMPLETE: recovery used every round without finishing";
    case CUPC_ECUDA: return "CUPC_ECUDA: CUDA runtime error";
    case CUPC_ETIMEOUT: return "CUPC_ETIMEOUT: bounded device wait expired";
  }
  return "unknown cupc_status";
}

}  // extern "C"
