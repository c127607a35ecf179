// Batched edge updates into the vertex sketches (App. A.1.1, "The AGM
// Algorithm": an update of edge (u,v) updates every sketch of u and of v;
// Theorem A.2: CameoSketch touches one bucket per column per update).
//
// One chunk of <= max_batch edges goes through four stream-ordered kernels:
//   k_count   per-vertex record counts (2 records per edge, one per endpoint)
//   k_plan    exclusive scan -> per-vertex cursors + work items of at most
//             kItemRecords records of one vertex (single CTA)
//   k_scatter endpoint records (the edge index u*V+v) grouped by vertex
//   k_apply   persistent CTAs pull work items; thread (layer r, slot s)
//             hashes every record of the item for column s of layer r (slot
//             C computes the checksum and owns the deterministic bucket),
//             folds them in shared memory, then read-modify-writes only the
//             touched buckets of that vertex in HBM with 16-byte accesses.
// XOR is associative and commutative, so the result is bit-identical to
// applying the updates one by one in stream order.
#include "common.cuh"

namespace cupc {

__global__ void k_keys(uint64_t seed, uint64_t* keys, uint32_t n) {
  const uint64_t phi = 0x9E3779B97F4A7C15ull;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    keys[j] = mix64(seed + phi * (uint64_t)(j + 1));
}

cudaError_t launch_keys(cupc_graph* g, cudaStream_t s) {
  uint32_t n = g->L * (g->C + 1);
  k_keys<<<1, 256, 0, s>>>(g->seed, g->keys, n);
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

// Block-wide exclusive scan of two u32 values per thread (1024 threads).
__device__ __forceinline__ void block_scan2(uint32_t a, uint32_t b, uint32_t& ea, uint32_t& eb, uint32_t& ta,
                                            uint32_t& tb, uint32_t* sa, uint32_t* sb) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t xa = __shfl_up_sync(0xffffffffu, ia, o), xb = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) {
      ia += xa;
      ib += xb;
    }
  }
  if (lane == 31) {
    sa[wid] = ia;
    sb[wid] = ib;
  }
  __syncthreads();
  if (wid == 0) {
    uint32_t va = lane < nw ? sa[lane] : 0, vb = lane < nw ? sb[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t xa = __shfl_up_sync(0xffffffffu, va, o), xb = __shfl_up_sync(0xffffffffu, vb, o);
      if (lane >= o) {
        va += xa;
        vb += xb;
      }
    }
    if (lane < nw) {
      sa[lane] = va;
      sb[lane] = vb;
    }
  }
  __syncthreads();
  uint32_t wa = wid ? sa[wid - 1] : 0, wb = wid ? sb[wid - 1] : 0;
  ea = wa + ia - a;
  eb = wb + ib - b;
  ta = sa[nw - 1];
  tb = sb[nw - 1];
  __syncthreads();
}

// Exclusive scan of the per-vertex record counts into cursors, and the work
// item list: vertex w with n_w records yields ceil(n_w / kItemRecords) items
// {w, begin, end, exclusive}; exclusive = the vertex has a single item, so
// its write-back needs no atomics. Resets cnt for the next chunk.
__global__ void __launch_bounds__(1024) k_plan(uint32_t* cnt, uint32_t* cursor, uint4* items, uint32_t V,
                                                 uint32_t* gc) {
  __shared__ uint32_t sa[32], sb[32];
  if (ld_cg(&gc[GC_ERR]) & kErrInval) return;
  uint32_t carry_rec = 0, carry_item = 0;
  for (uint32_t base = 0; base < V; base += 4 * blockDim.x) {
    uint32_t w0 = base + 4 * threadIdx.x;
    uint32_t c[4], ni[4], lr = 0, li = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      c[k] = (w0 + k < V) ? cnt[w0 + k] : 0;
      ni[k] = (c[k] + kItemRecords - 1) / kItemRecords;
      lr += c[k];
      li += ni[k];
    }
    uint32_t er, ei, tr, ti;
    block_scan2(lr, li, er, ei, tr, ti, sa, sb);
    uint32_t pr = carry_rec + er, pi = carry_item + ei;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      uint32_t w = w0 + k;
      if (w < V) {
        cursor[w] = pr;
        cnt[w] = 0;
        for (uint32_t q = 0; q < ni[k]; q++) {
          uint32_t b = pr + q * kItemRecords;
          uint32_t e = min(pr + c[k], b + kItemRecords);
          items[pi + q] = make_uint4(w, b, e, ni[k] == 1 ? 1u : 0u);
        }
      }
      pr += c[k];
      pi += ni[k];
    }
    carry_rec += tr;
    carry_item += ti;
  }
  if (threadIdx.x == 0) {
    gc[GC_NITEMS] = carry_item;
    gc[GC_NEXT_ITEM] = 0;
    gc[GC_BATCHES] += 1;
  }
}

__global__ void k_scatter(const uint32_t* __restrict__ edges, size_t n, uint32_t V, uint32_t* cursor,
                          uint64_t* __restrict__ rec, const uint32_t* gc) {
  if (ld_cg(&gc[GC_ERR]) & kErrInval) return;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t u = edges[2 * i], v = edges[2 * i + 1];
    uint32_t a = min(u, v), b = max(u, v);
    uint64_t idx = (uint64_t)a * V + b;
    rec[atomicAdd(&cursor[u], 1u)] = idx;
    rec[atomicAdd(&cursor[v], 1u)] = idx;
  }
}

__device__ __forceinline__ void xor_bucket_atomic(ulonglong2* p, ulonglong2 v) {
  atomicXor(&p->x, v.x);
  atomicXor(&p->y, v.y);
}

// The SplitMix64 finalizer of idx ^ key, split so that its first step is
// shared by every lane: with z = idx ^ key, z ^ (z >> 30) equals
// pre(idx) ^ pre(key), pre(x) = x ^ (x >> 30), because XOR commutes with a
// logical shift. pre(idx) is computed once per record when the record is
// staged in shared memory; pre(key) is a per-lane constant.
__device__ __forceinline__ uint64_t pre_mix(uint64_t x) { return x ^ (x >> 30); }
__device__ __forceinline__ uint64_t mix_tail(uint64_t z) {
  z *= 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Row of an index from its hash: trailing zeros, capped at D-1. With
// D <= 32 the low hash word decides (a zero low word means depth >= 32 >=
// D-1); wider sketches fall back to the 64-bit count in that rare case.
template <bool kWide>
__device__ __forceinline__ uint32_t depth_fast(uint64_t h, uint32_t D) {
  const uint32_t lo = (uint32_t)h;
  uint32_t d = (uint32_t)__ffs(lo) - 1u;  // lo == 0 gives 0xFFFFFFFF
  if (kWide && lo == 0) d = depth_of(h, D);
  return min(d, D - 1);
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Fold the records of one work item into the sketches of its vertex.
// Thread layout: tid = r*P + s; r < L is the layer, s < C a column, s == C
// the checksum lane, which owns the deterministic bucket (its row 0). A lane
// is the only writer of its rows in shared memory, so no shared atomics are
// needed, and every lane runs the same branch-free instruction stream (lanes
// past the layout fold into their own rows, which are never written back);
// the checksum of a record reaches the column lanes by shuffle. Records are
// hashed one group of four ahead of the group being folded, so the hashing
// fills the latency of the fold's shared-memory read-modify-writes.
template <bool kWide>
__global__ void k_apply(ulonglong2* __restrict__ sketch, const uint64_t* __restrict__ keys,
                        const uint64_t* __restrict__ rec, const uint4* __restrict__ items, uint32_t* gc,
                        uint32_t V, uint32_t L, uint32_t C, uint32_t D, uint32_t W, uint32_t P, uint32_t R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* s_xp = reinterpret_cast<ulonglong2*>(smem_raw);  // {idx, pre(idx)}
  ulonglong2* s_acc = s_xp + kItemRecords;
  __shared__ uint32_t s_item;

  if (ld_cg(&gc[GC_ERR]) & kErrInval) return;
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  const uint32_t r = tid / P, s = tid % P;
  const bool active = r < L && s <= C;
  const bool row0 = !active || s == C;  // checksum lane and idle lanes use row 0 only
  const uint64_t kpre = active ? pre_mix(keys[r * (C + 1) + s]) : 0;
  const uint32_t chk_lane = (lane & ~(P - 1)) | C;
  const uint32_t jbase = s == C ? 0u : 1u + s * D;  // first bucket of this lane's column
  const uint32_t nrows = s == C ? 1u : R;
  // row d of this lane lives at s_acc[d * blockDim.x + tid]: the 8 lanes of a
  // shared-memory phase always hit 8 distinct 16-byte bank groups
  ulonglong2* my_rows = s_acc + tid;
  const uint32_t rs = blockDim.x;
  for (uint32_t d = 0; d < R; d++) my_rows[d * rs] = make_ulonglong2(0, 0);

  const uint32_t nitems = ld_cg(&gc[GC_NITEMS]);
  for (;;) {
    if (tid == 0) s_item = atomicAdd(&gc[GC_NEXT_ITEM], 1u);
    __syncthreads();
    const uint32_t it = s_item;
    if (it >= nitems) break;
    const uint4 item = items[it];
    const uint32_t w = item.x, beg = item.y, n = item.z - item.y;
    const bool excl = item.w != 0;
    ulonglong2* gb = sketch + ((size_t)(r < L ? r : 0) * V + w) * W + jbase;
    if (active) {  // bring this lane's buckets to L2 for the write-back
      prefetch_l2(gb);
      if (nrows > 1) {
        prefetch_l2(gb + 6);
        prefetch_l2(gb + nrows - 1);
      }
    }
    for (uint32_t i = tid; i < n; i += blockDim.x) {
      const uint64_t x = rec[beg + i];
      s_xp[i] = make_ulonglong2(x, pre_mix(x));
    }
    __syncthreads();

    auto fold = [&](uint64_t x, uint64_t h, uint64_t g) {
      uint32_t d = depth_fast<kWide>(h, D);
      if (row0) d = 0;
      if (d < R) {
        ulonglong2 v = my_rows[d * rs];
        v.x ^= x;
        v.y ^= g;
        my_rows[d * rs] = v;
      } else {
        xor_bucket_atomic(gb + d, make_ulonglong2(x, g));
      }
    };

    const uint32_t nfull = n >> 2;
    ulonglong2 xc[4];
    uint64_t hc[4];
#pragma unroll
    for (uint32_t k = 0; k < 4; k++) {
      xc[k] = s_xp[min(k, n - 1)];
      hc[k] = mix_tail(xc[k].y ^ kpre);
    }
    for (uint32_t g = 0; g < nfull; g++) {
      uint64_t gm[4], hn[4];
      ulonglong2 xn[4];
#pragma unroll
      for (uint32_t k = 0; k < 4; k++) gm[k] = __shfl_sync(0xffffffffu, hc[k], chk_lane);
#pragma unroll
      for (uint32_t k = 0; k < 4; k++) {  // next group (clamped: the last one is recomputed harmlessly)
        xn[k] = s_xp[min(4 * g + 4 + k, n - 1)];
        hn[k] = mix_tail(xn[k].y ^ kpre);
      }
#pragma unroll
      for (uint32_t k = 0; k < 4; k++) fold(xc[k].x, hc[k], gm[k]);
#pragma unroll
      for (uint32_t k = 0; k < 4; k++) {
        xc[k] = xn[k];
        hc[k] = hn[k];
      }
    }
    for (uint32_t i = 4 * nfull; i < n; i++) {
      const ulonglong2 x = s_xp[i];
      const uint64_t h = mix_tail(x.y ^ kpre);
      fold(x.x, h, __shfl_sync(0xffffffffu, h, chk_lane));
    }

    // write back only the touched (non-zero) rows of this vertex
    if (active) {
      for (uint32_t d0 = 0; d0 < nrows; d0 += 4) {
        ulonglong2 v[4], o[4];
        bool nz[4];
#pragma unroll
        for (uint32_t q = 0; q < 4; q++) {
          const uint32_t d = d0 + q;
          nz[q] = false;
          if (d < nrows) {
            v[q] = my_rows[d * rs];
            nz[q] = (v[q].x | v[q].y) != 0;
            if (nz[q]) my_rows[d * rs] = make_ulonglong2(0, 0);
          }
        }
        if (excl) {
#pragma unroll
          for (uint32_t q = 0; q < 4; q++)
            if (nz[q]) o[q] = __ldcg(gb + d0 + q);
#pragma unroll
          for (uint32_t q = 0; q < 4; q++)
            if (nz[q]) gb[d0 + q] = make_ulonglong2(o[q].x ^ v[q].x, o[q].y ^ v[q].y);
        } else {
#pragma unroll
          for (uint32_t q = 0; q < 4; q++)
            if (nz[q]) xor_bucket_atomic(gb + d0 + q, v[q]);
        }
      }
    } else {
      for (uint32_t d = 0; d < R; d++) my_rows[d * rs] = make_ulonglong2(0, 0);
    }
    __syncthreads();
  }
}

// The dynamic shared-memory limit of k_apply is process-wide: only ever
// raise it, so that a graph created later never shrinks it below what an
// earlier graph's launches need.
cudaError_t raise_apply_smem_limit(int bytes) {
  const void* fns[2] = {(const void*)k_apply<false>, (const void*)k_apply<true>};
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
  g->P = 1;
  while (g->P < g->C + 1) g->P <<= 1;
  g->R = g->D < kSmemRows ? g->D : kSmemRows;
  g->apply_threads = (int)(((g->L * g->P) + 31) / 32 * 32);
  g->apply_smem = (int)(kItemRecords * sizeof(ulonglong2) + (size_t)g->R * g->apply_threads * sizeof(ulonglong2));
  cudaError_t e = raise_apply_smem_limit(g->apply_smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, g->D > 32 ? k_apply<true> : k_apply<false>,
                                                    g->apply_threads, g->apply_smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  g->apply_grid = per_sm * g->sms;
  return cudaSuccess;
}

cudaError_t launch_update_chunk(cupc_graph* g, const uint32_t* edges, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)g->sms * 8);
  {
    ProfScope ps(g, s, PC_GROUP, 3);
    k_count<<<grid, 256, 0, s>>>(edges, n, g->cnt, g->gc);
    k_plan<<<1, 1024, 0, s>>>(g->cnt, g->cursor, g->items, g->V, g->gc);
    k_scatter<<<grid, 256, 0, s>>>(edges, n, g->V, g->cursor, g->rec, g->gc);
  }
  ProfScope ps(g, s, PC_APPLY, 1);
  int agrid = (int)std::min<size_t>((size_t)g->apply_grid, 2 * n);
  auto kern = g->D > 32 ? k_apply<true> : k_apply<false>;
  kern<<<agrid, g->apply_threads, g->apply_smem, s>>>(g->sketch, g->keys, g->rec, g->items, g->gc, g->V, g->L, g->C,
                                                       g->D, g->W, g->P, g->R);
  return cudaGetLastError();
}

}  // namespace cupc
