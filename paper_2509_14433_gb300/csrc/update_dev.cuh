// Device-side pieces of the sketch update shared by the single-graph and the
// multi-graph apply kernels (see update.cu and batch.cu).
#pragma once

#include "common.cuh"

namespace cupc {

// Block-wide exclusive scan of three u32 values per thread (any multiple of
// 32 threads up to 1024). e* = exclusive prefix, t* = block totals.
__device__ __forceinline__ void block_scan3(const uint32_t (&v)[3], uint32_t (&e)[3], uint32_t (&t)[3],
                                            uint32_t (*sw)[32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc[3] = {v[0], v[1], v[2]};
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, inc[k], o);
      if (lane >= o) inc[k] += x;
    }
  }
  if (lane == 31)
#pragma unroll
    for (int k = 0; k < 3; k++) sw[k][wid] = inc[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint32_t x = lane < nw ? sw[k][lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane < nw) sw[k][lane] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 3; k++) {
    e[k] = (wid ? sw[k][wid - 1] : 0) + inc[k] - v[k];
    t[k] = sw[k][nw - 1];
  }
  __syncthreads();
}

// Vertices with at most this many endpoint records in a batch take the
// direct path: no shared-memory fold, each record's buckets are XORed
// straight into HBM with fire-and-forget atomics.
constexpr uint32_t kDirectMax = 2;
// Work item whose records belong to several direct-path vertices, and its
// size: small, so that a sparse batch still spreads over every SM.
constexpr uint32_t kDirectItem = 0xFFFFFFFFu;
constexpr uint32_t kDirectItemRecords = 64;  // at most; the single-graph plan
constexpr uint32_t kDirectItemMin = 16;      // sizes them to the apply grid

// Work plan of one batch, run by one CTA: vertices with more than
// kDirectMax records ("fold" vertices) get record segments after all direct
// records and ceil(n_w / item_records) items {w, begin, end, exclusive}
// (exclusive: the vertex has a single item, so its write-back needs no
// atomics); direct vertices' records come first and are cut into items of
// item_records records {kDirectItem, begin, end, 0}. Writes the per-vertex
// scatter cursors, resets cnt, returns the item count and the number of
// direct records (*nd). Direct items hold kDirectItemRecords records.
__device__ __forceinline__ uint32_t plan_vertices(uint32_t* cnt, uint32_t* cursor, uint4* items, uint32_t V,
                                                  uint32_t item_records, uint32_t* nd_out) {
  __shared__ uint32_t sw[3][32];
  __shared__ uint32_t s_nd;
  // pass 1: how many records go the direct way
  uint32_t dsum = 0;
  for (uint32_t w = threadIdx.x; w < V; w += blockDim.x) {
    const uint32_t c = cnt[w];
    dsum += c <= kDirectMax ? c : 0;
  }
  dsum = __reduce_add_sync(0xffffffffu, dsum);
  if (threadIdx.x == 0) s_nd = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) atomicAdd(&s_nd, dsum);
  __syncthreads();
  const uint32_t nd = s_nd;
  // pass 2: cursors and fold items
  uint32_t carry[3] = {0, 0, 0};  // fold records, direct records, fold items
  for (uint32_t base = 0; base < V; base += 4 * blockDim.x) {
    const uint32_t w0 = base + 4 * threadIdx.x;
    uint32_t c[4], v[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 4; k++) {
      c[k] = (w0 + k < V) ? cnt[w0 + k] : 0;
      if (c[k] > kDirectMax) {
        v[0] += c[k];
        v[2] += (c[k] + item_records - 1) / item_records;
      } else {
        v[1] += c[k];
      }
    }
    uint32_t e[3], t[3];
    block_scan3(v, e, t, sw);
    uint32_t pf = nd + carry[0] + e[0], pd = carry[1] + e[1], pi = carry[2] + e[2];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t w = w0 + k;
      if (w >= V) continue;
      cnt[w] = 0;
      if (c[k] > kDirectMax) {
        const uint32_t ni = (c[k] + item_records - 1) / item_records;
        cursor[w] = pf;
        for (uint32_t q = 0; q < ni; q++) {
          const uint32_t b = pf + q * item_records;
          items[pi + q] = make_uint4(w, b, min(pf + c[k], b + item_records), ni == 1 ? 1u : 0u);
        }
        pf += c[k];
        pi += ni;
      } else {
        cursor[w] = pd;
        pd += c[k];
      }
    }
#pragma unroll
    for (int k = 0; k < 3; k++) carry[k] += t[k];
  }
  // direct items after the fold items
  const uint32_t nfold = carry[2], ndi = (nd + kDirectItemRecords - 1) / kDirectItemRecords;
  for (uint32_t q = threadIdx.x; q < ndi; q += blockDim.x)
    items[nfold + q] = make_uint4(kDirectItem, q * kDirectItemRecords, min(nd, (q + 1) * kDirectItemRecords), 0u);
  *nd_out = nd;
  return nfold + ndi;
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

// What one thread of the apply kernel does for a graph: tid = r*P + s; r < L
// is the layer, s < C a column, s == C the checksum lane, which owns the
// deterministic bucket (its row 0). Lanes past the layout are idle: they fold
// into their own row 0, which is never written back.
struct ApplyLane {
  uint64_t kpre;       // pre(key) of this lane's column (or checksum) hash
  uint32_t chk_lane;   // warp lane holding the checksum of this lane's layer
  uint32_t jbase;      // first bucket of this lane's column in its layer
  uint32_t nrows;      // rows this lane may have to write back
  uint32_t layer;      // r (0 for idle lanes)
  bool active, row0;
};

__device__ __forceinline__ ApplyLane apply_lane(const uint64_t* keys, uint32_t L, uint32_t C, uint32_t D, uint32_t P,
                                                uint32_t R) {
  ApplyLane l;
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  const uint32_t r = tid / P, s = tid % P;
  l.active = r < L && s <= C;
  l.row0 = !l.active || s == C;
  l.kpre = l.active ? pre_mix(keys[r * (C + 1) + s]) : 0;
  l.chk_lane = (lane & ~(P - 1)) | C;
  l.jbase = s == C ? 0u : 1u + s * D;
  l.nrows = s == C ? 1u : R;
  l.layer = r < L ? r : 0;
  return l;
}

// Fold the records rec[0..n) of one work item into the sketch of its vertex,
// whose buckets for this lane start at gb. Rows of a lane live at
// my_rows[d * rs] (rs = blockDim.x), so the 8 lanes of a shared-memory phase
// always hit 8 distinct 16-byte bank groups; a lane is the only writer of its
// rows, so no shared atomics are needed, and every lane runs the same
// branch-free instruction stream. The next record is hashed while the current
// one folds. The loop is kept this lean on purpose: at <= 64 registers eight
// 128-thread CTAs fit an SM, and that occupancy hides the shared-memory
// latency of the fold better than hashing several records ahead (measured on
// GB300: 462 us for 2^20 edges at V = 16384 against 514 us with a four-record
// lookahead at 80 registers). `excl`: no other CTA writes this vertex, so the
// write-back is a plain read-modify-write. Call from every thread.
template <bool kWide>
__device__ __forceinline__ void apply_item(const ApplyLane& l, ulonglong2* gb, const uint64_t* __restrict__ rec,
                                           uint32_t n, bool excl, uint32_t D, uint32_t R, ulonglong2* s_xp,
                                           ulonglong2* my_rows, uint32_t rs) {
  const uint32_t tid = threadIdx.x;
  if (l.active) {  // bring this lane's buckets to L2 for the write-back
    prefetch_l2(gb);
    if (l.nrows > 1) {
      prefetch_l2(gb + 6);
      prefetch_l2(gb + l.nrows - 1);
    }
  }
  for (uint32_t i = tid; i < n; i += blockDim.x) {
    const uint64_t x = rec[i];
    s_xp[i] = make_ulonglong2(x, pre_mix(x));
  }
  __syncthreads();

  ulonglong2 xc = s_xp[0];
  uint64_t hc = mix_tail(xc.y ^ l.kpre);
  for (uint32_t i = 0; i < n; i++) {
    const uint64_t gm = __shfl_sync(0xffffffffu, hc, l.chk_lane);
    const ulonglong2 xn = s_xp[min(i + 1, n - 1)];  // the last one is recomputed harmlessly
    const uint64_t hn = mix_tail(xn.y ^ l.kpre);
    const uint32_t d = l.row0 ? 0u : depth_fast<kWide>(hc, D);
    if (d < R) {
      ulonglong2 v = my_rows[d * rs];
      v.x ^= xc.x;
      v.y ^= gm;
      my_rows[d * rs] = v;
    } else {
      xor_bucket_atomic(gb + d, make_ulonglong2(xc.x, gm));
    }
    xc = xn;
    hc = hn;
  }

  // write back only the touched (non-zero) rows of this vertex
  if (l.active) {
    for (uint32_t d0 = 0; d0 < l.nrows; d0 += 4) {
      ulonglong2 v[4], o[4];
      bool nz[4];
#pragma unroll
      for (uint32_t q = 0; q < 4; q++) {
        const uint32_t d = d0 + q;
        v[q] = make_ulonglong2(0, 0);
        nz[q] = false;
        if (d < l.nrows) {
          const ulonglong2 w = my_rows[d * rs];
          if ((w.x | w.y) != 0) {
            v[q] = w;
            my_rows[d * rs] = make_ulonglong2(0, 0);
          }
          nz[q] = (v[q].x | v[q].y) != 0;
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
    my_rows[0] = make_ulonglong2(0, 0);
  }
  __syncthreads();
}


// Direct-path item: records of several vertices, each record's buckets XORed
// straight into HBM (atomics, no write-back). recw[i] is record i's vertex.
template <bool kWide>
__device__ __forceinline__ void apply_direct(const ApplyLane& l, ulonglong2* sketch, uint32_t V, uint32_t W,
                                             const uint64_t* __restrict__ rec, const uint32_t* __restrict__ recw,
                                             uint32_t n, uint32_t D, ulonglong2* s_xp, uint32_t* s_w) {
  const uint32_t tid = threadIdx.x;
  for (uint32_t i = tid; i < n; i += blockDim.x) {
    const uint64_t x = rec[i];
    s_xp[i] = make_ulonglong2(x, pre_mix(x));
    s_w[i] = recw[i];
  }
  __syncthreads();
  ulonglong2* lbase = sketch + (size_t)l.layer * V * W + l.jbase;
  for (uint32_t i0 = 0; i0 < n; i0 += 4) {
    ulonglong2 x[4];
    uint64_t h[4], g[4];
#pragma unroll
    for (uint32_t k = 0; k < 4; k++) {
      x[k] = s_xp[min(i0 + k, n - 1)];
      h[k] = mix_tail(x[k].y ^ l.kpre);
    }
#pragma unroll
    for (uint32_t k = 0; k < 4; k++) g[k] = __shfl_sync(0xffffffffu, h[k], l.chk_lane);
#pragma unroll
    for (uint32_t k = 0; k < 4; k++) {
      uint32_t d = depth_fast<kWide>(h[k], D);
      if (l.row0) d = 0;
      if (l.active && i0 + k < n) xor_bucket_atomic(lbase + (size_t)s_w[i0 + k] * W + d, make_ulonglong2(x[k].x, g[k]));
    }
  }
  __syncthreads();
}

}  // namespace cupc
