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
// (exclusive: the vertex has a single item, so no other CTA writes its
// buckets); direct vertices' records come first and are cut into items of
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

// What one thread of the apply kernel does for a graph: tid = r*P + s; r < L
// is the layer, s < C a column, s == C the deterministic bucket. Lanes past
// the layout are idle: they fold into their own row 0, which is never
// written back.
//
// Column hash (Theorem A.1: 2-wise independent hash functions suffice):
// multiply-add-shift, h(x) = ((a*x + b) mod 2^64) div 2^(64-ell) with
// ell = 65 - 2*ceil(log2 V), strongly universal for indices x < V^2
// (Dietzfelbinger, STACS 1996); a second stage (a', b') continues the bit
// string when h(x) is zero. The depth is the number of leading zero bits of
// that string, capped at D-1. The deterministic and idle lanes use a = 0,
// b = 2^63, whose depth is always 0.
struct ApplyLane {
  uint64_t ka, kb;       // first-stage words of this lane's column
  const uint64_t* kx;    // {b, a', b'} of this lane's column (second stage)
  uint32_t ell, dmax;    // bits per stage, D-1
  uint32_t jbase;        // first bucket of this lane's column in its layer
  uint32_t nrows;        // rows this lane may have to write back
  uint32_t layer;        // r (0 for idle lanes)
  uint32_t si0, sr0;     // staging: first (record, layer) of this thread
  uint32_t sqi, sqr;     // staging: blockDim.x as (records, layers)
  bool active;
};

// keys: K(r*(C+1) + c) = a of column c (c < C), K(r*(C+1) + C) = checksum
// key of layer r, K(L*(C+1) + 3*(r*C + c) + {0,1,2}) = b, a', b'.
__device__ __forceinline__ ApplyLane apply_lane(const uint64_t* keys, uint32_t L, uint32_t C, uint32_t D, uint32_t P,
                                                uint32_t R, uint32_t ell) {
  ApplyLane l;
  const uint32_t tid = threadIdx.x;
  const uint32_t r = tid / P, s = tid % P;
  const bool col = r < L && s < C;
  l.active = r < L && s <= C;
  const uint64_t* kx = keys + (size_t)L * (C + 1) + 3 * (size_t)(r * C + s);
  l.ka = col ? keys[r * (C + 1) + s] : 0ull;
  l.kb = col ? kx[0] : (1ull << 63);
  l.kx = col ? kx : nullptr;
  l.ell = ell;
  l.dmax = D - 1;
  l.jbase = s == C ? 0u : 1u + s * D;
  l.nrows = s == C ? 1u : R;
  l.layer = r < L ? r : 0;
  l.si0 = tid / L;
  l.sr0 = tid % L;
  l.sqi = blockDim.x / L;
  l.sqr = blockDim.x % L;
  return l;
}

// The exact depth when the high word of the first stage does not decide it:
// leading zeros of the 2*ell-bit string h(x) h'(x) (probability 2^-min(ell,32)).
static __device__ __noinline__ uint32_t depth_long(const ApplyLane& l, uint64_t x, uint64_t z) {
  uint32_t d = min((uint32_t)__clzll((long long)z), l.ell);
  if (d == l.ell) {
    const uint64_t z2 = l.kx[1] * x + l.kx[2];
    d += min((uint32_t)__clzll((long long)z2), l.ell);
  }
  return d;
}

// Depth of index x in this lane's column. kLong: ell < D-1 or D-1 > 32, so
// the high word of a*x + b alone may not decide the depth (V > 2^16 at
// default parameters); otherwise min(clz(high word), D-1) is exact.
template <bool kLong>
__device__ __forceinline__ uint32_t lane_depth(const ApplyLane& l, uint64_t x) {
  const uint64_t z = l.ka * x + l.kb;
  uint32_t d = (uint32_t)__clz((int)(uint32_t)(z >> 32));
  if (kLong && d >= min(l.ell, 32u)) d = depth_long(l, x, z);
  return min(d, l.dmax);
}

// Shared memory of an apply CTA: fold rows (rows x threads buckets), then
// the staged records (two buffers: a pass writes one while the previous
// pass may still be read from the other), their per-layer checksums, the
// layer checksum keys and the records' vertices (direct path, two buffers).
struct ApplySmem {
  ulonglong2* rows;
  uint64_t* x;     // 2 * kStage
  uint64_t* g;     // kStage * L, [record][layer]
  uint64_t* kchk;  // L
  uint32_t* w;     // 2 * kStage
};
__device__ __forceinline__ ApplySmem apply_smem(unsigned char* raw, uint32_t rows, uint32_t L) {
  ApplySmem m;
  m.rows = reinterpret_cast<ulonglong2*>(raw);
  m.x = reinterpret_cast<uint64_t*>(m.rows + (size_t)rows * blockDim.x);
  m.g = m.x + 2 * kStage;
  m.kchk = m.g + (size_t)kStage * L;
  m.w = reinterpret_cast<uint32_t*>(m.kchk + L);
  return m;
}

// Fill the layer checksum keys of a graph (call from every thread; the
// first staging pass's barrier orders it before any use).
__device__ __forceinline__ void load_kchk(const ApplySmem& m, const uint64_t* keys, uint32_t L, uint32_t C) {
  for (uint32_t r = threadIdx.x; r < L; r += blockDim.x) m.kchk[r] = keys[r * (C + 1) + C];
}

// Records staged per pass by a CTA of blockDim.x threads: one record per
// thread, at most kStage.
__device__ __forceinline__ uint32_t stage_size() { return min(kStage, (uint32_t)blockDim.x); }

// Stage one pass of nc <= stage_size() records whose indices are in xr
// (thread t holds record t) into record buffer `buf` (0 or 1; consecutive
// passes alternate): idx, and G_r(idx) for every layer, computed once per
// (record, layer) and shared by the layer's lanes. The caller has already
// loaded xr (and w, for the direct path) from global memory. Returns the
// staged records.
__device__ __forceinline__ const uint64_t* stage_pass(const ApplyLane& l, const ApplySmem& m, uint64_t xr,
                                                      uint32_t wr, bool with_w, uint32_t nc, uint32_t L,
                                                      uint32_t buf) {
  uint64_t* xs = m.x + buf * kStage;
  if (threadIdx.x < nc) {
    xs[threadIdx.x] = xr;
    if (with_w) m.w[buf * kStage + threadIdx.x] = wr;
  }
  __syncthreads();  // the records are in; every lane is done with the previous pass
  const uint32_t total = nc * L;
  uint32_t i = l.si0, r = l.sr0;
  for (uint32_t k = threadIdx.x; k < total; k += blockDim.x) {
    m.g[k] = mix64(xs[i] ^ m.kchk[r]);
    i += l.sqi;
    r += l.sqr;
    if (r >= L) {
      r -= L;
      i++;
    }
  }
  __syncthreads();
  return xs;
}

__device__ __forceinline__ void fold_record(ulonglong2* gb, ulonglong2* my_rows, uint32_t rs, uint32_t R, uint32_t d,
                                            uint64_t x, uint64_t gm) {
  if (d < R) {
    ulonglong2 v = my_rows[d * rs];
    v.x ^= x;
    v.y ^= gm;
    my_rows[d * rs] = v;
  } else {
    xor_bucket_atomic(gb + d, make_ulonglong2(x, gm));
  }
}

// Two records into one lane's rows with both rows read before either is
// written, so the two read-modify-writes overlap instead of forming a chain.
// When both land in one row, the later store carries both records.
__device__ __forceinline__ void fold_pair(ulonglong2* gb, ulonglong2* my_rows, uint32_t rs, uint32_t R, uint32_t d0,
                                          uint64_t x0, uint64_t g0, uint32_t d1, uint64_t x1, uint64_t g1) {
  if (max(d0, d1) < R) {
    ulonglong2* p0 = my_rows + d0 * rs;
    ulonglong2* p1 = my_rows + d1 * rs;
    ulonglong2 v1 = *p1;
    ulonglong2 v0 = *p0;
    const uint64_t same = d0 == d1 ? ~0ull : 0ull;
    v1.x ^= x1;
    v1.y ^= g1;
    v0.x ^= x0 ^ (x1 & same);
    v0.y ^= g0 ^ (g1 & same);
    *p1 = v1;
    *p0 = v0;
  } else {
    fold_record(gb, my_rows, rs, R, d0, x0, g0);
    fold_record(gb, my_rows, rs, R, d1, x1, g1);
  }
}

// Fold the records rec[0..n) of one work item into the sketch of its vertex,
// whose buckets for this lane start at gb. Records pass through shared
// memory one pass at a time; each thread loads its record of the next pass
// while the current one folds. Rows of a lane live at my_rows[d * rs]
// (rs = blockDim.x), so the lanes of a shared-memory phase hit distinct
// 16-byte bank groups; a lane is the only writer of its rows, so no shared
// atomics are needed. Four records at a time: their loads and depths are
// independent, and they fold as two overlapping pairs. `excl`: no other CTA
// writes this vertex, so the write-back may be a plain read-modify-write.
// Call from every thread.
template <bool kLong>
__device__ __forceinline__ void apply_item(const ApplyLane& l, ulonglong2* gb, const uint64_t* __restrict__ rec,
                                           uint32_t n, bool excl, uint32_t L, uint32_t R, const ApplySmem& m,
                                           ulonglong2* my_rows, uint32_t rs) {
  const uint32_t cs = stage_size(), tid = threadIdx.x;
  const uint64_t* gcol = m.g + l.layer;
  uint64_t xr = tid < n ? __ldg(rec + tid) : 0ull;
  uint32_t buf = 0;
  for (uint32_t c0 = 0; c0 < n; c0 += cs, buf ^= 1) {
    const uint32_t nc = min(cs, n - c0);
    const uint64_t* xs = stage_pass(l, m, xr, 0u, false, nc, L, buf);
    const ulonglong2* x2 = reinterpret_cast<const ulonglong2*>(xs);
    if (c0 + cs + tid < n) xr = __ldg(rec + c0 + cs + tid);  // the next pass, in flight during this one
    uint32_t i = 0;
    for (; i + 4 <= nc; i += 4) {
      const ulonglong2 xa = x2[i >> 1], xb = x2[(i >> 1) + 1];
      const uint64_t x[4] = {xa.x, xa.y, xb.x, xb.y};
      uint64_t gm[4];
      uint32_t d[4];
#pragma unroll
      for (int k = 0; k < 4; k++) gm[k] = gcol[(i + k) * L];
#pragma unroll
      for (int k = 0; k < 4; k++) d[k] = lane_depth<kLong>(l, x[k]);
      fold_pair(gb, my_rows, rs, R, d[0], x[0], gm[0], d[1], x[1], gm[1]);
      fold_pair(gb, my_rows, rs, R, d[2], x[2], gm[2], d[3], x[3], gm[3]);
    }
    for (; i < nc; i++) {
      const uint64_t x = xs[i];
      fold_record(gb, my_rows, rs, R, lane_depth<kLong>(l, x), x, gcol[i * L]);
    }
  }

  // write back only the touched (non-zero) rows of this vertex. excl (the
  // vertex has this one item): load the old buckets, store the XOR; else
  // fire-and-forget XOR atomics, where a lane never waits for the old
  // bucket. Atomics are faster where vertices receive many records per
  // batch (fewer, hotter rows); load-then-store where they receive few.
  if (l.active) {
    if (excl) {
      for (uint32_t d0 = 0; d0 < l.nrows; d0 += 4) {
        ulonglong2 v[4], o[4];
        bool nz[4];
#pragma unroll
        for (uint32_t q = 0; q < 4; q++) {
          const uint32_t d = d0 + q;
          v[q] = make_ulonglong2(0, 0);
          nz[q] = false;
          if (d < l.nrows) {
            v[q] = my_rows[d * rs];
            nz[q] = (v[q].x | v[q].y) != 0;
            if (nz[q]) my_rows[d * rs] = make_ulonglong2(0, 0);
          }
        }
#pragma unroll
        for (uint32_t q = 0; q < 4; q++)
          if (nz[q]) o[q] = __ldcg(gb + d0 + q);
#pragma unroll
        for (uint32_t q = 0; q < 4; q++)
          if (nz[q]) gb[d0 + q] = make_ulonglong2(o[q].x ^ v[q].x, o[q].y ^ v[q].y);
      }
    } else {
      for (uint32_t d0 = 0; d0 < l.nrows; d0 += 4) {
#pragma unroll
        for (uint32_t q = 0; q < 4; q++) {
          const uint32_t d = d0 + q;
          if (d < l.nrows) {
            const ulonglong2 w = my_rows[d * rs];
            if ((w.x | w.y) != 0) {
              my_rows[d * rs] = make_ulonglong2(0, 0);
              xor_bucket_atomic(gb + d, w);
            }
          }
        }
      }
    }
  } else {
    my_rows[0] = make_ulonglong2(0, 0);
  }
  __syncthreads();
}

// Direct-path item: records of several vertices, each record's buckets XORed
// straight into HBM (atomics, no write-back). recw[i] is record i's vertex.
template <bool kLong>
__device__ __forceinline__ void apply_direct(const ApplyLane& l, ulonglong2* sketch, uint32_t V, uint32_t W,
                                             const uint64_t* __restrict__ rec, const uint32_t* __restrict__ recw,
                                             uint32_t n, uint32_t L, const ApplySmem& m) {
  ulonglong2* lbase = sketch + (size_t)l.layer * V * W + l.jbase;
  const uint64_t* gcol = m.g + l.layer;
  const uint32_t cs = stage_size(), tid = threadIdx.x;
  uint32_t buf = 0;
  for (uint32_t c0 = 0; c0 < n; c0 += cs, buf ^= 1) {
    const uint32_t nc = min(cs, n - c0);
    const bool mine = tid < nc;
    const uint64_t* xs =
        stage_pass(l, m, mine ? __ldg(rec + c0 + tid) : 0ull, mine ? __ldg(recw + c0 + tid) : 0u, true, nc, L, buf);
    const uint32_t* ws = m.w + buf * kStage;
    for (uint32_t i0 = 0; i0 < nc; i0 += 4) {
      uint64_t x[4], gm[4];
      uint32_t d[4], w[4];
#pragma unroll
      for (uint32_t k = 0; k < 4; k++) {
        const uint32_t i = min(i0 + k, nc - 1);
        x[k] = xs[i];
        gm[k] = gcol[i * L];
        w[k] = ws[i];
      }
#pragma unroll
      for (uint32_t k = 0; k < 4; k++) d[k] = lane_depth<kLong>(l, x[k]);
#pragma unroll
      for (uint32_t k = 0; k < 4; k++)
        if (l.active && i0 + k < nc) xor_bucket_atomic(lbase + (size_t)w[k] * W + d[k], make_ulonglong2(x[k], gm[k]));
    }
  }
  __syncthreads();
}

}  // namespace cupc
