// Device-side pieces of the sketch update shared by the single-graph and the
// multi-graph apply kernels (see update.cu and batch.cu).
#pragma once

#include "common.cuh"

namespace cupc {

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
// branch-free instruction stream. Records are hashed one group of four ahead
// of the group being folded, so the hashing fills the latency of the fold's
// shared-memory read-modify-writes. `excl`: no other CTA writes this vertex,
// so the write-back is a plain read-modify-write. Call from every thread.
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

  auto fold = [&](uint64_t x, uint64_t h, uint64_t g) {
    uint32_t d = depth_fast<kWide>(h, D);
    if (l.row0) d = 0;
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
    hc[k] = mix_tail(xc[k].y ^ l.kpre);
  }
  for (uint32_t g = 0; g < nfull; g++) {
    uint64_t gm[4], hn[4];
    ulonglong2 xn[4];
#pragma unroll
    for (uint32_t k = 0; k < 4; k++) gm[k] = __shfl_sync(0xffffffffu, hc[k], l.chk_lane);
#pragma unroll
    for (uint32_t k = 0; k < 4; k++) {  // next group (clamped: the last one is recomputed harmlessly)
      xn[k] = s_xp[min(4 * g + 4 + k, n - 1)];
      hn[k] = mix_tail(xn[k].y ^ l.kpre);
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
    const uint64_t h = mix_tail(x.y ^ l.kpre);
    fold(x.x, h, __shfl_sync(0xffffffffu, h, l.chk_lane));
  }

  // write back only the touched (non-zero) rows of this vertex
  if (l.active) {
    for (uint32_t d0 = 0; d0 < l.nrows; d0 += 4) {
      ulonglong2 v[4], o[4];
      bool nz[4];
#pragma unroll
      for (uint32_t q = 0; q < 4; q++) {
        const uint32_t d = d0 + q;
        nz[q] = false;
        if (d < l.nrows) {
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
    my_rows[0] = make_ulonglong2(0, 0);
  }
  __syncthreads();
}

}  // namespace cupc
