// Recovery state and warp helpers shared by the grid-wide recovery
// (recover.cu) and the one-cluster recovery of small graphs
// (recover_small.cu).
#pragma once

#include "common.cuh"

namespace cupc {

struct RecArgs {
  const ulonglong2* sketch;
  const uint64_t* keys;
  uint32_t V, L, C, D, W;
  uint32_t *label, *parent, *minv, *rcnt, *roff, *perm, *permb, *pcount;
  uint8_t *final_, *merged;
  uint64_t *best0, *best1, *forest, *log_ids;
  ulonglong2* cand;  // {edge, label[u] << 32 | label[v]} of a component's candidate
  ulonglong2* acc;
  uint32_t *log_live, *log_ncand;
  ulonglong2* hlist;  // kSmallHook: crossing candidates {edge, root_a << 32 | root_b} of a hook step
  uint32_t* ipar;     // V: union-find of incremental inserts, identity after a recovery
  const uint64_t* forest_sorted;
  uint8_t* fdead;     // V: forest_sorted[i] deleted since the last recovery
  const uint64_t* fadd;      // V: forest edges added by incremental merges since
  const uint8_t* fadd_dead;  // V: fadd[j] deleted since
  unsigned long long* ftab;  // 2^ftab_bits: the ids of fadd (cleared here)
  uint32_t ftab_bits;
  uint32_t inc, force;  // incremental mode; run even if the labels are valid
  uint32_t sum_zero;    // the XOR of all vertex sketches of a layer is zero (no import since reset)
  uint32_t* gc;
};

// u < v for an edge id x = u*V + v (32-bit division when x fits 32 bits).
__device__ __forceinline__ bool edge_id_ordered(uint64_t x, uint32_t V) {
  if ((x >> 32) == 0) {
    const uint32_t x32 = (uint32_t)x, u = x32 / V;
    return u < x32 - u * V;
  }
  const uint64_t u = x / V;
  return u < x - u * V;
}

// Sample a layer-r sum held by a warp (lane l holds buckets l + 32q,
// q < NQ): ZERO if the deterministic bucket is zero, else the first good
// bucket in index order j = l + 32q (deterministic bucket, then
// column-major), else FAIL. A bucket is good when its alpha is non-zero,
// its checksum holds and alpha is an edge id u*V+v with u < v. Returns 0/1/2
// in every lane and the edge id in `edge`. Bucket groups q are tested in
// order and the test stops at the first group holding a good bucket (the
// flag is warp-uniform, so later groups are skipped, not hashed).
template <uint32_t NQ>
__device__ __forceinline__ uint32_t warp_sample(const ulonglong2 (&acc)[NQ], uint32_t W, uint32_t V, uint64_t kchk,
                                                uint64_t& edge) {
  const uint32_t lane = threadIdx.x & 31;
  edge = 0;
  if (__shfl_sync(0xffffffffu, (acc[0].x | acc[0].y) == 0 ? 1u : 0u, 0)) return 0;
  uint32_t found = 0;
  uint64_t e = 0;
#pragma unroll
  for (uint32_t q = 0; q < NQ; q++) {
    if (!found) {
      const uint32_t j = lane + 32 * q;
      const bool good =
          j < W && acc[q].x != 0 && mix64(acc[q].x ^ kchk) == acc[q].y && edge_id_ordered(acc[q].x, V);
      const uint32_t m = __ballot_sync(0xffffffffu, good);
      if (m) {
        e = __shfl_sync(0xffffffffu, acc[q].x, __ffs(m) - 1);
        found = 1;
      }
    }
  }
  edge = e;
  return found ? 1u : 2u;
}

// lane l XORs buckets l + 32q of one member's row into acc
template <uint32_t NQ>
__device__ __forceinline__ void warp_xor_row(ulonglong2 (&acc)[NQ], const ulonglong2* __restrict__ row, uint32_t W,
                                             uint32_t lane) {
#pragma unroll
  for (uint32_t q = 0; q < NQ; q++) {
    const uint32_t b = lane + 32 * q;
    if (b < W) {
      const ulonglong2 x = __ldg(row + b);
      acc[q].x ^= x.x;
      acc[q].y ^= x.y;
    }
  }
}

// One-cluster recovery of graphs of at most kClMaxV vertices
// (recover_small.cu): setup picks it (g->rec_cluster = CTAs of the cluster,
// 0 = the grid-wide kernel), launch runs it.
cudaError_t setup_recover_cluster(cupc_graph* g);
cudaError_t launch_recover_cluster(cupc_graph* g, const RecArgs& a, cudaStream_t s);

}  // namespace cupc
