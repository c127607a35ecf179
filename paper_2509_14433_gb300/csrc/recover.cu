// Spanning-forest recovery by Boruvka rounds over the vertex sketches
// (App. A.1.1, "The AGM Algorithm": query each supernode's merged sketch for
// an edge leaving it, merge supernodes and their sketches, repeat for
// O(log V) rounds) and Connected(u,v) answers from the result (Problem 2).
//
// The whole recovery is one cooperative launch: every CTA is co-resident, and
// the phases of a round are separated by a grid barrier whose wait is bounded
// (on expiry it sets the timeout error and every CTA returns). Round r:
//   group       live vertices grouped by component label (count, segment
//               offsets, scatter); round 0 skips it: every vertex is its own
//               component
//   reduce      components of at most kRecSpan members: a warp per span,
//               lane l XORs buckets l + 32q of layer r of each member; bigger
//               ones in CTA tiles sized to the grid, thread t XORs bucket t.
//               A component inside one span or tile is sampled in place; one
//               over several is XORed into its accumulator and sampled by the
//               last span or tile to finish
//   sample      ZERO / GOOD(edge) / FAIL, first good bucket in index order;
//               32 samples of a warp are booked at once
//   hook        minimum spanning forest (weights = edge ids) of the candidate
//               edges over the round-start components: grid-wide Boruvka
//               steps with min-id edges until at most kSmallHook candidates
//               still cross two trees, then one CTA finishes in shared
//               memory; it adds exactly the edges Kruskal in ascending id
//               order would
//   relabel     every vertex takes the minimum vertex id of its component
// A component whose merged sketch is ZERO has an empty cut; it is not sampled
// again until it changes. With one live component left its merged sketch is
// zero by linearity, so the round is logged without reading its layer.
#include "recover_dev.cuh"

namespace cupc {


// Grid barrier for a cooperative launch: CTA thread 0 adds one to an arrival
// counter that only grows during the launch (the host zeroes it before) and
// waits until all CTAs of this barrier have arrived. The wait is bounded:
// after kWaitLimitNs it records kErrTimeout and returns false in every
// thread of the CTA, which must then return.
__device__ __forceinline__ bool grid_barrier(uint32_t* gc, uint32_t nblocks, uint32_t& epoch, int* s_ok,
                                             uint64_t limit_ns = kWaitLimitNs) {
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += 1;
    const uint32_t target = epoch * nblocks;
    int ok = 1;
    __threadfence();
    atomicAdd(&gc[GC_BAR_COUNT], 1u);
    volatile uint32_t* cnt = gc + GC_BAR_COUNT;
    uint64_t t0 = 0;
    for (uint32_t spin = 0; *cnt < target; spin++) {
      if ((spin & 63) == 63) {
        const uint64_t t = global_timer_ns();
        if (t0 == 0) t0 = t;
        if (ld_cg(&gc[GC_ERR]) & kErrTimeout) {
          ok = 0;
          break;
        }
        if (t - t0 > limit_ns) {
          atomicOr(&gc[GC_ERR], kErrTimeout);
          atomicOr(&gc[GC_REC_DIRTY], 1u);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Root of x in the hook forest; points x straight at it. Other threads may
// rewrite parent[] concurrently, but only ever to an ancestor, so every value
// read is an ancestor and the walk ends at the same root.
__device__ __forceinline__ uint32_t find_root(uint32_t* parent, uint32_t x, uint32_t V) {
  uint32_t r = x;
  for (uint32_t k = 0; k < V; k++) {
    const uint32_t p = ld_cg(&parent[r]);
    if (p == r) break;
    r = p;
  }
  if (r != x && ld_cg(&parent[x]) != r) parent[x] = r;
  return r;
}

// Book the samples stashed in a warp, one per lane (K = kNoneU32: none):
// ZERO marks the component final; GOOD with an edge that leaves K becomes
// its candidate (stored with both endpoint labels) and is logged; GOOD with
// an edge inside K is a checksum false positive. Counters are aggregated per
// warp. Every lane of the warp must call this.
__device__ __forceinline__ void book_samples(const RecArgs& a, uint32_t r, bool multi, uint32_t K, uint32_t res,
                                             uint64_t e) {
  const uint32_t lane = threadIdx.x & 31;
  const bool have = K != kNoneU32;
  bool cand = false;
  if (have) {
    if (res == 0) {
      a.final_[K] = 1;
    } else if (res == 1) {
      const uint32_t u = (uint32_t)(e / a.V), v = (uint32_t)(e % a.V);
      const uint32_t lu = multi ? ld_cg(&a.label[u]) : u, lv = multi ? ld_cg(&a.label[v]) : v;
      if ((lu == K) != (lv == K)) {
        cand = true;
        a.cand[K] = make_ulonglong2(e, ((uint64_t)lu << 32) | lv);
      }
    }
  }
  const uint32_t m_have = __ballot_sync(0xffffffffu, have);
  const uint32_t m_nz = __ballot_sync(0xffffffffu, have && res != 0);
  const uint32_t m_fail = __ballot_sync(0xffffffffu, have && res == 2);
  const uint32_t m_cand = __ballot_sync(0xffffffffu, cand);
  const uint32_t m_fp = m_nz & ~m_fail & ~m_cand;
  uint32_t base = 0;
  if (lane == 0) {
    if (m_have) atomicAdd(&a.log_live[r], (uint32_t)__popc(m_have));
    if (m_nz) atomicAdd(&a.gc[GC_NZ], (uint32_t)__popc(m_nz));
    if (m_fail) atomicAdd(&a.gc[GC_NFAIL], (uint32_t)__popc(m_fail));
    if (m_fp) atomicAdd(&a.gc[GC_NFP], (uint32_t)__popc(m_fp));
    if (m_cand) {
      base = atomicAdd(&a.gc[GC_LOGLEN], (uint32_t)__popc(m_cand));
      atomicAdd(&a.log_ncand[r], (uint32_t)__popc(m_cand));
    }
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  if (cand) a.log_ids[base + __popc(m_cand & ((1u << lane) - 1))] = e;
}

// Position of this lane's item in ctr[key]'s range: lanes of the warp with
// the same key share one atomicAdd. All 32 lanes call it; `take` selects the
// lanes that add one item.
__device__ __forceinline__ uint32_t warp_grab(uint32_t* ctr, uint32_t key, bool take) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t act = __ballot_sync(0xffffffffu, take);
  uint32_t pos = 0;
  if (take) {
    const uint32_t peers = __match_any_sync(act, key);
    const uint32_t leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&ctr[key], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    pos = base + __popc(peers & ((1u << lane) - 1));
  }
  return pos;
}

constexpr uint32_t kBigFlag = 0x80000000u;  // roff[K] flag: K's members are in permb
constexpr uint32_t kTileSegs = 2 + kRecTile / (kRecSpan + 1);  // components meeting one tile


// Root in a shared-memory forest with path halving; concurrent halving only
// ever points a node at an ancestor.
__device__ __forceinline__ uint32_t s_find(volatile uint32_t* par, uint32_t x) {
  for (uint32_t k = 0; k < 2 * kSmallHook; k++) {  // a path is shorter than the node count
    const uint32_t y = par[x];
    if (y == x) break;
    const uint32_t z = par[y];
    if (z != y) par[x] = z;
    x = y;
  }
  return x;
}

// The rest of a hook, run by one CTA once at most kSmallHook candidates
// still cross two trees (hlist[0..n): edge, both current roots): the same
// minimum spanning forest by Boruvka as the grid-wide steps (a root's key is
// edge << 11 | the root on the other side; two roots that chose the same
// edge hook once, the larger under the smaller), over local node ids, with
// __syncthreads between steps and pointer jumping after each hook step.
// Publishes parent[] of the roots that hooked and appends the forest edges.
// smem: 32 KB.
__device__ void small_hook(const RecArgs& a, uint32_t n, unsigned char* smem) {
  constexpr uint32_t kPer = kSmallHook / kRecThreads;  // candidates per thread
  constexpr uint32_t kNodeBits = 11;                    // nodes < 2 * kSmallHook
  static_assert(2 * kSmallHook <= (1u << kNodeBits), "node ids fit the key");
  uint64_t* s_best = reinterpret_cast<uint64_t*>(smem);  // 2 * kSmallHook
  uint32_t* s_par = reinterpret_cast<uint32_t*>(s_best + 2 * kSmallHook);
  uint32_t* s_lab = s_par + 2 * kSmallHook;  // node -> global root
  __shared__ uint32_t s_nn, s_nf, s_f0;
  const uint32_t tid = threadIdx.x, bd = blockDim.x;
  if (tid == 0) {
    s_nn = 0;
    s_nf = 0;
    s_f0 = ld_cg(&a.gc[GC_NFOREST]);  // the other CTAs wait at the grid barrier: this CTA owns the count
  }
  for (uint32_t x = tid; x < 2 * kSmallHook; x += bd) s_lab[x] = kNoneU32;
  __syncthreads();
  // node ids of the roots: the first claim of root x (a CAS on pcount[x],
  // zero at rest during the hook and cleared again at the end) takes a new
  // id, later claims read it; an id whose claim lost stays unused. All of a
  // thread's claims are in flight at once.
  uint64_t ce[kPer];  // this thread's candidates: edge, node pair
  uint32_t cab[kPer], root[2 * kPer], mine[2 * kPer], prev[2 * kPer];
#pragma unroll
  for (uint32_t k = 0; k < kPer; k++) {
    const uint32_t i = tid + k * bd;
    ce[k] = kNone;
    if (i < n) {
      const ulonglong2 h = __ldcg(&a.hlist[i]);
      ce[k] = h.x;
      root[2 * k] = (uint32_t)(h.y >> 32);
      root[2 * k + 1] = (uint32_t)h.y;
    }
  }
#pragma unroll
  for (uint32_t j = 0; j < 2 * kPer; j++)
    if (ce[j / 2] != kNone) mine[j] = atomicAdd(&s_nn, 1u);
#pragma unroll
  for (uint32_t j = 0; j < 2 * kPer; j++)
    if (ce[j / 2] != kNone) prev[j] = atomicCAS(&a.pcount[root[j]], 0u, mine[j] + 1);
#pragma unroll
  for (uint32_t k = 0; k < kPer; k++) {
    cab[k] = kNoneU32;
    if (ce[k] == kNone) continue;
    uint32_t node[2];
#pragma unroll
    for (uint32_t q = 0; q < 2; q++) {
      const uint32_t j = 2 * k + q;
      if (prev[j] == 0) s_lab[mine[j]] = root[j];
      node[q] = prev[j] == 0 ? mine[j] : prev[j] - 1;
    }
    cab[k] = node[0] | (node[1] << 16);
  }
  __syncthreads();
  const uint32_t nn = s_nn;
  for (uint32_t x = tid; x < nn; x += bd) {
    s_par[x] = x;
    s_best[x] = kNone;
  }
  __syncthreads();
  for (uint32_t iter = 0; iter < 64; iter++) {
    int any = 0;
#pragma unroll
    for (uint32_t k = 0; k < kPer; k++) {
      if (cab[k] == kNoneU32) continue;
      const uint32_t ra = s_find(s_par, cab[k] & 0xFFFFu), rb = s_find(s_par, cab[k] >> 16);
      if (ra != rb) {  // read first: most proposals to a big tree's root lose
        const uint64_t ka = ce[k] << kNodeBits | rb, kb = ce[k] << kNodeBits | ra;
        if (ka < s_best[ra]) atomicMin((unsigned long long*)&s_best[ra], (unsigned long long)ka);
        if (kb < s_best[rb]) atomicMin((unsigned long long*)&s_best[rb], (unsigned long long)kb);
        any = 1;
      } else {
        cab[k] = kNoneU32;  // both ends in one tree: never crosses again
      }
    }
    if (!__syncthreads_or(any)) break;
    for (uint32_t x = tid; x < nn; x += bd) {
      const uint64_t key = s_best[x];
      if (key == kNone) continue;
      const uint64_t e = key >> kNodeBits;
      const uint32_t o = (uint32_t)key & ((1u << kNodeBits) - 1);
      if ((s_best[o] >> kNodeBits) != e || x > o) {
        s_par[x] = o;
        a.forest[s_f0 + atomicAdd(&s_nf, 1u)] = e;
      }
    }
    __syncthreads();
    // flatten by pointer jumping, so that the next finds take one hop (the
    // hooks just made can form long chains); every value read is an ancestor
    for (uint32_t x = tid; x < nn; x += bd) s_best[x] = kNone;
    for (uint32_t pass = 0; pass < 16; pass++) {  // depth < 2^11 needs at most 11 passes
      int moved = 0;
      for (uint32_t x = tid; x < nn; x += bd) {
        const uint32_t p = s_par[x], pp = s_par[p];
        if (p != pp) {
          s_par[x] = pp;
          moved = 1;
        }
      }
      if (!__syncthreads_or(moved)) break;
    }
  }
  for (uint32_t x = tid; x < nn; x += bd) {
    const uint32_t lab = s_lab[x];
    if (lab == kNoneU32) continue;  // an id whose claim lost
    const uint32_t rt = s_find(s_par, x);
    if (rt != x) a.parent[lab] = s_lab[rt];
    a.pcount[lab] = 0;
  }
  if (tid == 0) a.gc[GC_NFOREST] = s_f0 + s_nf;
}

__global__ void __launch_bounds__(kRecThreads, 2) k_recover(RecArgs a) {
  __shared__ int s_ok;
  __shared__ uint32_t t_w[kRecTile], t_k[kRecTile + 1];
  static_assert(kRecTile <= kRecThreads, "one member id per thread");
  static_assert(sizeof(ulonglong2) * kTileSegs * kRecThreads >= 2 * kSmallHook * (8 + 4 + 4),
                "small_hook lives in t_stage");
  static_assert(kSmallHook % kRecThreads == 0, "small_hook: whole candidates per thread");
  __shared__ ulonglong2 t_stage[kTileSegs][kRecThreads];
  __shared__ uint32_t t_seg_k[kTileSegs];
  const uint32_t V = a.V, W = a.W, nb = gridDim.x, tid = threadIdx.x, lane = tid & 31;
  const uint32_t gtid = blockIdx.x * blockDim.x + tid, gstride = gridDim.x * blockDim.x;
  const uint32_t wpb = blockDim.x >> 5, gwarp = blockIdx.x * wpb + (tid >> 5), nwarps = gridDim.x * wpb;
  uint32_t* gc = a.gc;
  uint32_t epoch = 0;
#define CUPC_GRID_SYNC() \
  if (!grid_barrier(gc, nb, epoch, &s_ok)) return

  // incremental mode: the updates since the last recovery kept the labels
  // exact (see k_incr), so there is nothing to recover; or they deleted
  // forest edges (of the recovered forest, or added by merges since): then
  // the components are unions of the fragments of the remaining forest, and
  // Boruvka starts from those (warm start) instead of from single vertices
  const bool valid = ld_cg(&gc[GC_LABELS_VALID]) != 0, warm = !a.force && valid && ld_cg(&gc[GC_WARM]) != 0;
  if (!a.force && valid && !warm) return;
  const uint32_t nsorted = warm ? min(ld_cg(&gc[GC_NSORTED]), V) : 0;
  const uint32_t nadd = warm ? min(ld_cg(&gc[GC_NFADD]), V) : 0;
  // after a recovery that gave up at a barrier, the reduce accumulators and
  // the last-arriver counters may hold partial sums: clear them first
  const bool dirty = ld_cg(&gc[GC_REC_DIRTY]) != 0;
  for (uint32_t w = gtid; w < V; w += gstride) {
    a.label[w] = w;
    a.final_[w] = 0;
    a.parent[w] = w;
    a.minv[w] = kNoneU32;
    a.merged[w] = 0;
    a.cand[w] = make_ulonglong2(kNone, 0);
    a.best0[w] = kNone;
    a.best1[w] = kNone;
    a.rcnt[w] = 0;
    a.ipar[w] = w;
    if (!warm) a.fdead[w] = 0;  // a warm start reads them first
    if (dirty) a.pcount[w] = 0;
  }
  if (dirty)
    for (size_t i = gtid; i < (size_t)V * W; i += gstride) a.acc[i] = make_ulonglong2(0, 0);
  if (a.inc)  // the merge-edge table starts empty (fadd itself is read by a warm start below)
    for (size_t i = gtid; i < ((size_t)1 << a.ftab_bits); i += gstride) a.ftab[i] = 0ull;
  if (gtid == 0) {
    gc[GC_NLIVE] = 0;
    gc[GC_NFOREST] = 0;
    gc[GC_NFAIL] = 0;
    gc[GC_NFP] = 0;
    gc[GC_LOGLEN] = 0;
    gc[GC_COMPLETE] = 0;
    gc[GC_ROUNDS] = 0;
    gc[GC_NZ] = 0;
    gc[GC_ACTIVE] = 0;
    gc[GC_ACTIVE_ODD] = 0;
    gc[GC_NMEMBERS] = 0;
    gc[GC_NBIG] = 0;
    gc[GC_RECOVERIES] += 1;
  }
  for (uint32_t r = gtid; r < a.L; r += gstride) {
    a.log_live[r] = 0;
    a.log_ncand[r] = 0;
  }
  CUPC_GRID_SYNC();
  if (gtid == 0) {  // every CTA has read them (the early return and warm above depend on them)
    if (dirty) gc[GC_REC_DIRTY] = 0;
    gc[GC_NFADD] = 0;
    gc[GC_LABELS_VALID] = 0;
    gc[GC_FOREST_SORTED] = 0;
    gc[GC_WARM] = 0;
  }
  if (warm) {
    // fragments: union the endpoints of the forest edges still present (the
    // larger root under the smaller): the recovered forest's, then those
    // merges added. An edge whose union joins two fragments starts the new
    // forest (all of them with a valid stream; at most V - 1 in any case).
    const uint32_t nall = nsorted + nadd;
    for (uint32_t base = gwarp * 32; base < nall; base += nwarps * 32) {
      const uint32_t i = base + lane;
      bool keep = false;
      uint64_t e = 0;
      if (i < nsorted) {
        keep = !a.fdead[i];
        e = a.forest_sorted[i];
      } else if (i < nall) {
        keep = !a.fadd_dead[i - nsorted];
        e = a.fadd[i - nsorted];
      }
      if (keep) {
        uint32_t x = (uint32_t)(e / V), y = (uint32_t)(e % V);
        keep = false;
        for (uint32_t k = 0; k < V && x < V && y < V; k++) {  // bounded: each failed CAS is another thread's progress
          x = find_root(a.parent, x, V);
          y = find_root(a.parent, y, V);
          if (x == y) break;
          if (x > y) {
            const uint32_t t = x;
            x = y;
            y = t;
          }
          if (atomicCAS(&a.parent[y], y, x) == y) {
            keep = true;
            break;
          }
        }
      }
      const uint32_t m = __ballot_sync(0xffffffffu, keep);
      uint32_t at = 0;
      if (lane == 0 && m) at = atomicAdd(&gc[GC_NFOREST], (uint32_t)__popc(m));
      at = __shfl_sync(0xffffffffu, at, 0);
      if (keep) a.forest[at + __popc(m & ((1u << lane) - 1))] = e;
    }
    CUPC_GRID_SYNC();
    for (uint32_t w = gtid; w < V; w += gstride) a.label[w] = find_root(a.parent, w, V);  // the minimum id
    CUPC_GRID_SYNC();
    // A fragment that holds no endpoint of a deleted forest edge is a whole
    // component of the last complete recovery, joined with others only by
    // recorded merges: its cut is empty, so it starts final (its sample
    // would be ZERO). Only the split components are sampled again.
    for (uint32_t w = gtid; w < V; w += gstride)
      if (ld_cg(&a.label[w]) == w) a.final_[w] = 1;
    CUPC_GRID_SYNC();
    for (uint32_t i = gtid; i < nall; i += gstride) {
      const bool dead = i < nsorted ? a.fdead[i] != 0 : a.fadd_dead[i - nsorted] != 0;
      if (!dead) continue;
      const uint64_t e = i < nsorted ? a.forest_sorted[i] : a.fadd[i - nsorted];
      const uint32_t x = (uint32_t)(e / V), y = (uint32_t)(e % V);
      if (x < V && y < V) {
        a.final_[ld_cg(&a.label[x])] = 0;
        a.final_[ld_cg(&a.label[y])] = 0;
      }
    }
    CUPC_GRID_SYNC();
    // the split fragments are the live components of the first round: count members
    for (uint32_t base = gwarp * 32; base < V; base += nwarps * 32) {
      const uint32_t w = base + lane;
      uint32_t lab = 0;
      bool live = false;
      if (w < V) {
        lab = ld_cg(&a.label[w]);
        live = !ld_cg(&a.final_[lab]);
        a.parent[w] = w;
        a.fdead[w] = 0;
      }
      const uint32_t m_first = __ballot_sync(0xffffffffu, warp_grab(a.rcnt, lab, live) == 0 && live);
      if (lane == 0 && m_first) atomicAdd(&gc[GC_NLIVE], (uint32_t)__popc(m_first));
    }
    CUPC_GRID_SYNC();
  }

  for (uint32_t r = 0; r < a.L; r++) {
    const uint64_t kchk = a.keys[r * (a.C + 1) + a.C];
    const bool multi = r > 0 || warm;  // components may have several members
    // One live component left: every other component is final, and a final
    // component's merged sketch is zero (its cut is empty); the XOR of all
    // vertex sketches of a layer is zero (each edge enters both endpoints),
    // so the live one's merged sketch is zero too and it samples ZERO. Log
    // the round as sampled (one live component, no candidate) and stop.
    // Imported words need not come from a stream: then the round is run.
    if (multi && a.sum_zero && ld_cg(&gc[GC_NLIVE]) == 1) {
      if (gtid == 0) {
        a.log_live[r] = 1;
        gc[GC_ROUNDS] = r + 1;
        gc[GC_COMPLETE] = 1;
      }
      break;
    }
    // ---- group the live vertices of round r by component: the relabel of
    // round r-1 counted them; give each component a segment (warp-aggregated
    // atomics), then scatter
    uint32_t nmem = V;
    if (multi) {
      for (uint32_t base = blockIdx.x * blockDim.x; base < V; base += gstride) {
        const uint32_t K = base + tid;
        const uint32_t c = K < V ? ld_cg(&a.rcnt[K]) : 0;
        const bool big = c > kRecSpan;
        uint32_t is = big ? 0 : c, ib = big ? c : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t ys = __shfl_up_sync(0xffffffffu, is, o), yb = __shfl_up_sync(0xffffffffu, ib, o);
          if (lane >= (uint32_t)o) {
            is += ys;
            ib += yb;
          }
        }
        const uint32_t ts = __shfl_sync(0xffffffffu, is, 31), tb = __shfl_sync(0xffffffffu, ib, 31);
        uint32_t bs = 0, bb = 0;
        if (lane == 31 && ts) bs = atomicAdd(&gc[GC_NMEMBERS], ts);
        if (lane == 31 && tb) bb = atomicAdd(&gc[GC_NBIG], tb);
        bs = __shfl_sync(0xffffffffu, bs, 31);
        bb = __shfl_sync(0xffffffffu, bb, 31);
        if (c) {
          const uint32_t at = big ? bb + ib - c : bs + is - c;
          a.roff[K] = big ? (at | kBigFlag) : at;
          a.rcnt[K] = at;  // scatter cursor, then the segment end
        }
        if (K < V) {
          a.parent[K] = K;
          a.minv[K] = kNoneU32;
          a.merged[K] = 0;
        }
      }
      CUPC_GRID_SYNC();
      for (uint32_t base = gwarp * 32; base < V; base += nwarps * 32) {
        const uint32_t w = base + lane;
        const uint32_t K = w < V ? ld_cg(&a.label[w]) : 0;
        const bool live = w < V && !ld_cg(&a.final_[K]);
        const uint32_t pos = warp_grab(a.rcnt, K, live);
        if (live) ((ld_cg(&a.roff[K]) & kBigFlag) ? a.permb : a.perm)[pos] = w;
      }
      CUPC_GRID_SYNC();
      nmem = ld_cg(&gc[GC_NMEMBERS]);
    }

    // ---- reduce + sample, one warp per span of members (round 0: one
    // vertex per span, every vertex is its own component). A component over
    // several spans is XORed into acc[K]; the last span to finish samples it.
    if (multi) {
      // big components (more than kRecSpan members): each CTA takes one
      // contiguous chunk of their members and walks it in tiles of up to
      // kRecTile, thread t XORing bucket t of every member (8 rows in
      // flight). A component's partial sum carries from one tile to the
      // next, so that a CTA ends each component once: a component inside
      // one chunk is sampled by one warp, one over several chunks is XORed
      // into acc[K] once per chunk (the last chunk to finish samples it).
      const uint32_t nbig = ld_cg(&gc[GC_NBIG]);
      const uint32_t chunk = max(8u, (((nbig + nb - 1) / nb) + 7) & ~7u);
      const uint32_t c0 = min(nbig, blockIdx.x * chunk), c1 = min(nbig, c0 + chunk);
      ulonglong2 acc1 = make_ulonglong2(0, 0);
      for (uint32_t m0 = c0; m0 < c1; m0 += kRecTile) {
        const uint32_t cnt = min(kRecTile, c1 - m0);
        if (tid < cnt) {
          const uint32_t w = ld_cg(&a.permb[m0 + tid]);
          t_w[tid] = w;
          t_k[tid] = ld_cg(&a.label[w]);
        } else if (tid == cnt) {  // the next tile's first label, or none at the chunk's end
          t_k[cnt] = m0 + cnt < c1 ? ld_cg(&a.label[ld_cg(&a.permb[m0 + cnt])]) : kNoneU32;
        }
        __syncthreads();
        uint32_t nseg = 0;
        for (uint32_t m = 0; m < cnt; m += 8) {
          ulonglong2 x[8];
#pragma unroll
          for (uint32_t k = 0; k < 8; k++) {
            x[k] = make_ulonglong2(0, 0);
            if (tid < W && m + k < cnt) x[k] = __ldg(a.sketch + ((size_t)r * V + t_w[m + k]) * W + tid);
          }
#pragma unroll
          for (uint32_t k = 0; k < 8; k++) {
            const uint32_t mm = m + k;
            if (mm < cnt) {
              acc1.x ^= x[k].x;
              acc1.y ^= x[k].y;
              if (t_k[mm + 1] != t_k[mm]) {  // a component's part of this chunk ends here
                t_stage[nseg][tid] = acc1;
                acc1 = make_ulonglong2(0, 0);
                if (tid == 0) t_seg_k[nseg] = t_k[mm];
                nseg++;
              }
            }
          }
        }
        __syncthreads();
        for (uint32_t sg = tid >> 5; sg < nseg; sg += wpb) {
          const uint32_t K = t_seg_k[sg];
          const uint32_t s0 = ld_cg(&a.roff[K]) & ~kBigFlag, s1 = ld_cg(&a.rcnt[K]);
          const uint32_t ntk = (s1 - 1) / chunk - s0 / chunk + 1;  // chunks it meets
          ulonglong2 acc[kWarpBuckets];
#pragma unroll
          for (uint32_t q = 0; q < kWarpBuckets; q++) acc[q] = t_stage[sg][lane + 32 * q];
          bool mine = true;
          if (ntk > 1) {
            ulonglong2* dst = a.acc + (size_t)K * W;
#pragma unroll
            for (uint32_t q = 0; q < kWarpBuckets; q++) {
              const uint32_t b = lane + 32 * q;
              if (b < W && (acc[q].x | acc[q].y)) {
                atomicXor(&dst[b].x, acc[q].x);
                atomicXor(&dst[b].y, acc[q].y);
              }
            }
            __threadfence();
            uint32_t prev = 0;
            if (lane == 0) prev = atomicAdd(&a.pcount[K], 1u);
            mine = __shfl_sync(0xffffffffu, prev, 0) + 1 == ntk;
            if (mine) {
              __threadfence();
#pragma unroll
              for (uint32_t q = 0; q < kWarpBuckets; q++) {
                const uint32_t b = lane + 32 * q;
                acc[q] = make_ulonglong2(0, 0);
                if (b < W) {
                  acc[q] = __ldcg(dst + b);
                  dst[b] = make_ulonglong2(0, 0);
                }
              }
              if (lane == 0) a.pcount[K] = 0;
            }
          }
          if (mine) {
            uint64_t e = 0;
            const uint32_t res = warp_sample(acc, W, V, kchk, e);
            book_samples(a, r, multi, lane == 0 ? K : kNoneU32, res, e);
          }
        }
        __syncthreads();
      }
    }

    // small components (and every vertex in round 0): one warp per span
    const uint32_t span = multi ? kRecSpan : 1u;
    const uint32_t nspans = (nmem + span - 1) / span;
    uint32_t st_k = kNoneU32, st_res = 0, nst = 0;  // this lane's stashed sample
    uint64_t st_e = 0;
    for (uint32_t sp = gwarp; sp < nspans; sp += nwarps) {
      const uint32_t i0 = sp * span, cnt = min(span, nmem - i0);
      if (!multi && sp + nwarps < nspans && lane * 8 < W)  // round 0: bring this warp's next row to L2
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.sketch + (size_t)(sp + nwarps) * W + lane * 8));
      uint32_t mw = 0, mk = kNoneU32;
      if (lane < cnt) {
        mw = multi ? ld_cg(&a.perm[i0 + lane]) : i0 + lane;
        mk = multi ? ld_cg(&a.label[mw]) : mw;
      }
      if (multi && lane < cnt) {  // every member's row heads for L2 while the first ones fold
        const ulonglong2* row = a.sketch + ((size_t)r * V + mw) * W;
        for (uint32_t b = 0; b < W; b += 8) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + b));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(row + W - 1));
      }
      uint32_t i = 0;
      while (i < cnt) {
        const uint32_t K = __shfl_sync(0xffffffffu, mk, i);
        const uint32_t rest = ~(__ballot_sync(0xffffffffu, mk == K) >> i);
        const uint32_t j = i + (rest ? (uint32_t)__ffs(rest) - 1 : 32 - i);
        ulonglong2 acc[kWarpBuckets];
#pragma unroll
        for (uint32_t q = 0; q < kWarpBuckets; q++) acc[q] = make_ulonglong2(0, 0);
        for (uint32_t m = i; m < j; m++) {
          const uint32_t w = __shfl_sync(0xffffffffu, mw, m);
          warp_xor_row(acc, a.sketch + ((size_t)r * V + w) * W, W, lane);
        }
        uint32_t nsp = 1;
        if (multi) {
          const uint32_t s0 = ld_cg(&a.roff[K]), s1 = ld_cg(&a.rcnt[K]);
          nsp = (s1 - 1) / span - s0 / span + 1;
        }
        bool mine = true;
        if (nsp > 1) {
          ulonglong2* dst = a.acc + (size_t)K * W;
#pragma unroll
          for (uint32_t q = 0; q < kWarpBuckets; q++) {
            const uint32_t b = lane + 32 * q;
            if (b < W && (acc[q].x | acc[q].y)) {
              atomicXor(&dst[b].x, acc[q].x);
              atomicXor(&dst[b].y, acc[q].y);
            }
          }
          __threadfence();
          uint32_t prev = 0;
          if (lane == 0) prev = atomicAdd(&a.pcount[K], 1u);
          mine = __shfl_sync(0xffffffffu, prev, 0) + 1 == nsp;
          if (mine) {  // the last span: every other span's XOR is in acc[K]
            __threadfence();
#pragma unroll
            for (uint32_t q = 0; q < kWarpBuckets; q++) {
              const uint32_t b = lane + 32 * q;
              acc[q] = make_ulonglong2(0, 0);
              if (b < W) {
                acc[q] = __ldcg(dst + b);
                dst[b] = make_ulonglong2(0, 0);
              }
            }
            if (lane == 0) a.pcount[K] = 0;
          }
        }
        if (mine) {
          uint64_t e = 0;
          const uint32_t res = warp_sample(acc, W, V, kchk, e);
          if (lane == nst) {
            st_k = K;
            st_res = res;
            st_e = e;
          }
          if (++nst == 32) {  // book 32 samples at once, one per lane
            book_samples(a, r, multi, st_k, st_res, st_e);
            st_k = kNoneU32;
            nst = 0;
          }
        }
        i = j;
      }
    }
    if (nst) book_samples(a, r, multi, st_k, st_res, st_e);
    CUPC_GRID_SYNC();
    if (gtid == 0) gc[GC_ROUNDS] = r + 1;
    if (ld_cg(&gc[GC_NZ]) == 0) {
      if (gtid == 0) gc[GC_COMPLETE] = 1;
      break;
    }

    // ---- hook: minimum spanning forest of the candidates by Boruvka. A
    // root's key is edge << vbits | (root on the other side), so the min key names
    // the min-id crossing edge and where it leads; two roots that chose the
    // same edge hook once (the larger id under the smaller). A round with
    // few candidates hooks in one CTA (small_hook) behind a single barrier.
    const uint32_t vbits = 32 - __clz(V - 1);  // bits of a vertex id (V <= 2^21: keys fit 64 bits)
    const uint64_t vmask = (1ull << vbits) - 1;
    for (uint32_t iter = 0; iter < 64; iter++) {
      uint64_t* bc = (iter & 1) ? a.best1 : a.best0;
      uint64_t* bn = (iter & 1) ? a.best0 : a.best1;
      // candidates still crossing two trees: count them, list the first kSmallHook
      const uint32_t act = (iter & 1) ? GC_ACTIVE_ODD : GC_ACTIVE, act_next = (iter & 1) ? GC_ACTIVE : GC_ACTIVE_ODD;
      for (uint32_t base = gwarp * 32; base < V; base += nwarps * 32) {
        const uint32_t K = base + lane;
        bool cross = false;
        uint64_t e = 0;
        uint32_t ra = 0, rb = 0;
        if (K < V) {
          const ulonglong2 c = __ldcg(&a.cand[K]);
          if (c.x != kNone) {
            e = c.x;
            ra = find_root(a.parent, (uint32_t)(c.y >> 32), V);
            rb = find_root(a.parent, (uint32_t)c.y, V);
            if (ra != rb) {  // read first: most proposals to a big tree's root lose
              const uint64_t ka = e << vbits | rb, kb = e << vbits | ra;
              if (ka < ld_cg(&bc[ra])) atomicMin((unsigned long long*)&bc[ra], (unsigned long long)ka);
              if (kb < ld_cg(&bc[rb])) atomicMin((unsigned long long*)&bc[rb], (unsigned long long)kb);
              cross = true;
            }
          }
        }
        const uint32_t m = __ballot_sync(0xffffffffu, cross);
        if (m) {
          uint32_t at = 0;
          if (lane == 0) at = atomicAdd(&gc[act], (uint32_t)__popc(m));
          at = __shfl_sync(0xffffffffu, at, 0) + __popc(m & ((1u << lane) - 1));
          if (cross && at < kSmallHook) a.hlist[at] = make_ulonglong2(e, (uint64_t)ra << 32 | rb);
        }
      }
      CUPC_GRID_SYNC();
      const uint32_t nact = ld_cg(&gc[act]);
      if (nact == 0) break;
      if (nact <= kSmallHook) {  // finish in one CTA behind a single barrier
        if (blockIdx.x == 0) small_hook(a, nact, reinterpret_cast<unsigned char*>(&t_stage[0][0]));
        CUPC_GRID_SYNC();
        break;
      }
      for (uint32_t base = gwarp * 32; base < V; base += nwarps * 32) {
        const uint32_t x = base + lane;
        bool hook = false;
        uint64_t e = 0;
        uint32_t o = 0;
        if (x < V) {
          bn[x] = kNone;
          const uint64_t key = ld_cg(&bc[x]);
          if (key != kNone) {
            e = key >> vbits;
            o = (uint32_t)(key & vmask);
            const bool mutual = (ld_cg(&bc[o]) >> vbits) == e;
            hook = !mutual || x > o;
          }
        }
        const uint32_t m = __ballot_sync(0xffffffffu, hook);
        if (m) {
          uint32_t at = 0;
          if (lane == 0) at = atomicAdd(&gc[GC_NFOREST], (uint32_t)__popc(m));
          at = __shfl_sync(0xffffffffu, at, 0);
          if (hook) {
            a.parent[x] = o;
            a.forest[at + __popc(m & ((1u << lane) - 1))] = e;
          }
        }
      }
      if (gtid == 0) gc[act_next] = 0;
      CUPC_GRID_SYNC();
    }

    // ---- relabel to the minimum vertex id of each component; clear the
    // round's scratch
    for (uint32_t base = gwarp * 32; base < V; base += nwarps * 32) {
      const uint32_t w = base + lane;
      bool lab = false;
      uint32_t root = 0;
      if (w < V) {
        a.rcnt[w] = 0;
        a.cand[w] = make_ulonglong2(kNone, 0);
        a.best0[w] = kNone;
        a.best1[w] = kNone;
        if (ld_cg(&a.label[w]) == w) {
          lab = true;
          root = find_root(a.parent, w, V);
        }
      }
      const uint32_t act = __ballot_sync(0xffffffffu, lab);
      if (lab) {  // the lanes of one root: min id and "merged" with one write each
        const uint32_t peers = __match_any_sync(act, root);
        const uint32_t mn = __reduce_min_sync(peers, w);
        const bool mg = __any_sync(peers, root != w);
        if (lane == (uint32_t)__ffs(peers) - 1) {
          atomicMin(&a.minv[root], mn);
          if (mg) a.merged[root] = 1;
        }
      }
    }
    if (gtid == 0) {
      gc[GC_NZ] = 0;
      gc[GC_NMEMBERS] = 0;
      gc[GC_NBIG] = 0;
      gc[GC_ACTIVE] = 0;
      gc[GC_ACTIVE_ODD] = 0;
      gc[GC_NLIVE] = 0;
    }
    CUPC_GRID_SYNC();
    // new labels; the members of next round's live components are counted
    // here (a merged component is live; an unmerged one keeps its flag)
    for (uint32_t base = gwarp * 32; base < V; base += nwarps * 32) {
      const uint32_t w = base + lane;
      uint32_t nl = 0;
      bool live = false;
      if (w < V) {
        const uint32_t K = ld_cg(&a.label[w]);
        const uint32_t root = find_root(a.parent, K, V);
        nl = ld_cg(&a.minv[root]);
        const bool mg = ld_cg(&a.merged[root]) != 0;
        a.label[w] = nl;
        if (w == root && mg) a.final_[nl] = 0;
        live = mg || !ld_cg(&a.final_[root]);
      }
      // the member that took position 0 of its component counts the component
      const uint32_t m_first = __ballot_sync(0xffffffffu, warp_grab(a.rcnt, nl, live) == 0 && live);
      if (lane == 0 && m_first) atomicAdd(&gc[GC_NLIVE], (uint32_t)__popc(m_first));
    }
    CUPC_GRID_SYNC();
  }
  // a complete recovery starts an incremental epoch
  if (a.inc && gtid == 0) gc[GC_LABELS_VALID] = ld_cg(&gc[GC_COMPLETE]);
#undef CUPC_GRID_SYNC
}

// Self-test of the bounded waits: every CTA but `absent` meets at two grid
// barriers; `absent` returns at once, so the others give up after limit_ns
// and record kErrTimeout.
__global__ void k_wait_selftest(uint32_t* gc, uint32_t absent, uint64_t limit_ns) {
  __shared__ int s_ok;
  uint32_t epoch = 0;
  if (blockIdx.x == absent) return;
  if (!grid_barrier(gc, gridDim.x, epoch, &s_ok, limit_ns)) return;
  grid_barrier(gc, gridDim.x, epoch, &s_ok, limit_ns);
}

cudaError_t setup_recover(cupc_graph* g) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_recover, kRecThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // about four vertices per warp in round 0 (every vertex samples its own
  // sketch); fewer CTAs for small V keep the grid barriers cheap
  uint32_t want = (g->V + 31) / 32;
  if (want < 16) want = 16;
  uint32_t cap = (uint32_t)(per_sm * g->sms);
  g->rec_grid = (int)(want < cap ? want : cap);
  return setup_recover_cluster(g);
}

cudaError_t launch_recover(cupc_graph* g, cudaStream_t s, bool force) {
  RecArgs a;
  a.sketch = g->sketch;
  a.keys = g->keys;
  a.V = g->V;
  a.L = g->L;
  a.C = g->C;
  a.D = g->D;
  a.W = g->W;
  a.label = g->label;
  a.parent = g->parent;
  a.minv = g->minv;
  a.rcnt = g->rcnt;
  a.roff = g->roff;
  a.perm = g->perm;
  a.permb = g->permb;
  a.pcount = g->pcount;
  a.final_ = g->final_;
  a.merged = g->merged;
  a.best0 = g->best;
  a.best1 = g->best2;
  a.cand = g->cand;
  a.forest = g->forest;
  a.log_ids = g->log_ids;
  a.acc = g->acc;
  a.log_live = g->log_live;
  a.log_ncand = g->log_ncand;
  a.hlist = g->hlist;
  a.ipar = g->ipar;
  a.forest_sorted = g->forest_sorted;
  a.fdead = g->fdead;
  a.fadd = g->fadd;
  a.fadd_dead = g->fadd_dead;
  a.ftab = (unsigned long long*)g->ftab;
  a.ftab_bits = g->ftab_bits;
  a.inc = g->inc ? 1u : 0u;
  a.force = force ? 1u : 0u;
  a.sum_zero = g->imported ? 0u : 1u;
  a.gc = g->gc;
  if (g->rec_cluster) {
    ProfScope ps(g, s, PC_RECOVER, 1);
    return launch_recover_cluster(g, a, s);
  }
  cudaError_t e = cudaMemsetAsync(g->gc + GC_BAR_COUNT, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  ProfScope ps(g, s, PC_RECOVER, 1);
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)k_recover, dim3(g->rec_grid), dim3(kRecThreads), args, 0, s);
}

}  // namespace cupc

extern "C" cupc_status cupc_selftest_wait_timeout(uint32_t ctas, uint32_t limit_us, int absent_cta,
                                                  cupc_stream stream) {
  using namespace cupc;
  if (ctas < 2 || ctas > 64 || limit_us == 0 || limit_us > 1000000) return CUPC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* gc = nullptr;
  if (cudaMalloc((void**)&gc, GC_SLOTS * sizeof(uint32_t)) != cudaSuccess) return CUPC_ENOMEM;
  cupc_status st = CUPC_OK;
  uint32_t h[GC_SLOTS];
  uint32_t absent = absent_cta < 0 ? 0xFFFFFFFFu : (uint32_t)absent_cta;
  uint64_t limit = (uint64_t)limit_us * 1000;
  void* args[] = {&gc, &absent, &limit};
  if (cudaMemsetAsync(gc, 0, GC_SLOTS * sizeof(uint32_t), s) != cudaSuccess ||
      cudaLaunchCooperativeKernel((const void*)k_wait_selftest, dim3(ctas), dim3(32), args, 0, s) != cudaSuccess ||
      cudaMemcpyAsync(h, gc, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    st = CUPC_ECUDA;
  } else if (h[GC_ERR] & kErrTimeout) {
    st = CUPC_ETIMEOUT;
  }
  cudaFree(gc);
  return st;
}

namespace cupc {

// ---- Connected(u,v) from the recovered labels (Problem 2)
__global__ void k_query(const uint32_t* __restrict__ pairs, size_t m, uint8_t* __restrict__ out,
                        const uint32_t* __restrict__ label, uint32_t V, uint32_t* gc) {
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t u = pairs[2 * i], v = pairs[2 * i + 1];
    if (u >= V || v >= V) {
      bad = true;
      out[i] = 0;
    } else {
      out[i] = __ldcg(&label[u]) == __ldcg(&label[v]);
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&gc[GC_ERR], kErrQuery);
}

cudaError_t launch_query(cupc_graph* g, const uint32_t* pairs, size_t m, uint8_t* out, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  int grid = (int)std::min<size_t>((m + 255) / 256, (size_t)g->sms * 4);
  ProfScope ps(g, s, PC_QUERY, 1);
  k_query<<<grid, 256, 0, s>>>(pairs, m, out, g->label, g->V, g->gc);
  return cudaGetLastError();
}

// ---- forest ids in ascending order: bitonic sort of 1024-id chunks in
// shared memory, then each id's final rank = its rank in its chunk + its
// lower bound in every other chunk (ids are distinct).
constexpr uint32_t kSortChunk = 1024;

__global__ void __launch_bounds__(512) k_sort_chunks(uint64_t* ids, const uint32_t* gc) {
  __shared__ uint64_t s[kSortChunk];
  if (ld_cg(&gc[GC_FOREST_SORTED])) return;  // done since the last recovery
  const uint32_t n = ld_cg(&gc[GC_NFOREST]);
  const uint32_t base = blockIdx.x * kSortChunk;
  if (base >= n) return;
  for (uint32_t i = threadIdx.x; i < kSortChunk; i += blockDim.x) s[i] = base + i < n ? ids[base + i] : kNone;
  __syncthreads();
  for (uint32_t k = 2; k <= kSortChunk; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < kSortChunk; i += blockDim.x) {
        uint32_t p = i ^ j;
        if (p > i) {
          bool up = (i & k) == 0;
          uint64_t x = s[i], y = s[p];
          if ((x > y) == up) {
            s[i] = y;
            s[p] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < kSortChunk && base + i < n; i += blockDim.x) ids[base + i] = s[i];
}

__global__ void k_merge_rank(const uint64_t* __restrict__ ids, uint64_t* __restrict__ out, const uint32_t* gc) {
  if (ld_cg(&gc[GC_FOREST_SORTED])) return;
  const uint32_t n = ld_cg(&gc[GC_NFOREST]);
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t x = ids[i];
  const uint32_t mine = i / kSortChunk, nch = (n + kSortChunk - 1) / kSortChunk;
  uint32_t rank = i - mine * kSortChunk;
  for (uint32_t c = 0; c < nch; c++) {
    if (c == mine) continue;
    uint32_t lo = c * kSortChunk, hi = min(n, lo + kSortChunk);
    while (lo < hi) {  // first position with ids[pos] >= x
      uint32_t mid = (lo + hi) >> 1;
      if (ids[mid] < x)
        lo = mid + 1;
      else
        hi = mid;
    }
    rank += lo - c * kSortChunk;
  }
  out[rank] = x;
}

__global__ void k_mark_sorted(uint32_t* gc) {
  if (gc[GC_FOREST_SORTED]) return;
  gc[GC_NSORTED] = gc[GC_NFOREST];
  gc[GC_FOREST_SORTED] = 1;
}

cudaError_t launch_forest_sort(cupc_graph* g, cudaStream_t s) {
  uint32_t nch = (g->V + kSortChunk - 1) / kSortChunk;
  ProfScope ps(g, s, PC_SORT, 3);
  k_sort_chunks<<<nch, 512, 0, s>>>(g->forest, g->gc);
  k_merge_rank<<<(g->V + 255) / 256, 256, 0, s>>>(g->forest, g->forest_sorted, g->gc);
  k_mark_sorted<<<1, 1, 0, s>>>(g->gc);
  return cudaGetLastError();
}

}  // namespace cupc
