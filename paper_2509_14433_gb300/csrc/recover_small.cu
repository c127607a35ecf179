// Spanning-forest recovery of small graphs (V <= kClMaxV) in one
// thread-block cluster: the same Boruvka rounds and the same results as the
// grid-wide k_recover (App. A.1.1, "The AGM Algorithm"), with the
// per-vertex state in the shared memory of the cluster's first CTA (the
// leader) and hardware cluster barriers (about 0.2 us) in place of grid
// barriers (1.2-1.6 us on GB300). Round r:
//   leader    groups the members of the live components by label (a
//             counting sort in shared memory) and publishes the groups
//             (perm: label << 16 | vertex, roff: segment start | end << 16)
//   all CTAs  reduce layer r over the groups: warp g takes members
//             [g q, (g+1) q); a component inside one range is sampled by its
//             warp, one over several ranges is XORed into acc[K] and sampled
//             by the last range to finish; every sample goes to cand[K]
//   leader    books the samples (ZERO: the component is final; GOOD with an
//             edge leaving it: its candidate; GOOD inside it: a checksum
//             false positive; FAIL), then hooks and relabels
// Hook. Each live component K with a candidate edge e(K) points at the
// component t(K) on the edge's other side, so the candidate graph is
// functional: every weak component is a tree (some node has no candidate,
// or two nodes picked the same edge) or holds exactly one cycle. Kruskal
// over the candidates in ascending id order keeps every candidate edge but
// the largest edge of each cycle (the cycle property of minimum spanning
// forests with distinct weights), i.e. the same forest edges the grid-wide
// hook adds. The leader finds each cycle's largest edge by pointer doubling
// (the maximum over the jumped path rides with the pointer), drops it,
// finds the roots by pointer jumping and gives every component of a tree
// the smallest vertex id in the tree.
// Control flow is uniform over the cluster: the leader decides whether a
// round runs and publishes that in gc[GC_ACTIVE] before a cluster barrier;
// every CTA reads it after the barrier, so all CTAs pass the same barriers.
// The barrier's arrive has release and its wait acquire semantics at
// cluster scope, which order the global writes of one CTA before the reads
// of another; data written by another CTA is read through L2 (ld.cg).
#include "recover_dev.cuh"

namespace cupc {

namespace {

// Members of a warp's range whose rows are prefetched ahead of the fold.
constexpr uint32_t kClAhead = 4;

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Rows of two members at once, all loads issued before the first XOR.
template <uint32_t NQ>
__device__ __forceinline__ void warp_xor_rows2(ulonglong2 (&acc)[NQ], const ulonglong2* __restrict__ r0,
                                               const ulonglong2* __restrict__ r1, uint32_t W, uint32_t lane) {
  ulonglong2 x[NQ], y[NQ];
#pragma unroll
  for (uint32_t q = 0; q < NQ; q++) {
    const uint32_t b = lane + 32 * q;
    x[q] = make_ulonglong2(0, 0);
    y[q] = make_ulonglong2(0, 0);
    if (b < W) {
      x[q] = __ldg(r0 + b);
      y[q] = __ldg(r1 + b);
    }
  }
#pragma unroll
  for (uint32_t q = 0; q < NQ; q++) {
    acc[q].x ^= x[q].x ^ y[q].x;
    acc[q].y ^= x[q].y ^ y[q].y;
  }
}

// The leader's shared memory, V entries each: x (grouping: count and cursor
// of a label; hook: max edge << 32 | pointer), lab (vertex -> label), e
// (candidate edge of a label, kNoneU32: none), f (pointer of a label in the
// hook forest), minv (smallest label of a tree), fin (the label's component
// sampled ZERO), flag (hook and relabel marks).
struct ClSmem {
  uint64_t* x;
  uint32_t *lab, *e, *f, *minv;
  uint8_t *fin, *flag;
};

__device__ __forceinline__ ClSmem cl_smem(unsigned char* base, uint32_t V) {
  ClSmem m;
  m.x = reinterpret_cast<uint64_t*>(base);
  m.lab = reinterpret_cast<uint32_t*>(m.x + V);
  m.e = m.lab + V;
  m.f = m.e + V;
  m.minv = m.f + V;
  m.fin = reinterpret_cast<uint8_t*>(m.minv + V);
  m.flag = m.fin + V;
  return m;
}

// Root in a shared-memory union-find with path halving; concurrent halving
// only ever points a node at an ancestor.
__device__ __forceinline__ uint32_t cl_find(volatile uint32_t* par, uint32_t x, uint32_t V) {
  for (uint32_t k = 0; k < V; k++) {
    const uint32_t y = par[x];
    if (y == x) break;
    const uint32_t z = par[y];
    if (z != y) par[x] = z;
    x = y;
  }
  return x;
}

// Block-wide sum of a per-thread value (every thread gets it). s_red: 32
// words per summed value.
__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* s_red) {
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = __reduce_add_sync(0xffffffffu, v);
  __syncthreads();
  if (lane == 0) s_red[wid] = v;
  __syncthreads();
  uint32_t t = lane < nw ? s_red[lane] : 0;
  return __reduce_add_sync(0xffffffffu, t);
}

// Four block-wide sums behind one pair of barriers.
__device__ __forceinline__ uint4 block_sum4(uint4 v, uint32_t* s_red) {
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v.x = __reduce_add_sync(0xffffffffu, v.x);
  v.y = __reduce_add_sync(0xffffffffu, v.y);
  v.z = __reduce_add_sync(0xffffffffu, v.z);
  v.w = __reduce_add_sync(0xffffffffu, v.w);
  __syncthreads();
  if (lane == 0) {
    s_red[wid] = v.x;
    s_red[32 + wid] = v.y;
    s_red[64 + wid] = v.z;
    s_red[96 + wid] = v.w;
  }
  __syncthreads();
  uint4 t = make_uint4(0, 0, 0, 0);
  if (lane < nw) t = make_uint4(s_red[lane], s_red[32 + lane], s_red[64 + lane], s_red[96 + lane]);
  return make_uint4(__reduce_add_sync(0xffffffffu, t.x), __reduce_add_sync(0xffffffffu, t.y),
                    __reduce_add_sync(0xffffffffu, t.z), __reduce_add_sync(0xffffffffu, t.w));
}

// Leader: group the members of the live components (label not final) by
// label. perm[pos] = label << 16 | vertex, roff[K] = start | end << 16.
// Returns the member count. Labels split into contiguous chunks, one per
// thread, for the scan.
__device__ uint32_t cl_group(const RecArgs& a, const ClSmem& m, uint32_t V, uint32_t* s_red) {
  const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  uint32_t* cnt = reinterpret_cast<uint32_t*>(m.x);  // cnt[2K]: count, then start; cnt[2K+1]: cursor
  for (uint32_t K = tid; K < V; K += nt) m.x[K] = 0;
  __syncthreads();
  for (uint32_t w = tid; w < V; w += nt) {
    const uint32_t K = m.lab[w];
    if (!m.fin[K]) atomicAdd(&cnt[2 * K], 1u);
  }
  __syncthreads();
  const uint32_t per = (V + nt - 1) / nt, k0 = min(V, tid * per), k1 = min(V, k0 + per);
  uint32_t sum = 0;
  for (uint32_t K = k0; K < k1; K++) sum += cnt[2 * K];
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= (uint32_t)o) inc += y;
  }
  if (lane == 31) s_red[wid] = inc;
  __syncthreads();
  uint32_t wbase = 0, total = 0;
  for (uint32_t k = 0; k < nw; k++) {
    const uint32_t t = s_red[k];
    if (k < wid) wbase += t;
    total += t;
  }
  uint32_t at = wbase + inc - sum;
  for (uint32_t K = k0; K < k1; K++) {
    const uint32_t c = cnt[2 * K];
    if (c) a.roff[K] = at | ((at + c) << 16);
    cnt[2 * K] = at;
    at += c;
  }
  __syncthreads();
  for (uint32_t w = tid; w < V; w += nt) {
    const uint32_t K = m.lab[w];
    if (!m.fin[K]) a.perm[cnt[2 * K] + atomicAdd(&cnt[2 * K + 1], 1u)] = K << 16 | w;
  }
  return total;
}

// Leader: hook the candidate graph (m.e, m.f of every label; f = K where K
// has no candidate) and relabel. Appends the forest edges at *nforest.
// J: pointer-doubling steps, 2^J >= the number of candidates.
__device__ void cl_hook(const RecArgs& a, const ClSmem& m, uint32_t V, uint32_t J, uint32_t* nforest) {
  const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  // two components that picked the same edge: the larger stops pointing
  for (uint32_t K = tid; K < V; K += nt) {
    const uint32_t eK = m.e[K];
    if (eK == kNoneU32) continue;
    const uint32_t y = m.f[K];
    if (K > y && m.f[y] == K && m.e[y] == eK) m.flag[K] = 1;
  }
  __syncthreads();
  for (uint32_t K = tid; K < V; K += nt) {
    if (m.flag[K]) {  // the edge stays with the smaller one
      m.f[K] = K;
      m.e[K] = kNoneU32;
      m.flag[K] = 0;
    }
    m.x[K] = m.f[K] != K ? ((uint64_t)m.e[K] << 32 | m.f[K]) : (uint64_t)K;
  }
  __syncthreads();
  // pointer doubling in place: x[K] = (largest edge on the path jumped, end).
  // A 64-bit shared word is read and written whole, and a path only grows,
  // so after step j every path is at least 2^(j+1) long or ends at a root.
  for (uint32_t j = 0; j < J; j++) {
    for (uint32_t K = tid; K < V; K += nt) {
      if (m.f[K] == K) continue;
      const uint64_t p = m.x[K], q = m.x[(uint32_t)p];
      m.x[K] = (max(p >> 32, q >> 32) << 32) | (uint32_t)q;
    }
    __syncthreads();
  }
  // a path of 2^J >= (tail + cycle) steps ends on its cycle (or at its
  // root); from a cycle node it has covered the whole cycle, so the end's
  // maximum is the cycle's largest edge: its owner stops pointing
  for (uint32_t K = tid; K < V; K += nt) {
    if (m.f[K] == K) continue;
    const uint32_t y = (uint32_t)m.x[K];
    if (m.f[y] == y) continue;
    const uint32_t M = (uint32_t)(m.x[y] >> 32);
    const uint32_t K1 = m.lab[M / V], K2 = m.lab[M % V];
    m.flag[m.e[K1] == M ? K1 : K2] = 1;
  }
  __syncthreads();
  // the edges still pointing are the forest edges
  for (uint32_t base = tid & ~31u; base < V; base += nt) {
    const uint32_t K = base + lane;
    bool keep = false;
    if (K < V) {
      if (m.flag[K]) {
        m.f[K] = K;
        m.flag[K] = 0;
      } else {
        keep = m.f[K] != K;
      }
      m.minv[K] = kNoneU32;
    }
    const uint32_t mk = __ballot_sync(0xffffffffu, keep);
    uint32_t at = 0;
    if (lane == 0 && mk) at = atomicAdd(nforest, (uint32_t)__popc(mk));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (keep) a.forest[at + __popc(mk & ((1u << lane) - 1))] = m.e[K];
  }
  __syncthreads();
  // roots by pointer jumping
  for (uint32_t it = 0; it < 32; it++) {
    int moved = 0;
    for (uint32_t K = tid; K < V; K += nt) {
      const uint32_t y = m.f[K], z = m.f[y];
      if (z != y) {
        m.f[K] = z;
        moved = 1;
      }
    }
    if (!__syncthreads_or(moved)) break;
  }
  // every label takes the smallest label of its tree (labels are smallest
  // vertex ids); a tree of several labels is merged: its new label is live
  for (uint32_t K = tid; K < V; K += nt) {
    if (m.lab[K] != K) continue;
    const uint32_t root = m.f[K];
    atomicMin(&m.minv[root], K);
    if (root != K) m.flag[root] = 1;
  }
  __syncthreads();
  for (uint32_t w = tid; w < V; w += nt) {
    m.lab[w] = m.minv[m.f[m.lab[w]]];
    if (m.flag[w]) {  // w is a merged tree's root
      m.fin[m.minv[w]] = 0;
      m.flag[w] = 0;
    }
  }
  __syncthreads();
}

}  // namespace

// NQ: buckets per lane (W <= 32 NQ).
template <uint32_t NQ>
__global__ void __launch_bounds__(kClThreads, 1) k_recover_cl(RecArgs a) {
  extern __shared__ __align__(16) unsigned char cl_dyn[];
  __shared__ uint32_t s_red[128];
  __shared__ uint32_t c_nforest, c_loglen, c_nfail, c_nfp, c_rounds, c_complete, c_nlive, c_done;
  __shared__ uint32_t c_ncand;
  const uint32_t V = a.V, W = a.W, tid = threadIdx.x, lane = tid & 31, nt = blockDim.x;
  const bool leader = blockIdx.x == 0;
  const uint32_t nwarps = gridDim.x * (nt >> 5), gwarp = blockIdx.x * (nt >> 5) + (tid >> 5);
  const uint32_t ctid = blockIdx.x * nt + tid, cstride = gridDim.x * nt;
  uint32_t* gc = a.gc;
  const ClSmem m = cl_smem(cl_dyn, V);

  // nobody writes these flags before the first cluster barrier, so every CTA
  // takes the same early return and the same warm/cold start
  const bool valid = ld_cg(&gc[GC_LABELS_VALID]) != 0, warm = !a.force && valid && ld_cg(&gc[GC_WARM]) != 0;
  if (!a.force && valid && !warm) return;
  const uint32_t nsorted = warm ? min(ld_cg(&gc[GC_NSORTED]), V) : 0;
  const uint32_t nadd = warm ? min(ld_cg(&gc[GC_NFADD]), V) : 0;
  const bool dirty = ld_cg(&gc[GC_REC_DIRTY]) != 0;
  for (uint32_t w = ctid; w < V; w += cstride) {
    a.ipar[w] = w;
    if (dirty) a.pcount[w] = 0;
    if (!warm) a.fdead[w] = 0;  // a warm start reads them first
  }
  if (dirty)
    for (size_t i = ctid; i < (size_t)V * W; i += cstride) a.acc[i] = make_ulonglong2(0, 0);
  if (a.inc)
    for (size_t i = ctid; i < ((size_t)1 << a.ftab_bits); i += cstride) a.ftab[i] = 0ull;
  for (uint32_t r = ctid; r < a.L; r += cstride) {
    a.log_live[r] = 0;
    a.log_ncand[r] = 0;
  }
  if (leader) {
    for (uint32_t w = tid; w < V; w += nt) {
      m.lab[w] = w;
      m.fin[w] = 0;
      m.flag[w] = 0;
      m.f[w] = w;
    }
    if (tid == 0) {
      c_nforest = 0;
      c_loglen = 0;
      c_nfail = 0;
      c_nfp = 0;
      c_rounds = 0;
      c_complete = 0;
      c_nlive = V;
      c_done = 0;
    }
  }
  cluster_sync_all();
  if (leader) {
    if (tid == 0) {
      gc[GC_REC_DIRTY] = 0;
      gc[GC_NFADD] = 0;
      gc[GC_LABELS_VALID] = 0;
      gc[GC_FOREST_SORTED] = 0;
      gc[GC_WARM] = 0;
      gc[GC_COMPLETE] = 0;
      gc[GC_RECOVERIES] += 1;
    }
    if (warm) {
      // fragments: union the endpoints of the forest edges still present
      // (the larger root under the smaller); an edge whose union joins two
      // fragments starts the new forest
      const uint32_t nall = nsorted + nadd;
      for (uint32_t i = tid; i < nall; i += nt) {
        bool keep;
        uint64_t e;
        if (i < nsorted) {
          keep = !a.fdead[i];
          e = a.forest_sorted[i];
        } else {
          keep = !a.fadd_dead[i - nsorted];
          e = a.fadd[i - nsorted];
        }
        if (keep) {
          uint32_t x = (uint32_t)(e / V), y = (uint32_t)(e % V);
          keep = false;
          for (uint32_t k = 0; k < V && x < V && y < V; k++) {  // bounded: each failed CAS is another thread's progress
            x = cl_find(m.f, x, V);
            y = cl_find(m.f, y, V);
            if (x == y) break;
            if (x > y) {
              const uint32_t t = x;
              x = y;
              y = t;
            }
            if (atomicCAS(&m.f[y], y, x) == y) {
              keep = true;
              break;
            }
          }
        }
        if (keep) a.forest[atomicAdd(&c_nforest, 1u)] = e;
      }
      __syncthreads();
      for (uint32_t w = tid; w < V; w += nt) m.lab[w] = cl_find(m.f, w, V);  // the smallest id of the fragment
      __syncthreads();
      // A fragment that holds no endpoint of a deleted forest edge is a whole
      // component of the last complete recovery, joined with others only by
      // recorded merges: its cut is empty, so it starts final (its sample
      // would be ZERO). Only the split components are sampled again.
      for (uint32_t w = tid; w < V; w += nt) m.fin[w] = m.lab[w] == w;
      __syncthreads();
      for (uint32_t i = tid; i < nall; i += nt) {
        const bool dead = i < nsorted ? a.fdead[i] != 0 : a.fadd_dead[i - nsorted] != 0;
        if (!dead) continue;
        const uint64_t e = i < nsorted ? a.forest_sorted[i] : a.fadd[i - nsorted];
        const uint32_t x = (uint32_t)(e / V), y = (uint32_t)(e % V);
        if (x < V && y < V) {
          m.fin[m.lab[x]] = 0;
          m.fin[m.lab[y]] = 0;
        }
      }
      __syncthreads();
      uint32_t nl = 0;
      for (uint32_t w = tid; w < V; w += nt) {
        a.fdead[w] = 0;
        nl += m.lab[w] == w && !m.fin[w];
      }
      nl = block_sum(nl, s_red);
      if (tid == 0) c_nlive = nl;
      __syncthreads();
    }
  }

  for (uint32_t r = 0;; r++) {
    const bool multi = r > 0 || warm;  // components may have several members
    if (leader) {
      // One live component left: every other component is final and its
      // merged sketch is zero, and the XOR of all vertex sketches of a layer
      // is zero, so the live one samples ZERO: log the round, stop. Imported
      // words need not come from a stream: then the round is run.
      bool stop = c_done || r >= a.L;
      if (!stop && multi && a.sum_zero && c_nlive == 1) {
        if (tid == 0) {
          a.log_live[r] = 1;
          c_rounds = r + 1;
          c_complete = 1;
        }
        stop = true;
      }
      uint32_t n = 0;
      if (!stop) n = multi ? cl_group(a, m, V, s_red) : V;
      if (tid == 0) {
        gc[GC_NMEMBERS] = n;
        gc[GC_ACTIVE] = stop ? 0u : (multi ? 2u : 1u);
      }
    }
    cluster_sync_all();  // release/acquire at cluster scope: the groups and gc words are visible
    const uint32_t ctl = ld_cg(&gc[GC_ACTIVE]);
    if (ctl == 0) break;
    const uint32_t n = ld_cg(&gc[GC_NMEMBERS]);
    const bool grouped = ctl == 2;
    // ---- reduce + sample: warp g takes members [g q, (g+1) q), q <= 32
    {
      const uint64_t kchk = a.keys[r * (a.C + 1) + a.C];
      const uint32_t q = (n + nwarps - 1) / nwarps;
      const uint32_t p0 = gwarp * q, p1 = min(n, p0 + q);
      if (p0 < p1) {
        const uint32_t cnt = p1 - p0;
        uint32_t pk = kNoneU32;
        if (lane < cnt) pk = grouped ? ld_cg(&a.perm[p0 + lane]) : ((p0 + lane) << 16 | (p0 + lane));
        const ulonglong2* layer = a.sketch + (size_t)r * V * W;
        // rows of the next kClAhead members head for L1 while earlier ones fold
        uint32_t pf = 0;
        auto prefetch_to = [&](uint32_t until) {
          for (; pf < until; pf++) {
            const ulonglong2* row = layer + (size_t)(__shfl_sync(0xffffffffu, pk, pf) & 0xFFFFu) * W;
#pragma unroll
            for (uint32_t b = 0; b < NQ; b++)
              if (lane + 32 * b < W) asm volatile("prefetch.global.L1 [%0];" ::"l"(row + lane + 32 * b));
          }
        };
        uint32_t i = 0;
        while (i < cnt) {
          const uint32_t K = __shfl_sync(0xffffffffu, pk, i) >> 16;
          const uint32_t run = ~(__ballot_sync(0xffffffffu, (pk >> 16) == K) >> i);  // members i.. of K
          const uint32_t j = min(cnt, run ? i + (uint32_t)__ffs(run) - 1 : 32u);
          const uint32_t seg = grouped ? ld_cg(&a.roff[K]) : 0u;
          ulonglong2 acc[NQ];
#pragma unroll
          for (uint32_t b = 0; b < NQ; b++) acc[b] = make_ulonglong2(0, 0);
          uint32_t mm = i;
          for (; mm + 2 <= j; mm += 2) {
            prefetch_to(min(cnt, mm + 2 + kClAhead));
            const uint32_t w0 = __shfl_sync(0xffffffffu, pk, mm) & 0xFFFFu;
            const uint32_t w1 = __shfl_sync(0xffffffffu, pk, mm + 1) & 0xFFFFu;
            warp_xor_rows2(acc, layer + (size_t)w0 * W, layer + (size_t)w1 * W, W, lane);
          }
          if (mm < j) {
            prefetch_to(min(cnt, mm + 1 + kClAhead));
            const uint32_t w0 = __shfl_sync(0xffffffffu, pk, mm) & 0xFFFFu;
            warp_xor_row(acc, layer + (size_t)w0 * W, W, lane);
          }
          uint32_t s0 = p0 + i, s1 = s0 + 1;
          if (grouped) {
            s0 = seg & 0xFFFFu;
            s1 = seg >> 16;
          }
          const uint32_t npieces = (s1 - 1) / q - s0 / q + 1;
          bool mine = true;
          if (npieces > 1) {
            ulonglong2* dst = a.acc + (size_t)K * W;
#pragma unroll
            for (uint32_t b = 0; b < NQ; b++) {
              const uint32_t bb = lane + 32 * b;
              if (bb < W && (acc[b].x | acc[b].y)) {
                atomicXor((unsigned long long*)&dst[bb].x, (unsigned long long)acc[b].x);
                atomicXor((unsigned long long*)&dst[bb].y, (unsigned long long)acc[b].y);
              }
            }
            __threadfence();
            uint32_t prev = 0;
            if (lane == 0) prev = atomicAdd(&a.pcount[K], 1u);
            mine = __shfl_sync(0xffffffffu, prev, 0) + 1 == npieces;
            if (mine) {  // the last range: every other range's XOR is in acc[K]
              __threadfence();
#pragma unroll
              for (uint32_t b = 0; b < NQ; b++) {
                const uint32_t bb = lane + 32 * b;
                acc[b] = make_ulonglong2(0, 0);
                if (bb < W) {
                  acc[b] = __ldcg(dst + bb);
                  dst[bb] = make_ulonglong2(0, 0);
                }
              }
              if (lane == 0) a.pcount[K] = 0;
            }
          }
          if (mine) {
            uint64_t e = 0;
            const uint32_t res = warp_sample(acc, W, V, kchk, e);
            if (lane == 0) a.cand[K] = make_ulonglong2(e, res);
          }
          i = j;
        }
      }
    }
    cluster_sync_all();  // the samples in cand are visible to the leader
    if (!leader) continue;
    // ---- book the samples of the live components
    for (uint32_t K = tid; K < V; K += nt) {
      m.e[K] = kNoneU32;
      m.f[K] = K;
    }
    if (tid == 0) c_ncand = 0;
    __syncthreads();
    uint32_t live = 0, nz = 0, fail = 0, fp = 0;
    for (uint32_t K = tid; K < V; K += nt) {
      if (m.lab[K] != K || m.fin[K]) continue;  // not a label, or final
      live++;
      const ulonglong2 c = __ldcg(&a.cand[K]);
      if (c.y == 0) {
        m.fin[K] = 1;
        continue;
      }
      nz++;
      if (c.y == 2 || c.x >= (uint64_t)V * V) {  // a GOOD sample is an edge id below V^2
        fail++;
        continue;
      }
      const uint32_t x = (uint32_t)c.x, u = x / V, lu = m.lab[u], lv = m.lab[x - u * V];
      if ((lu == K) != (lv == K)) {
        m.e[K] = (uint32_t)c.x;  // < V^2 <= 2^26
        m.f[K] = lu == K ? lv : lu;
        a.log_ids[c_loglen + atomicAdd(&c_ncand, 1u)] = c.x;
      } else {
        fp++;
      }
    }
    const uint4 sums = block_sum4(make_uint4(live, nz, fail, fp), s_red);
    live = sums.x;
    nz = sums.y;
    fail = sums.z;
    fp = sums.w;
    const uint32_t ncand = c_ncand;  // final: block_sum4 synchronised after the last atomicAdd
    if (tid == 0) {
      a.log_live[r] = live;
      a.log_ncand[r] = ncand;
      c_loglen += ncand;
      c_nfail += fail;
      c_nfp += fp;
      c_rounds = r + 1;
      if (nz == 0) {
        c_complete = 1;
        c_done = 1;
      }
    }
    if (nz != 0) {
      uint32_t J = 0;
      while ((1u << J) < ncand) J++;
      cl_hook(a, m, V, J, &c_nforest);
      uint32_t nl = 0;
      for (uint32_t w = tid; w < V; w += nt) nl += m.lab[w] == w && !m.fin[w];
      nl = block_sum(nl, s_red);
      if (tid == 0) c_nlive = nl;
    }
    __syncthreads();
  }
  if (leader) {
    for (uint32_t w = tid; w < V; w += nt) a.label[w] = m.lab[w];
    if (tid == 0) {
      gc[GC_NFOREST] = c_nforest;
      gc[GC_LOGLEN] = c_loglen;
      gc[GC_NFAIL] = c_nfail;
      gc[GC_NFP] = c_nfp;
      gc[GC_ROUNDS] = c_rounds;
      gc[GC_COMPLETE] = c_complete;
      // a complete recovery starts an incremental epoch
      if (a.inc) gc[GC_LABELS_VALID] = c_complete;
    }
  }
}

static size_t cl_smem_bytes(uint32_t V) { return (size_t)V * (8 + 4 * 4 + 2); }

// Buckets per lane of the instantiation that serves W buckets.
static uint32_t cl_nq(uint32_t W) { return W <= 128 ? 4 : W <= 160 ? 5 : W <= 192 ? 6 : 8; }

static const void* cl_kernel(uint32_t nq) {
  switch (nq) {
    case 4: return (const void*)k_recover_cl<4>;
    case 5: return (const void*)k_recover_cl<5>;
    case 6: return (const void*)k_recover_cl<6>;
    default: return (const void*)k_recover_cl<8>;
  }
}

cudaError_t setup_recover_cluster(cupc_graph* g) {
  g->rec_cluster = 0;
  if (g->V > kClMaxV || g->W > 32 * kWarpBuckets) return cudaSuccess;
  const void* fn = cl_kernel(cl_nq(g->W));
  const size_t smem = cl_smem_bytes(kClMaxV);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cudaSuccess;  // the grid-wide kernel serves
  }
  // the largest cluster that runs, as long as every warp's member range
  // stays within 32 (V <= 32 * warps)
  for (int c = 16; c >= 4; c /= 2) {
    if ((size_t)g->V > (size_t)32 * c * (kClThreads / 32)) break;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = cl_smem_bytes(g->V);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg) == cudaSuccess && ncl >= 1) {
      g->rec_cluster = c;
      break;
    }
    cudaGetLastError();
  }
  return cudaSuccess;
}

cudaError_t launch_recover_cluster(cupc_graph* g, const RecArgs& a, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = g->rec_cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(g->rec_cluster);
  cfg.blockDim = dim3(kClThreads);
  cfg.dynamicSmemBytes = cl_smem_bytes(g->V);
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  RecArgs args = a;
  void* params[] = {&args};
  return cudaLaunchKernelExC(&cfg, cl_kernel(cl_nq(g->W)), params);
}

}  // namespace cupc
