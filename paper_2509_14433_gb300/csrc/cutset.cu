// Parallel cutset (§3.1, Lemma 3.1): the sketch of every tree of a dynamic
// forest F over the graph's vertex sketches, maintained under link and cut
// by logging the sketch additions a link or cut needs and replaying the log
// with one thread per word of a sketch.
//
// The forest is kept as Euler tours (one node per vertex, two arc nodes per
// forest edge) in randomized search trees ordered by tour position (treaps,
// on the host). Every treap node owns an aggregate sketch slot in device
// memory: the XOR of the vertex sketches in its subtree (arc nodes own a
// zero sketch), so a tree's sketch is the aggregate of its tour's root. A
// link or cut splits and merges tours; every node whose children changed,
// and every ancestor of one, gets its aggregate recomputed as
//     agg[n] = own(n) ^ agg[left(n)] ^ agg[right(n)]
// in post-order (children first). These additions are logged as tasks; one
// launch replays the batch's log: thread t owns word t of every sketch and
// follows the whole log in order for that word, so the words proceed
// independently and the log's order is kept per word (the paper's parallel
// execution of the logged additions). A vertex whose sketch changed (after
// cupc_update_batch) is refreshed the same way: its node and its ancestors.
#include <stdlib.h>
#include <string.h>

#include <new>
#include <random>
#include <unordered_map>
#include <vector>

#include "common.cuh"

using namespace cupc;

namespace {

// Task of the log: agg[dst] = own vertex sketch (own >= 0) ^ agg[l] ^ agg[r]
// (each term absent when negative).
__global__ void k_cutset_replay(const int4* __restrict__ tasks, uint32_t ntasks, uint64_t* agg,
                                const uint64_t* __restrict__ sketch, uint32_t V, uint32_t W, size_t SW) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < SW; t += (size_t)gridDim.x * blockDim.x) {
    // word t of a sketch laid out [layer][bucket][alpha, gamma]
    const size_t r = t / (2 * (size_t)W), j2 = t - r * 2 * W;
    const uint64_t* own_base = sketch + r * V * 2 * W + j2;
    for (uint32_t k = 0; k < ntasks; k++) {
      const int4 tk = tasks[k];
      uint64_t v = tk.y >= 0 ? own_base[(size_t)tk.y * 2 * W] : 0ull;
      if (tk.z >= 0) v ^= agg[(size_t)tk.z * SW + t];
      if (tk.w >= 0) v ^= agg[(size_t)tk.w * SW + t];
      agg[(size_t)tk.x * SW + t] = v;
    }
  }
}

// Query of one layer of a tree sketch (§2.1, Theorem A.2): ZERO when the
// deterministic bucket is zero, else the first good bucket in index order
// (deterministic bucket, then column-major), else FAIL. One thread.
__global__ void k_cutset_sample(const ulonglong2* __restrict__ layer, uint32_t W, uint32_t V, uint64_t kchk,
                                uint64_t* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint64_t res = 2, edge = 0;
  if ((layer[0].x | layer[0].y) == 0) {
    res = 0;
  } else {
    for (uint32_t j = 0; j < W; j++) {
      const ulonglong2 b = layer[j];
      if (b.x != 0 && mix64(b.x ^ kchk) == b.y && b.x / V < b.x % V) {
        res = 1;
        edge = b.x;
        break;
      }
    }
  }
  out[0] = res;
  out[1] = edge;
}

struct Node {
  int left = -1, right = -1, parent = -1;
  uint32_t prio = 0, size = 1;
  int vertex = -1;  // the vertex of a vertex node, -1 for an arc node
  bool dirty = false, closed = false, live = false;
};

}  // namespace

struct cupc_cutset {
  cupc_graph* g;
  uint32_t V, L, W;
  size_t SW;  // u64 words of one sketch: L * W * 2
  uint32_t nslots;
  uint64_t* agg;  // nslots * SW
  int4* dtasks;
  size_t dtask_cap;
  uint64_t* dsample;  // 2 words
  std::vector<Node> nodes;
  std::vector<int> free_arcs;
  std::unordered_map<uint64_t, std::pair<int, int>> arcs;  // edge id -> (arc u->v, arc v->u)
  std::vector<int> dirty;
  std::vector<int4> tasks;
  std::mt19937 rng;
  uint64_t stat_tasks = 0, stat_launches = 0, stat_links = 0, stat_cuts = 0;
};

namespace {

uint32_t sz(const cupc_cutset* c, int n) { return n < 0 ? 0u : c->nodes[n].size; }

void touch(cupc_cutset* c, int n) {
  Node& x = c->nodes[n];
  x.size = 1 + sz(c, x.left) + sz(c, x.right);
  if (x.left >= 0) c->nodes[x.left].parent = n;
  if (x.right >= 0) c->nodes[x.right].parent = n;
  if (!x.dirty) {
    x.dirty = true;
    c->dirty.push_back(n);
  }
}

// (first k nodes of t, the rest); the roots' parents are cleared
void split(cupc_cutset* c, int t, uint32_t k, int* a, int* b) {
  if (t < 0) {
    *a = *b = -1;
    return;
  }
  Node& x = c->nodes[t];
  if (sz(c, x.left) < k) {
    int ra, rb;
    split(c, x.right, k - sz(c, x.left) - 1, &ra, &rb);
    c->nodes[t].right = ra;
    touch(c, t);
    *a = t;
    *b = rb;
  } else {
    int la, lb;
    split(c, x.left, k, &la, &lb);
    c->nodes[t].left = lb;
    touch(c, t);
    *a = la;
    *b = t;
  }
  if (*a >= 0) c->nodes[*a].parent = -1;
  if (*b >= 0) c->nodes[*b].parent = -1;
}

int merge(cupc_cutset* c, int a, int b) {
  if (a < 0) return b;
  if (b < 0) return a;
  if (c->nodes[a].prio > c->nodes[b].prio) {
    c->nodes[a].right = merge(c, c->nodes[a].right, b);
    touch(c, a);
    c->nodes[a].parent = -1;
    return a;
  }
  c->nodes[b].left = merge(c, a, c->nodes[b].left);
  touch(c, b);
  c->nodes[b].parent = -1;
  return b;
}

int root_of(const cupc_cutset* c, int n) {
  while (c->nodes[n].parent >= 0) n = c->nodes[n].parent;
  return n;
}

// tour position of node n (0-based)
uint32_t position(const cupc_cutset* c, int n) {
  uint32_t p = sz(c, c->nodes[n].left);
  while (c->nodes[n].parent >= 0) {
    const int q = c->nodes[n].parent;
    if (c->nodes[q].right == n) p += sz(c, c->nodes[q].left) + 1;
    n = q;
  }
  return p;
}

// the tour of v's tree rotated to start at v's node
int reroot(cupc_cutset* c, int v) {
  const int t = root_of(c, v);
  int a, b;
  split(c, t, position(c, v), &a, &b);
  return merge(c, b, a);
}

int new_arc(cupc_cutset* c) {
  const int n = c->free_arcs.back();
  c->free_arcs.pop_back();
  Node& x = c->nodes[n];
  x = Node();
  x.prio = c->rng();
  x.live = true;
  x.dirty = true;
  c->dirty.push_back(n);
  return n;
}

bool do_link(cupc_cutset* c, uint32_t u, uint32_t v) {
  if (u == v || root_of(c, u) == root_of(c, v) || c->free_arcs.size() < 2) return false;
  const int tu = reroot(c, u), tv = reroot(c, v);
  const int a = new_arc(c), b = new_arc(c);
  c->arcs[(uint64_t)std::min(u, v) * c->V + std::max(u, v)] = u < v ? std::make_pair(a, b) : std::make_pair(b, a);
  merge(c, merge(c, merge(c, tu, a), tv), b);
  c->stat_links++;
  return true;
}

bool do_cut(cupc_cutset* c, uint32_t u, uint32_t v) {
  auto it = c->arcs.find((uint64_t)std::min(u, v) * c->V + std::max(u, v));
  if (u == v || it == c->arcs.end()) return false;
  int x = it->second.first, y = it->second.second;
  c->arcs.erase(it);
  uint32_t px = position(c, x), py = position(c, y);
  if (px > py) {
    std::swap(x, y);
    std::swap(px, py);
  }
  // tour = P [x] Q [y] R  ->  trees Q and P R
  int P, rest, X, rest2, Q, Y, R;
  split(c, root_of(c, x), px, &P, &rest);
  split(c, rest, 1, &X, &rest2);
  split(c, rest2, py - px - 1, &Q, &rest);
  split(c, rest, 1, &Y, &R);
  merge(c, P, R);
  for (int n : {X, Y}) {
    c->nodes[n] = Node();
    c->free_arcs.push_back(n);
  }
  c->stat_cuts++;
  return true;
}

void mark_vertex(cupc_cutset* c, uint32_t w) {
  Node& x = c->nodes[w];
  if (!x.dirty) {
    x.dirty = true;
    c->dirty.push_back((int)w);
  }
}

// Tasks for every dirty node and its ancestors, children before parents;
// then launch the replay of the log.
cudaError_t flush(cupc_cutset* c, cudaStream_t s) {
  std::vector<int> roots;
  for (int n : c->dirty) {  // upward closure
    if (!c->nodes[n].live) continue;
    for (int m = n; m >= 0 && !c->nodes[m].closed; m = c->nodes[m].parent) {
      c->nodes[m].closed = true;
      c->nodes[m].dirty = true;
      if (c->nodes[m].parent < 0) roots.push_back(m);
    }
  }
  c->tasks.clear();
  std::vector<std::pair<int, bool>> st;  // post-order over dirty nodes
  for (int r : roots) {
    st.push_back({r, false});
    while (!st.empty()) {
      auto [n, expanded] = st.back();
      st.pop_back();
      const Node& x = c->nodes[n];
      if (expanded) {
        c->tasks.push_back(make_int4(n, x.vertex, x.left, x.right));
        continue;
      }
      st.push_back({n, true});
      if (x.right >= 0 && c->nodes[x.right].closed) st.push_back({x.right, false});
      if (x.left >= 0 && c->nodes[x.left].closed) st.push_back({x.left, false});
    }
  }
  for (int n : c->dirty) c->nodes[n].dirty = c->nodes[n].closed = false;
  for (const int4& t : c->tasks) c->nodes[t.x].dirty = c->nodes[t.x].closed = false;
  c->dirty.clear();
  const size_t nt = c->tasks.size();
  if (nt == 0) return cudaSuccess;
  if (nt > c->dtask_cap) {
    if (c->dtasks) cudaFree(c->dtasks);
    c->dtasks = nullptr;
    size_t cap = 1024;
    while (cap < nt) cap *= 2;
    cudaError_t e = cudaMalloc((void**)&c->dtasks, cap * sizeof(int4));
    if (e != cudaSuccess) {
      c->dtask_cap = 0;
      return e;
    }
    c->dtask_cap = cap;
  }
  cudaError_t e = cudaMemcpyAsync(c->dtasks, c->tasks.data(), nt * sizeof(int4), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const int threads = 256;
  const int grid = (int)std::min<size_t>((c->SW + threads - 1) / threads, (size_t)c->g->sms * 8);
  k_cutset_replay<<<grid, threads, 0, s>>>(c->dtasks, (uint32_t)nt, c->agg, (const uint64_t*)c->g->sketch, c->V,
                                           c->W, c->SW);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the host log is reused by the next batch only after this copy is done
  e = cudaStreamSynchronize(s);
  c->stat_tasks += nt;
  c->stat_launches++;
  return e;
}

}  // namespace

extern "C" {

cupc_status cupc_cutset_create(cupc_graph* g, cupc_stream stream, cupc_cutset** out) {
  if (!g || !out) return CUPC_EINVAL;
  *out = nullptr;
  cupc_cutset* c = new (std::nothrow) cupc_cutset();
  if (!c) return CUPC_ENOMEM;
  c->g = g;
  c->V = g->V;
  c->L = g->L;
  c->W = g->W;
  c->SW = (size_t)g->L * g->W * 2;
  c->nslots = 3 * g->V;
  c->rng.seed(0x5EEDu ^ g->V);
  if (cudaMalloc((void**)&c->agg, (size_t)c->nslots * c->SW * sizeof(uint64_t)) != cudaSuccess ||
      cudaMalloc((void**)&c->dsample, 2 * sizeof(uint64_t)) != cudaSuccess) {
    cudaGetLastError();
    cupc_cutset_destroy(c);
    return CUPC_ENOMEM;
  }
  c->nodes.resize(c->nslots);
  for (uint32_t w = 0; w < c->V; w++) {
    Node& x = c->nodes[w];
    x.prio = c->rng();
    x.vertex = (int)w;
    x.live = true;
    x.dirty = true;
    c->dirty.push_back((int)w);
  }
  for (uint32_t n = c->nslots; n-- > c->V;) c->free_arcs.push_back((int)n);
  if (flush(c, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    cupc_cutset_destroy(c);
    return CUPC_ECUDA;
  }
  *out = c;
  return CUPC_OK;
}

cupc_status cupc_cutset_apply(cupc_cutset* c, const uint32_t* ops, size_t n, size_t* applied, cupc_stream stream) {
  if (!c || (n && !ops)) return CUPC_EINVAL;
  size_t i = 0;
  bool ok = true;
  for (; i < n && ok; i++) {
    const uint32_t kind = ops[3 * i], u = ops[3 * i + 1], v = ops[3 * i + 2];
    if (u >= c->V || (kind != CUPC_CUTSET_REFRESH && v >= c->V)) {
      ok = false;
    } else if (kind == CUPC_CUTSET_LINK) {
      ok = do_link(c, u, v);
    } else if (kind == CUPC_CUTSET_CUT) {
      ok = do_cut(c, u, v);
    } else if (kind == CUPC_CUTSET_REFRESH) {
      mark_vertex(c, u);
    } else {
      ok = false;
    }
    if (!ok) break;
  }
  if (applied) *applied = i;
  if (flush(c, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return CUPC_ECUDA;
  }
  return ok ? CUPC_OK : CUPC_EINVAL;
}

cupc_status cupc_cutset_connected(const cupc_cutset* c, uint32_t u, uint32_t v, int* out) {
  if (!c || !out || u >= c->V || v >= c->V) return CUPC_EINVAL;
  *out = root_of(c, (int)u) == root_of(c, (int)v);
  return CUPC_OK;
}

cupc_status cupc_cutset_tree_sketch(const cupc_cutset* c, uint32_t w, void* dst, cupc_stream stream) {
  if (!c || !dst || w >= c->V) return CUPC_EINVAL;
  const int r = root_of(c, (int)w);
  if (cudaMemcpyAsync(dst, c->agg + (size_t)r * c->SW, c->SW * sizeof(uint64_t), cudaMemcpyDefault,
                      (cudaStream_t)stream) != cudaSuccess ||
      cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return CUPC_ECUDA;
  }
  return CUPC_OK;
}

cupc_status cupc_cutset_query(const cupc_cutset* c, uint32_t w, uint32_t r, uint32_t* result, uint64_t* edge,
                              cupc_stream stream) {
  if (!c || !result || !edge || w >= c->V || r >= c->L) return CUPC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int root = root_of(c, (int)w);
  const ulonglong2* layer = reinterpret_cast<const ulonglong2*>(c->agg + (size_t)root * c->SW) + (size_t)r * c->W;
  uint64_t kchk = 0, host[2];
  // the layer's checksum key, from the graph's key table
  if (cudaMemcpyAsync(&kchk, c->g->keys + (size_t)r * (c->g->C + 1) + c->g->C, sizeof(uint64_t),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CUPC_ECUDA;
  }
  k_cutset_sample<<<1, 32, 0, s>>>(layer, c->W, c->V, kchk, c->dsample);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(host, c->dsample, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CUPC_ECUDA;
  }
  *result = (uint32_t)host[0];
  *edge = host[1];
  return CUPC_OK;
}

cupc_status cupc_cutset_stats(const cupc_cutset* c, uint64_t* out4) {
  if (!c || !out4) return CUPC_EINVAL;
  out4[0] = c->stat_tasks;
  out4[1] = c->stat_launches;
  out4[2] = c->stat_links;
  out4[3] = c->stat_cuts;
  return CUPC_OK;
}

void cupc_cutset_destroy(cupc_cutset* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  if (c->agg) cudaFree(c->agg);
  if (c->dtasks) cudaFree(c->dtasks);
  if (c->dsample) cudaFree(c->dsample);
  delete c;
}

}  // extern "C"
