/*
 * CPU oracle for sketch-based connectivity, arXiv 2509.14433.
 * TEST INFRASTRUCTURE ONLY: see cupc_oracle.h for who may use it, the
 * readings it takes where the paper is silent, and what pins each part.
 *
 * Plain and slow on purpose: one update at a time, one vertex at a time,
 * no blocking, no fusion, no threads.
 */
#include "cupc_oracle.h"

#include <stdlib.h>
#include <string.h>

typedef struct {
  uint64_t alpha; /* XOR of the indices that landed in the bucket */
  uint64_t gamma; /* XOR of their checksums */
} orc_bucket;

struct orc_graph {
  uint32_t V, L, C, D, W;
  uint64_t seed;
  uint32_t ell;        /* output bits of one multiply-add-shift stage */
  uint64_t* keys;      /* key_count(L, C) words of the SplitMix64 stream */
  orc_bucket* sketch;  /* vertex-major: [w][r][j], j = 0 det, 1 + c*D + d */
  uint32_t* label;     /* component label = min vertex id */
  uint64_t* forest;
  size_t n_forest;
  int dirty;
  int sticky;
  int status;
  uint64_t rounds_run, n_fail, n_false_pos;
  int complete;
  uint32_t* log_live;  /* [L] */
  uint32_t* log_ncand; /* [L] */
  uint64_t* log_ids;
  size_t log_len;
};

/* ---- SplitMix64 finalizer (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014). */
uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

void orc_keys(uint64_t seed, uint64_t* out, size_t n) {
  const uint64_t phi = 0x9E3779B97F4A7C15ULL;
  for (size_t j = 0; j < n; j++) out[j] = orc_mix64(seed + phi * (uint64_t)(j + 1));
}

static uint32_t ceil_log2(uint32_t V) {
  uint32_t lg = 0;
  while (((uint64_t)1 << lg) < (uint64_t)V) lg++;
  return lg < 1 ? 1 : lg;
}

/* App. A.1.1: O(log V) sketches per vertex, each an l0 sampler with
 * O(log n) rows (n = V^2 indices) and O(log 1/delta) columns. */
void orc_params(uint32_t V, uint32_t* L, uint32_t* C, uint32_t* D) {
  uint32_t lg = ceil_log2(V);
  if (*L == 0) *L = lg + 2;
  if (*C == 0) *C = 7;
  if (*D == 0) *D = 2 * lg;
}

/* Number of key words of a graph: the SplitMix64 stream K(0..) laid out as
 *   K(r*(C+1) + c), c < C ... multiplier a of column c of layer r
 *   K(r*(C+1) + C) .......... checksum key of layer r
 *   K(L*(C+1) + 3*(r*C + c) + k), k = 0, 1, 2 ... b, a', b' of column c */
static size_t key_count(uint32_t L, uint32_t C) { return (size_t)L * (C + 1) + (size_t)3 * L * C; }

/* Output bits of one multiply-add-shift stage for indices below 2^w,
 * w = 2*ceil(log2 V): Dietzfelbinger's bound w + ell - 1 <= 64. */
uint32_t orc_hash_bits(uint32_t V) { return 65 - 2 * ceil_log2(V); }

/* Leading zero bits of an ell-bit value h (ell when h = 0). */
static uint32_t lead_zeros(uint64_t h, uint32_t ell) {
  uint32_t z = 0;
  for (int bit = (int)ell - 1; bit >= 0 && ((h >> bit) & 1) == 0; bit--) z++;
  return z;
}

/* Depth of index x in one column (Theorem A.1 asks only for 2-wise
 * independent hash functions; Theorem A.2's column takes the bucket at the
 * index's depth). The column hash is multiply-add-shift (Dietzfelbinger,
 * "Universal hashing and k-wise independent random variables via integer
 * arithmetic without primes", STACS 1996):
 *   h(x) = ((a*x + b) mod 2^64) div 2^(64-ell)
 * with a, b uniform 64-bit words, which is strongly universal (2-wise
 * independent and uniform) onto ell-bit values when x < 2^(65-ell). Two
 * independent stages (a, b) and (a', b') give the 2*ell-bit string
 * h(x) h'(x), and the depth is its number of leading zero bits, capped at
 * the last row: P(depth >= j) = 2^-j for j <= 2*ell, and the depths of
 * two different indices are independent. The second stage matters only
 * when the first is zero, i.e. when ell < D-1 (V > 2^16 at default
 * parameters). */
uint32_t orc_mas_depth(uint64_t a, uint64_t b, uint64_t a2, uint64_t b2, uint32_t ell, uint32_t D, uint64_t x) {
  uint64_t h = (a * x + b) >> (64 - ell);
  uint32_t d = lead_zeros(h, ell);
  if (d == ell) {
    uint64_t h2 = (a2 * x + b2) >> (64 - ell);
    d += lead_zeros(h2, ell);
  }
  return d < D - 1 ? d : D - 1;
}

static uint64_t key_of(const orc_graph* g, uint32_t r, uint32_t c) { return g->keys[(size_t)r * (g->C + 1) + c]; }

static uint64_t checksum(const orc_graph* g, uint32_t r, uint64_t idx) { return orc_mix64(idx ^ key_of(g, r, g->C)); }

static uint32_t column_depth(const orc_graph* g, uint32_t r, uint32_t c, uint64_t idx) {
  const uint64_t* k = g->keys + (size_t)g->L * (g->C + 1) + (size_t)3 * (r * g->C + c);
  return orc_mas_depth(key_of(g, r, c), k[0], k[1], k[2], g->ell, g->D, idx);
}

static orc_bucket* vertex_layer(const orc_graph* g, uint32_t w, uint32_t r) {
  return g->sketch + ((size_t)w * g->L + r) * g->W;
}

orc_graph* orc_create(uint32_t V, uint64_t seed, uint32_t L, uint32_t C, uint32_t D) {
  if (V < 2) return NULL;
  orc_graph* g = (orc_graph*)calloc(1, sizeof(orc_graph));
  if (!g) return NULL;
  orc_params(V, &L, &C, &D);
  g->V = V;
  g->L = L;
  g->C = C;
  g->D = D;
  g->W = 1 + C * D;
  g->seed = seed;
  g->ell = orc_hash_bits(V);
  g->keys = (uint64_t*)malloc(sizeof(uint64_t) * key_count(L, C));
  g->sketch = (orc_bucket*)calloc((size_t)V * L * g->W, sizeof(orc_bucket));
  g->label = (uint32_t*)malloc(sizeof(uint32_t) * V);
  g->forest = (uint64_t*)malloc(sizeof(uint64_t) * V);
  g->log_live = (uint32_t*)calloc(L, sizeof(uint32_t));
  g->log_ncand = (uint32_t*)calloc(L, sizeof(uint32_t));
  g->log_ids = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)V * L);
  if (!g->keys || !g->sketch || !g->label || !g->forest || !g->log_live || !g->log_ncand || !g->log_ids) {
    orc_destroy(g);
    return NULL;
  }
  orc_keys(seed, g->keys, key_count(L, C));
  for (uint32_t w = 0; w < V; w++) g->label[w] = w;
  g->dirty = 0; /* empty graph: every vertex alone, recovery already exact */
  g->complete = 1;
  return g;
}

void orc_destroy(orc_graph* g) {
  if (!g) return;
  free(g->keys);
  free(g->sketch);
  free(g->label);
  free(g->forest);
  free(g->log_live);
  free(g->log_ncand);
  free(g->log_ids);
  free(g);
}

void orc_get_params(const orc_graph* g, uint32_t* out4) {
  out4[0] = g->L;
  out4[1] = g->C;
  out4[2] = g->D;
  out4[3] = g->W;
}

/* Update of the l0 sketch of vertex w, layer r, by index idx of F_2^n
 * (Theorem A.2): XOR (idx, G(idx)) into the deterministic bucket and into
 * one bucket per column, the one at the index's depth in that column. */
static void sketch_layer_update(const orc_graph* g, orc_bucket* layer, uint32_t r, uint64_t idx) {
  uint64_t gam = checksum(g, r, idx);
  layer[0].alpha ^= idx;
  layer[0].gamma ^= gam;
  for (uint32_t c = 0; c < g->C; c++) {
    orc_bucket* b = &layer[1 + c * g->D + column_depth(g, r, c, idx)];
    b->alpha ^= idx;
    b->gamma ^= gam;
  }
}

/* App. A.1.1 ("The AGM Algorithm"): an update of edge (u,v) updates all of
 * the O(log V) sketches of u and of v. Over F_2 insert and delete are the
 * same toggle of coordinate idx of f_u and f_v. */
static void apply_edge(orc_graph* g, uint32_t u, uint32_t v) {
  uint32_t a = u < v ? u : v, b = u < v ? v : u;
  uint64_t idx = (uint64_t)a * g->V + b;
  for (uint32_t r = 0; r < g->L; r++) {
    sketch_layer_update(g, vertex_layer(g, a, r), r, idx);
    sketch_layer_update(g, vertex_layer(g, b, r), r, idx);
  }
}

int orc_update_batch(orc_graph* g, const uint32_t* edges, const int8_t* ops, size_t n) {
  /* Problem 1's stream: ((u,v), Delta), u != v in V, Delta in {-1, +1}. */
  for (size_t i = 0; i < n; i++) {
    uint32_t u = edges[2 * i], v = edges[2 * i + 1];
    if (u >= g->V || v >= g->V || u == v || (ops[i] != 1 && ops[i] != -1)) {
      g->sticky = ORC_EINVAL;
      return ORC_EINVAL;
    }
  }
  if (g->sticky) return ORC_OK; /* a pending error drops later batches too */
  for (size_t i = 0; i < n; i++) apply_edge(g, edges[2 * i], edges[2 * i + 1]);
  if (n > 0) g->dirty = 1;
  return ORC_OK;
}

int orc_sync(orc_graph* g) {
  int s = g->sticky;
  g->sticky = ORC_OK;
  return s;
}

static int bucket_good(const orc_graph* g, const orc_bucket* b, uint32_t r) {
  if (b->alpha == 0) return 0;
  if (checksum(g, r, b->alpha) != b->gamma) return 0;
  uint64_t u = b->alpha / g->V, v = b->alpha % g->V;
  return u < v;
}

/* Query of an l0 sketch (§2.1, Theorem A.2): return a non-zero coordinate
 * (an edge) or fail. The deterministic bucket tells ZERO from FAIL. */
static int sample_layer(const orc_graph* g, const orc_bucket* S, uint32_t r, uint64_t* edge) {
  if (S[0].alpha == 0 && S[0].gamma == 0) return ORC_ZERO;
  if (bucket_good(g, &S[0], r)) {
    *edge = S[0].alpha;
    return ORC_GOOD;
  }
  for (uint32_t c = 0; c < g->C; c++)
    for (uint32_t d = 0; d < g->D; d++) {
      const orc_bucket* b = &S[1 + c * g->D + d];
      if (bucket_good(g, b, r)) {
        *edge = b->alpha;
        return ORC_GOOD;
      }
    }
  return ORC_FAIL;
}

int orc_sample(const orc_graph* g, const uint64_t* layer, uint32_t r, uint64_t* edge) {
  return sample_layer(g, (const orc_bucket*)layer, r, edge);
}

static uint32_t uf_find(uint32_t* parent, uint32_t x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]]; /* path halving: same root, shorter paths */
    x = parent[x];
  }
  return x;
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* App. A.1.1: Boruvka over supernodes. Query each supernode's merged
 * sketch for an edge leaving it, merge the supernodes it joins (and so
 * their sketches, by XOR), repeat; O(log V) rounds, one sketch layer each. */
int orc_recover(orc_graph* g) {
  if (!g->dirty) return g->complete ? ORC_OK : ORC_EINCOMPLETE;
  const uint32_t V = g->V, W = g->W;
  uint8_t* final = (uint8_t*)calloc(V, 1);
  uint32_t* parent = (uint32_t*)malloc(sizeof(uint32_t) * V);
  uint32_t* count = (uint32_t*)malloc(sizeof(uint32_t) * V);
  uint32_t* minv = (uint32_t*)malloc(sizeof(uint32_t) * V);
  uint64_t* cand = (uint64_t*)malloc(sizeof(uint64_t) * V);
  orc_bucket* S = (orc_bucket*)malloc(sizeof(orc_bucket) * W);
  /* members of each component, as lists: head[K] -> next[w] -> ... */
  uint32_t* head = (uint32_t*)malloc(sizeof(uint32_t) * V);
  uint32_t* next = (uint32_t*)malloc(sizeof(uint32_t) * V);
  const uint32_t NIL = 0xFFFFFFFFu;

  for (uint32_t w = 0; w < V; w++) g->label[w] = w;
  g->n_forest = 0;
  g->rounds_run = 0;
  g->n_fail = 0;
  g->n_false_pos = 0;
  g->complete = 0;
  g->log_len = 0;

  for (uint32_t r = 0; r < g->L; r++) {
    /* component member lists from the labels at the start of round r */
    for (uint32_t w = 0; w < V; w++) head[w] = NIL;
    for (uint32_t w = V; w-- > 0;) {
      next[w] = head[g->label[w]];
      head[g->label[w]] = w;
    }
    size_t ncand = 0;
    uint32_t live = 0;
    int any_nonzero = 0;
    for (uint32_t K = 0; K < V; K++) {
      if (g->label[K] != K || final[K]) continue;
      live++;
      /* merged sketch of supernode K: XOR of its members' layer-r sketches */
      memset(S, 0, sizeof(orc_bucket) * W);
      for (uint32_t w = head[K]; w != NIL; w = next[w]) {
        const orc_bucket* x = vertex_layer(g, w, r);
        for (uint32_t j = 0; j < W; j++) {
          S[j].alpha ^= x[j].alpha;
          S[j].gamma ^= x[j].gamma;
        }
      }
      uint64_t e = 0;
      int res = sample_layer(g, S, r, &e);
      if (res == ORC_ZERO) {
        final[K] = 1;
        continue;
      }
      any_nonzero = 1;
      if (res == ORC_FAIL) {
        g->n_fail++;
        continue;
      }
      uint32_t u = (uint32_t)(e / V), v = (uint32_t)(e % V);
      int in_u = g->label[u] == K, in_v = g->label[v] == K;
      if (in_u != in_v)
        cand[ncand++] = e;
      else
        g->n_false_pos++;
    }
    g->rounds_run = r + 1;
    g->log_live[r] = live;
    if (!any_nonzero) {
      g->log_ncand[r] = 0;
      g->complete = 1;
      break;
    }
    /* Kruskal over the distinct candidates in ascending edge id, on the
     * components as they were at the start of the round */
    qsort(cand, ncand, sizeof(uint64_t), cmp_u64);
    size_t nd = 0;
    for (size_t i = 0; i < ncand; i++)
      if (nd == 0 || cand[nd - 1] != cand[i]) cand[nd++] = cand[i];
    g->log_ncand[r] = (uint32_t)nd;
    for (size_t i = 0; i < nd; i++) g->log_ids[g->log_len++] = cand[i];
    for (uint32_t w = 0; w < V; w++) parent[w] = w;
    for (size_t i = 0; i < nd; i++) {
      uint32_t u = (uint32_t)(cand[i] / V), v = (uint32_t)(cand[i] % V);
      uint32_t a = uf_find(parent, g->label[u]), b = uf_find(parent, g->label[v]);
      if (a != b) {
        parent[a] = b;
        g->forest[g->n_forest++] = cand[i];
      }
    }
    /* relabel to the minimum vertex id; a component that absorbed another
     * one has changed and is sampled again */
    for (uint32_t w = 0; w < V; w++) {
      minv[w] = NIL;
      count[w] = 0;
    }
    for (uint32_t K = 0; K < V; K++)
      if (g->label[K] == K) count[uf_find(parent, K)]++;
    for (uint32_t w = 0; w < V; w++) {
      uint32_t root = uf_find(parent, g->label[w]);
      if (w < minv[root]) minv[root] = w;
    }
    for (uint32_t w = 0; w < V; w++) {
      uint32_t root = uf_find(parent, g->label[w]);
      uint32_t newlabel = minv[root];
      if (count[root] > 1) final[newlabel] = 0;
      g->label[w] = newlabel;
    }
  }
  qsort(g->forest, g->n_forest, sizeof(uint64_t), cmp_u64);
  g->dirty = 0;
  free(final);
  free(parent);
  free(count);
  free(minv);
  free(cand);
  free(S);
  free(head);
  free(next);
  return g->complete ? ORC_OK : ORC_EINCOMPLETE;
}

/* Problem 2: Connected(u,v) on the graph defined by the updates so far. */
int orc_query(orc_graph* g, const uint32_t* pairs, size_t m, uint8_t* out) {
  for (size_t i = 0; i < m; i++)
    if (pairs[2 * i] >= g->V || pairs[2 * i + 1] >= g->V) return ORC_EINVAL;
  int s = orc_recover(g);
  for (size_t i = 0; i < m; i++) out[i] = g->label[pairs[2 * i]] == g->label[pairs[2 * i + 1]];
  return s;
}

/* Problem 1: a spanning forest of the graph, edge ids ascending. */
int orc_spanning_forest(orc_graph* g, uint64_t* out, size_t cap, size_t* n_out) {
  int s = orc_recover(g);
  *n_out = g->n_forest;
  if (cap < g->n_forest) return ORC_EINVAL;
  memcpy(out, g->forest, sizeof(uint64_t) * g->n_forest);
  return s;
}

void orc_labels(const orc_graph* g, uint32_t* out) { memcpy(out, g->label, sizeof(uint32_t) * g->V); }

void orc_stats(const orc_graph* g, uint64_t* stats) {
  stats[0] = g->rounds_run;
  stats[1] = g->n_fail;
  stats[2] = g->n_false_pos;
  stats[3] = (uint64_t)g->complete;
  stats[4] = g->log_len;
}

void orc_round_log(const orc_graph* g, uint32_t* live, uint32_t* ncand, uint64_t* ids) {
  for (uint64_t r = 0; r < g->rounds_run; r++) {
    live[r] = g->log_live[r];
    ncand[r] = g->log_ncand[r];
  }
  memcpy(ids, g->log_ids, sizeof(uint64_t) * g->log_len);
}

void orc_export(const orc_graph* g, uint64_t* dst) {
  for (uint32_t r = 0; r < g->L; r++)
    for (uint32_t w = 0; w < g->V; w++) {
      const orc_bucket* x = vertex_layer(g, w, r);
      uint64_t* o = dst + 2 * (((size_t)r * g->V + w) * g->W);
      for (uint32_t j = 0; j < g->W; j++) {
        o[2 * j] = x[j].alpha;
        o[2 * j + 1] = x[j].gamma;
      }
    }
}

/* The inverse of orc_export: every sketch word from src (same layout). The
 * sketches are the whole state, so the next query recovers from them. */
void orc_import(orc_graph* g, const uint64_t* src) {
  for (uint32_t r = 0; r < g->L; r++)
    for (uint32_t w = 0; w < g->V; w++) {
      orc_bucket* x = vertex_layer(g, w, r);
      const uint64_t* in = src + 2 * (((size_t)r * g->V + w) * g->W);
      for (uint32_t j = 0; j < g->W; j++) {
        x[j].alpha = in[2 * j];
        x[j].gamma = in[2 * j + 1];
      }
    }
  g->dirty = 1;
}

void orc_sketch_sum(const orc_graph* g, const uint32_t* verts, size_t n, uint32_t r, uint64_t* out) {
  memset(out, 0, sizeof(uint64_t) * 2 * g->W);
  for (size_t i = 0; i < n; i++) {
    const orc_bucket* x = vertex_layer(g, verts[i], r);
    for (uint32_t j = 0; j < g->W; j++) {
      out[2 * j] ^= x[j].alpha;
      out[2 * j + 1] ^= x[j].gamma;
    }
  }
}

void orc_vertex_sketch(uint32_t V, uint64_t seed, uint32_t L, uint32_t C, uint32_t D, uint32_t w,
                       const uint32_t* nbrs, size_t k, uint64_t* out) {
  orc_graph tmp;
  memset(&tmp, 0, sizeof(tmp));
  orc_params(V, &L, &C, &D);
  tmp.V = V;
  tmp.L = L;
  tmp.C = C;
  tmp.D = D;
  tmp.W = 1 + C * D;
  tmp.ell = orc_hash_bits(V);
  tmp.keys = (uint64_t*)malloc(sizeof(uint64_t) * key_count(L, C));
  orc_keys(seed, tmp.keys, key_count(L, C));
  memset(out, 0, sizeof(uint64_t) * 2 * (size_t)L * tmp.W);
  for (size_t i = 0; i < k; i++) {
    uint32_t a = w < nbrs[i] ? w : nbrs[i], b = w < nbrs[i] ? nbrs[i] : w;
    uint64_t idx = (uint64_t)a * V + b;
    for (uint32_t r = 0; r < L; r++)
      sketch_layer_update(&tmp, (orc_bucket*)(out + 2 * (size_t)r * tmp.W), r, idx);
  }
  free(tmp.keys);
}
