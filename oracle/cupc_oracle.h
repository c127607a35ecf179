/*
 * CPU oracle for sketch-based connectivity (CameoSketch vertex sketches +
 * Boruvka recovery), arXiv 2509.14433.
 *
 * TEST INFRASTRUCTURE ONLY. This library is the plain, slow reference the
 * CUDA path is checked against. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it. It shares no code, header,
 * table or constant generator with the CUDA library, and the CUDA library
 * never calls it.
 *
 * Everything is integer arithmetic; results are exact.
 *
 * What each part follows in the paper:
 *   - l0 sketch of a vector over F_2 (CameoSketch): App. A.1.1, Theorem A.2;
 *     sketch addition = elementwise XOR of machine words: App. A.1.1.
 *   - characteristic vector f_u and O(log V) sketches per vertex, update of
 *     both endpoints: App. A.1.1, paragraph "The AGM Algorithm".
 *   - recovery by Boruvka rounds over merged sketches: same paragraph.
 *   - spanning forest output: App. A.1, Problem 1.
 *   - Connected(u,v) after a prefix of the stream: App. A.2, Problem 2; §2.1.
 * The paper fixes no bucket layout, hash function, checksum, scan order or
 * parameter constants. The readings used here are:
 *   - edge (u,v), u<v<V, has index idx = u*V + v;
 *   - lg = ceil(log2 V) (at least 1); layers L = lg+2; rows D = 2*lg;
 *     columns C = 7; a layer is 1 deterministic bucket + C*D column buckets;
 *   - a bucket is {alpha = XOR of idx, gamma = XOR of G(idx)}, 2 x u64;
 *   - mix() is the SplitMix64 output finalizer (Steele, Lea, Flood,
 *     OOPSLA 2014); key K(j) = mix(seed + phi*(j+1)), phi =
 *     0x9E3779B97F4A7C15, i.e. the SplitMix64 stream seeded with `seed`;
 *   - column hash (Theorem A.1 needs 2-wise independence): two stages of
 *     multiply-add-shift (Dietzfelbinger, STACS 1996),
 *     h(x) = ((a*x + b) mod 2^64) div 2^(64-ell), ell = 65 - 2*lg, strongly
 *     universal onto ell bits for x < 2^(2*lg); column c of layer r uses
 *     a = K(r*(C+1) + c) and b, a', b' = K(L*(C+1) + 3*(r*C + c) + 0, 1, 2);
 *     depth d = min(leading zeros of the 2*ell-bit string h(x) h'(x), D-1)
 *     (h' is read only when h(x) = 0);
 *   - checksum G_r(idx) = mix(idx ^ K(r*(C+1) + C));
 *   - a bucket is good iff alpha != 0, G_r(alpha) == gamma and alpha decodes
 *     to u < v < V;
 *   - sample: det zero -> ZERO; det good -> det; else first good bucket in
 *     column-major order (c = 0..C-1, then d = 0..D-1); else FAIL;
 *   - round r of recovery uses layer r only; a component whose merged sketch
 *     is ZERO has an empty cut and is not sampled again until it changes;
 *     candidate edges are hooked by Kruskal in ascending edge id; labels are
 *     the minimum vertex id of each component.
 *
 * Parity pins (what checks this code against something other than itself):
 *   orc_mix64 / keys ......... published SplitMix64 test vectors
 *   orc_mas_depth ............ closed forms for chosen keys (powers of two,
 *                              zero multiplier, wrap-around, second stage);
 *                              over random keys: the geometric depth law
 *                              and pairwise independence of two indices
 *                              (Theorem A.1's requirement)
 *   updates .................. linearity, insert/delete cancellation,
 *                              all-vertex XOR = 0, single-edge recovery
 *   orc_sample ............... cut property on random subsets, ZERO iff the
 *                              cut is empty, scan-order special cases
 *   orc_recover / query ...... BFS / union-find on exhaustive and random
 *                              small graphs; forest properties; graphs that
 *                              are forests recover themselves; planted
 *                              sketches traced by hand: a checksum-valid
 *                              sample that does not cross the cut is
 *                              counted and not hooked, and a ZERO component
 *                              that absorbs another is sampled again
 */
#ifndef CUPC_ORACLE_H
#define CUPC_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_OK = 0,
  ORC_EINVAL = 1,
  ORC_ENOMEM = 2,
  ORC_EINCOMPLETE = 3
};

enum { ORC_ZERO = 0, ORC_GOOD = 1, ORC_FAIL = 2 };

typedef struct orc_graph orc_graph;

uint64_t orc_mix64(uint64_t z);
/* Fill out[0..n) with key j = mix(seed + phi*(j+1)). */
void orc_keys(uint64_t seed, uint64_t* out, size_t n);
/* Parameter derivation; a non-zero input overrides the default. */
void orc_params(uint32_t V, uint32_t* L, uint32_t* C, uint32_t* D);
/* Output bits ell of one multiply-add-shift stage for graphs of V vertices. */
uint32_t orc_hash_bits(uint32_t V);
/* Depth of index x in a column with keys (a, b, a2, b2): the leading zero
 * bits of the 2*ell-bit string ((a*x+b) mod 2^64) >> (64-ell) followed by
 * ((a2*x+b2) mod 2^64) >> (64-ell), capped at D-1. */
uint32_t orc_mas_depth(uint64_t a, uint64_t b, uint64_t a2, uint64_t b2, uint32_t ell, uint32_t D, uint64_t x);

orc_graph* orc_create(uint32_t V, uint64_t seed, uint32_t L, uint32_t C, uint32_t D);
void orc_destroy(orc_graph* g);
void orc_get_params(const orc_graph* g, uint32_t* out4 /* L,C,D,W */);

/* Apply a batch of n edge updates; edges = u0,v0,u1,v1,...; ops = +1/-1.
 * The whole batch is validated first: on any invalid entry nothing is
 * applied, a sticky error is recorded and ORC_EINVAL returned. */
int orc_update_batch(orc_graph* g, const uint32_t* edges, const int8_t* ops, size_t n);
/* Return and clear the sticky error. */
int orc_sync(orc_graph* g);

/* Boruvka recovery (recomputed only when an update happened since the
 * last one). Returns ORC_OK or ORC_EINCOMPLETE. */
int orc_recover(orc_graph* g);
int orc_query(orc_graph* g, const uint32_t* pairs, size_t m, uint8_t* out);
int orc_spanning_forest(orc_graph* g, uint64_t* out, size_t cap, size_t* n_out);
void orc_labels(const orc_graph* g, uint32_t* out);
/* stats[0]=rounds run, [1]=FAIL samples, [2]=checksum false positives,
 * [3]=complete flag, [4]=number of candidate entries logged */
void orc_stats(const orc_graph* g, uint64_t* stats);
/* Per-round log of the live-component count and the distinct candidate ids
 * of the last recovery: counts[r] for r < rounds run; ids concatenated. */
void orc_round_log(const orc_graph* g, uint32_t* live, uint32_t* ncand, uint64_t* ids);

/* Export all sketches as [layer r][vertex w][bucket j] x {alpha, gamma}. */
void orc_export(const orc_graph* g, uint64_t* dst);
/* Overwrite every sketch word (orc_export's layout); the next query
 * recovers from them. Lets tests plant sketch contents no stream makes. */
void orc_import(orc_graph* g, const uint64_t* src);
/* Layer-r buckets of the sum of the sketches of vertices verts[0..n). */
void orc_sketch_sum(const orc_graph* g, const uint32_t* verts, size_t n, uint32_t r, uint64_t* out);
/* Sample a W-bucket layer-r sketch; returns ORC_ZERO/GOOD/FAIL. */
int orc_sample(const orc_graph* g, const uint64_t* layer, uint32_t r, uint64_t* edge);

/* Sketch of one vertex w whose neighbour set is nbrs[0..k) (its
 * characteristic vector), without any graph state: out is [r][j] x 2 u64. */
void orc_vertex_sketch(uint32_t V, uint64_t seed, uint32_t L, uint32_t C, uint32_t D,
                       uint32_t w, const uint32_t* nbrs, size_t k, uint64_t* out);

#ifdef __cplusplus
}
#endif
#endif
