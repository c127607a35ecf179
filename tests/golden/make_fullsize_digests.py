"""Write the oracle's digests of two workloads at full size.

Runs the CPU oracle (oracle/, single thread) on the whole stream of

  dense_v16384:    V = 16384, ER(0.5) edges inserted in a seeded random order,
                   then a uniform random 10% deleted (workloads.dense_stream,
                   seed 1), hash seed 1; then one 1k-pair Connected batch and
                   the spanning forest;
  cliques_v131072: V = 131072 as 256 cliques of 512 (33.5M edges), then 8
                   bridge insert and 8 bridge delete batches of 64k with a
                   1k-pair Connected batch after each (workloads.clique_stream,
                   seed 7), hash seed 1; then the spanning forest;

and stores, per workload (tests/golden/fullsize_<workload>.json), SHA-256 digests of every sketch word (the export
layout [layer][vertex][bucket][alpha, gamma], little-endian u64), the labels,
the forest (ids ascending), the round log of every recovery (live components
and candidate ids per round) and the answers of every query batch, with the
recovery counters (rounds, FAIL samples, checksum false positives, complete).
The GPU tests recompute the same digests from the CUDA path.

Usage: python tests/golden/make_fullsize_digests.py [dense_v16384|cliques_v131072 ...]
(about 15 minutes per workload on one core). Nothing here calls the CUDA
library; the inputs come from the seeded generators only.
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2509_14433_gb300 import workloads as WL  # noqa: E402

def out_path(name: str) -> str:
    return os.path.join(HERE, f"fullsize_{name}.json")


SEED = 1
CHUNK = 1 << 20


def sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def round_log_digest(log) -> str:
    h = hashlib.sha256()
    for live, ids in log:
        h.update(np.array([live, len(ids)], np.uint64).tobytes())
        h.update(np.ascontiguousarray(np.sort(ids), np.uint64).tobytes())
    return h.hexdigest()


def recovery_record(g, status, answers=None) -> dict:
    st = g.stats()
    rec = {"status": int(status), "rounds": st["rounds"], "fail": st["fail"], "false_pos": st["false_pos"],
           "complete": bool(st["complete"]), "round_log": round_log_digest(g.round_log())}
    if answers is not None:
        rec["answers"] = sha(np.asarray(answers, np.uint8))
        rec["connected"] = int(np.count_nonzero(answers))
    return rec


def apply(g, E, op):
    for i in range(0, len(E), CHUNK):
        e = E[i:i + CHUNK]
        assert g.update(e, np.full(len(e), op, np.int8)) == O.OK


def final_record(g) -> dict:
    s, forest = g.spanning_forest()
    return {"forest_status": int(s), "forest_edges": int(len(forest)), "forest": sha(forest.astype(np.uint64)),
            "labels": sha(g.labels()), "sketches": sha(g.export())}


def dense_v16384() -> dict:
    V = 16384
    E, n_del, order = WL.dense_stream(V=V, p=0.5, batch=CHUNK, delete_frac=0.1, seed=SEED)
    D = E[order[:n_del]]
    g = O.Graph(V, SEED)
    apply(g, E, 1)
    apply(g, D, -1)
    pairs = WL.uniform_pairs(V, 1000, WL.rng(77), distinct=False)
    s, ans = g.query(pairs)
    out = {"workload": "dense_stream(V=16384, p=0.5, delete_frac=0.1, seed=1), hash seed 1, "
                       "query pairs uniform_pairs(V, 1000, rng(77), distinct=False)",
           "updates": int(len(E) + len(D)), "queries": [recovery_record(g, s, ans)]}
    out.update(final_record(g))
    g.close()
    return out


def cliques_v131072() -> dict:
    V = 131072
    cl, order, pairs, _ = WL.clique_stream(V=V, seed=7)
    g = O.Graph(V, SEED)
    apply(g, cl, 1)
    qs = []
    for E, op in order:
        apply(g, E, op)
        s, ans = g.query(pairs)
        qs.append(recovery_record(g, s, ans))
    out = {"workload": "clique_stream(V=131072, k=256, s=512, 8+8 bridge batches of 65536, seed=7), hash seed 1, "
                       "the stream's 1k pairs after every bridge batch",
           "updates": int(len(cl) + sum(len(E) for E, _ in order)), "queries": qs}
    out.update(final_record(g))
    g.close()
    return out


def main():
    for name in sys.argv[1:] or ["dense_v16384", "cliques_v131072"]:
        t = time.time()
        rec = globals()[name]()
        rec["oracle_seconds"] = round(time.time() - t, 1)
        with open(out_path(name), "w") as f:
            json.dump(rec, f, indent=1, sort_keys=True)
        print(name, "done in", rec["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
