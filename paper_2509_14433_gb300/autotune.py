"""Autotuner for the update's apply kernel.

The apply kernel has three launch tunables (cupc_set_tuning): endpoint
records per work item, rows per column folded in shared memory, and CTAs per
SM. None of them changes the result; they trade shared-memory footprint,
occupancy and per-item overhead, and the best setting depends on how many
records a vertex receives per batch, i.e. on V and the batch size.

tune() times every candidate setting on the device (CUDA events recorded by
the library around each apply launch) for each batch-size bucket (powers of
four edges) and keeps the fastest, then times the write-back of single-item
vertices both ways (load-and-store, XOR atomics) with it and keeps the
faster; the table is stored as JSON keyed by GPU
name and graph shape. apply() sets the setting of one batch size as a
graph's default; apply_buckets() gives the graph every bucket's setting, and
the library then picks one per batch by its size. Run `python -m paper_2509_14433_gb300.autotune --V 16384` on the
target GPU to (re)write the table; `--batches rmat` times R-MAT batches (the
degree skew of the batched R-MAT workload) instead of uniform ones.
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "tuning_gb300.json")

ITEM_RECORDS = (64, 128, 256, 512)
SMEM_ROWS = (8, 12, 16)
CTAS_PER_SM = (0, 2)


def bucket_of(n_edges: int) -> int:
    """Bucket = floor(log4(n)), at least 5 (1024 edges)."""
    b = 5
    while (4 ** (b + 1)) <= n_edges:
        b += 1
    return b


def shape_key(V: int, L: int, C: int, D: int) -> str:
    return f"V={V},L={L},C={C},D={D}"


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(0)


def load(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _entry(table: dict, V: int, L: int, C: int, D: int, n_edges: int):
    try:
        import torch
        name = torch.cuda.get_device_name(0)
    except Exception:
        return None
    ent = table.get(name, {}).get(shape_key(V, L, C, D))
    if not ent:
        return None
    b = bucket_of(n_edges)
    keys = sorted(int(k) for k in ent)
    return ent[str(min(keys, key=lambda k: abs(k - b)))]


def lookup(table: dict, V: int, L: int, C: int, D: int, n_edges: int):
    """(item_records, smem_rows, ctas_per_sm) for this GPU, shape and batch
    size, or None (defaults stay)."""
    e = _entry(table, V, L, C, D, n_edges)
    return None if e is None else tuple(e["setting"])


def apply(g, V: int, n_edges: int, table: dict | None = None) -> bool:
    """Set the tuned setting for a batch of n_edges on graph handle g."""
    from . import cupc as C
    p = np.zeros(4, np.uint32)
    C.cupc_get_params(g, p)
    L, Cc, D, _ = (int(x) for x in p)
    e = _entry(load() if table is None else table, V, L, Cc, D, n_edges)
    if e is None:
        return False
    if "writeback" in e:
        C.check(C.cupc_set_writeback_bucket(g, bucket_of(n_edges), int(e["writeback"])))
    return C.cupc_set_tuning(g, *e["setting"]) == C.CUPC_OK


def apply_buckets(g, V: int, table: dict | None = None) -> int:
    """Set every tuned batch-size bucket of this GPU and graph shape on
    graph handle g (cupc_set_tuning_bucket), so that each batch runs with
    the setting of its own size. Returns the number of buckets set."""
    from . import cupc as C
    try:
        import torch
        name = torch.cuda.get_device_name(0)
    except Exception:
        return 0
    p = np.zeros(4, np.uint32)
    C.cupc_get_params(g, p)
    L, Cc, D, _ = (int(x) for x in p)
    ent = (load() if table is None else table).get(name, {}).get(shape_key(V, L, Cc, D), {})
    k = 0
    for b, e in ent.items():
        if 5 <= int(b) <= 15 and C.cupc_set_tuning_bucket(g, int(b), *e["setting"]) == C.CUPC_OK:
            k += 1
            if "writeback" in e:
                C.check(C.cupc_set_writeback_bucket(g, int(b), int(e["writeback"])))
    return k


def _time_setting(C, g, e_d, o_d, n, reps, setting, writeback=0):
    if C.cupc_set_tuning(g, *setting) != C.CUPC_OK:
        return None
    if C.cupc_set_writeback_bucket(g, bucket_of(n), writeback) != C.CUPC_OK:
        return None
    C.check(C.cupc_update_batch(g, e_d, o_d, n, None))  # warm
    C.cupc_profile_enable(g, 1)
    for _ in range(reps):
        C.check(C.cupc_update_batch(g, e_d, o_d, n, None))
    ms = np.zeros(8)
    nl = np.zeros(8, np.uint64)
    C.cupc_profile_read(g, ms, nl, 8)
    C.cupc_profile_enable(g, 0)
    return float(ms[2]) / max(1, int(nl[2]))


RMAT_PROBS = (0.57, 0.19, 0.19, 0.05)


def _batch(WL, V: int, n: int, rng, batches: str, gen):
    """n edge pairs (uint32 [n, 2], u != v) on the device: uniform random, or
    R-MAT (V a power of two; a self-loop's second end moves to the next id)."""
    import torch
    if batches == "rmat":
        levels = V.bit_length() - 1
        u, v = WL.rmat_pairs(n, levels, RMAT_PROBS, gen, "cuda")
        v = torch.where(u == v, (v + 1) % V, v)
        return torch.stack([u, v], 1).to(torch.int32).reshape(-1).contiguous()
    return torch.from_numpy(WL.uniform_pairs(V, n, rng).reshape(-1)).cuda()


def tune(V: int, sizes=None, reps: int = 3, seed: int = 1, path: str = DEFAULT_CACHE, verbose: bool = True,
         batches: str = "uniform"):
    """Time every setting per batch-size bucket on a graph of V vertices
    with uniform random or R-MAT batches (the degree skew of the batches
    decides how many records a vertex gets); merge the winners into the
    JSON table."""
    import torch

    from . import cupc as C
    from . import workloads as WL
    if sizes is None:
        sizes = [4 ** b for b in range(5, 12) if 4 ** b <= (1 << 22)]
    st, g = C.cupc_init(V, seed, (0, 0, 0, max(sizes)), None, None)  # each batch is one launch
    C.check(st, "cupc_init")
    p = np.zeros(4, np.uint32)
    C.cupc_get_params(g, p)
    L, Cc, D, _ = (int(x) for x in p)
    if batches == "rmat" and V & (V - 1):
        raise ValueError("R-MAT batches need V a power of two")
    rng = WL.rng(seed)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    table = load(path)
    ent = table.setdefault(gpu_name(), {}).setdefault(shape_key(V, L, Cc, D), {})
    try:
        for n in sizes:
            e_d = _batch(WL, V, n, rng, batches, gen)
            o_d = torch.ones(n, dtype=torch.int8, device="cuda")
            results = []
            for it in ITEM_RECORDS:
                for rows in SMEM_ROWS:
                    if rows > D:
                        continue
                    for cps in CTAS_PER_SM:
                        t = _time_setting(C, g, e_d, o_d, n, reps, (it, rows, cps))
                        if t is not None:
                            results.append((t, (it, rows, cps)))
            results.sort()
            best_t, best = results[0]
            default = [t for t, s in results if s == (256, min(8, D), 0)]
            # the write-back of single-item vertices, forced each way, for the best setting
            wb_t = {m: _time_setting(C, g, e_d, o_d, n, reps, best, m)
                    for m in (C.CUPC_WRITEBACK_LOAD_STORE, C.CUPC_WRITEBACK_ATOMIC)}
            wb = min(wb_t, key=lambda m: wb_t[m])
            C.cupc_set_writeback_bucket(g, bucket_of(n), C.CUPC_WRITEBACK_AUTO)
            ent[str(bucket_of(n))] = {"setting": list(best), "apply_ms": min(best_t, wb_t[wb]),
                                      "default_ms": default[0] if default else None, "edges": n,
                                      "batches": batches, "writeback": wb,
                                      "writeback_ms": {str(m): t for m, t in wb_t.items()}}
            if verbose:
                print(f"V={V} n={n}: best {best} {best_t:.4f} ms (default {default[0] if default else '-'} ms), "
                      f"write-back load-store {wb_t[1]:.4f} / atomic {wb_t[2]:.4f} ms", flush=True)
    finally:
        C.cupc_destroy(g)
    with open(path + ".tmp", "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(path + ".tmp", path)
    return ent


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--V", type=int, nargs="+", default=[16384])
    ap.add_argument("--max-edges", type=int, default=1 << 22)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=DEFAULT_CACHE)
    ap.add_argument("--batches", nargs="+", default=["uniform"], choices=["uniform", "rmat"],
                    help="batch kind per --V entry (the last one repeats)")
    a = ap.parse_args()
    for k, V in enumerate(a.V):
        sizes = [4 ** b for b in range(5, 12) if 4 ** b <= a.max_edges]
        tune(V, sizes, reps=a.reps, path=a.out, batches=a.batches[min(k, len(a.batches) - 1)])


if __name__ == "__main__":
    main()
