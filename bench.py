"""Throughput benchmark of the sketch-connectivity hot path on GB300.

Headline workload (one step = one whole job, inputs resident in HBM before
timing): the batched R-MAT stream on V = 2^17 vertices, (a, b, c, d) =
(.57, .19, .19, .05), 1e9 updates of which 20% delete previously inserted
edges, in batches of log-uniform size in [1k, 4M], applied as back-to-back
batches (cupc_update_batches: coalesced into 4M-edge launches of the
persistent apply kernel with autotuned per-size settings), then one 1k-pair
Connected batch (the Boruvka recovery) and the spanning forest. The stream
(9 GB) and the sketches (9.5 GB) are larger than L2, so no flush is needed.
value = edge updates per second over the whole job (all ranks).

Also reported: the same job end to end through the C-ABI from pinned host
buffers (e2e), the one-batch-per-launch arm, the live roofline of the
dominant kernel (the sketch apply kernel), the other workloads (plain
V=1024 toggle stream, dense V=16384, 64-graph serving closed and open loop,
256 cliques on V=2^17, the paper's stream shapes) with query p50/p99 over
at least 1000 query batches each, and the CPU oracle timed on a stated
bounded sample of each.

--impl reference times the CPU oracle on the headline workload (a bounded
sample per step) and prints the same JSON line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2509_14433_gb300 import workloads as WL  # noqa: E402

METRIC = "edge updates/s and p99 Connected-query latency on 1 GB300, bit-exact; HBM GB/s"
UNIT = "edge updates/s"
SEED = 1  # hash seed of every graph
# headline: the batched R-MAT workload
V_RMAT, RMAT_LEVELS, RMAT_UPDATES, RMAT_SEED, MAXB = 1 << 17, 17, 1_000_000_000, 3, 4 << 20
# dense ER(0.5) workload
V_DENSE, P_DENSE, BATCH = 16384, 0.5, 1 << 20
QUERY_SAMPLES = 1000  # query batches behind every p50/p99
CPU_RMAT_SAMPLE = 1 << 19  # headline oracle sample (updates)
REF_RMAT_SAMPLE = 1 << 18  # reference arm sample per step (updates)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(value: float, device=None) -> float:
    """The slowest rank's value (all ranks must call it); the value itself on
    a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step: int, steps: int, world: int, max_ms: float) -> float:
    """Weak scaling: every rank processes units_per_step per step; the job's
    rate is all ranks' units over the slowest rank's time."""
    return units_per_step * steps * world / (max_ms / 1e3)


def pcts(lat_us):
    a = np.asarray(lat_us, np.float64)
    return {"p50_us": float(np.percentile(a, 50)), "p99_us": float(np.percentile(a, 99)), "samples": int(a.size)}


def headline_config(n, nb, sizes):
    return {"workload": f"batched R-MAT(V={V_RMAT}, a=.57 b=.19 c=.19 d=.05): {n} updates (20% deletes of present "
                        f"edges) in {nb} batches of log-uniform size in [1000, {MAXB}] (min {min(sizes)}, max "
                        f"{max(sizes)}), applied back to back in {MAXB}-edge launches, then a 1k-pair Connected "
                        "batch and the spanning forest",
            "V": V_RMAT, "updates_per_step": int(n), "batches": int(nb), "max_launch_edges": MAXB,
            "stream_seed": RMAT_SEED, "hash_seed": SEED,
            "apply_tuning": "autotuned per batch-size bucket (paper_2509_14433_gb300/tuning_gb300.json)",
            "l2": "inputs larger than L2 (sketches 9.5 GB, edge stream 9 GB): no flush"}


def expected_touched_buckets(counts, L, C, D):
    """Expected distinct buckets an update batch touches, given the number of
    batch records n_w of each vertex: per vertex and layer, the deterministic
    bucket plus, per column, sum_d 1 - (1 - p_d)^n_w with p_d = 2^-(d+1)
    (the last row takes the tail 2^-(D-1)). Depths are uniform over the hash
    keys, so the sum over ~10^6 independent columns is tight around this
    expectation."""
    vals, mult = np.unique(counts[counts > 0], return_counts=True)
    p = 2.0 ** -(np.arange(D) + 1.0)
    p[-1] = 2.0 ** -(D - 1)
    per_col = (1.0 - (1.0 - p[None, :]) ** vals[:, None].astype(np.float64)).sum(axis=1)
    return float(L * (mult * (1.0 + C * per_col)).sum())


def dense_sweep_bytes(counts, L, W):
    """Bytes a dense sweep of the batch would move: read and write back the
    whole sketch (L layers x W buckets x 16 B) of every vertex the batch
    touches, against the distinct buckets k_apply touches."""
    return float(2 * 16 * L * W * np.count_nonzero(counts))


def apply_source_digest():
    """md5 over the source k_apply compiles from: the shared device header
    (update_dev.cuh), the kernel's own text in update.cu, and the device
    functions and constants of common.cuh it uses."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2509_14433_gb300", "csrc")
    h = hashlib.md5()
    h.update(open(os.path.join(csrc, "update_dev.cuh"), "rb").read())
    upd = open(os.path.join(csrc, "update.cu")).read()
    m = re.search(r"__global__ void k_apply\(.*?\n}\n", upd, re.S)
    h.update((m.group(0) if m else upd).encode())
    com = open(os.path.join(csrc, "common.cuh")).read()
    for m in re.finditer(r"^__(?:host__ __)?device__ .*?\n}\n|^__device__ [^\n]*}\n", com, re.S | re.M):
        h.update(m.group(0).encode())
    for m in re.finditer(r"^constexpr uint32_t k(?:ErrInval|DirectItem\w*|SmemRows\w*|\w*ItemRecords|Stage) = [^;]*;"
                         r"|^  GC_(?:ERR|NITEMS|NEXT_ITEM) = \d+", com, re.M):
        h.update(m.group(0).encode())
    return h.hexdigest()


def apply_traffic(workload):
    """DRAM bytes per k_apply launch on this workload from the committed ncu
    summary; None when the kernel's source changed since the counters were
    taken or the summary covers another workload."""
    tp = os.path.join(ROOT, "profiles", "k_apply_traffic.json")
    try:
        rec = json.load(open(tp))
    except (OSError, ValueError):
        return None
    if rec.get("source_md5") != apply_source_digest() or rec.get("workload") != workload:
        return None
    return rec.get("bytes_per_launch")


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(index)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- inputs -----------------------------------------------------------------

def gen_rmat_stream(torch, dev, n_updates=RMAT_UPDATES, seed=RMAT_SEED):
    """The batched workload's stream, generated on `dev` and stored back to
    back: edges int32 [n, 2], ops int8 [n], batch offsets (k+1, host)."""
    s = WL.RmatStream(levels=RMAT_LEVELS, seed=seed, device=dev)
    cap = n_updates + MAXB
    E = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    O = torch.empty(cap, dtype=torch.int8, device=dev)
    offs = [0]
    while offs[-1] < n_updates:
        e, o = s.next_batch()
        a, n = offs[-1], len(o)
        E[a:a + n] = e
        O[a:a + n] = o
        offs.append(a + n)
    fallbacks = s.fallbacks
    del s
    torch.cuda.empty_cache()
    n = offs[-1]
    return E[:n], O[:n], np.array(offs, np.uint64), fallbacks


def make_dense_stream():
    E, n_del, order = WL.dense_stream(V=V_DENSE, p=P_DENSE, batch=BATCH, delete_frac=0.1, seed=SEED)
    return E, E[order[:n_del]]


# ---- CPU oracle samples (bounded; one thread) --------------------------------

def oracle_rmat_sample(E_h, n):
    """The oracle on the first n updates of the headline stream (one batch),
    one 1k-pair Connected batch (the recovery) and the spanning forest."""
    import oracle as O
    pairs = WL.uniform_pairs(V_RMAT, 1000, WL.rng(SEED + 7), distinct=False)
    g = O.Graph(V_RMAT, SEED)
    t = time.perf_counter()
    assert g.update(E_h[:n]) == O.OK
    tq = time.perf_counter()
    s, _ = g.query(pairs)
    tq = time.perf_counter() - tq
    assert s in (O.OK, O.EINCOMPLETE)
    g.spanning_forest()
    dt = time.perf_counter() - t
    g.close()
    return dt, tq


def cpu_samples(E_rmat_h, dense_E, plain_steps, cl, bridge_batch, serving_one):
    """The oracle timed on a stated sample of every workload."""
    import oracle as O
    out = {}
    dt, tq = oracle_rmat_sample(E_rmat_h, CPU_RMAT_SAMPLE)
    out["rmat_v131072"] = {"updates_per_s": CPU_RMAT_SAMPLE / dt, "query_batch_ms": 1e3 * tq,
                           "sample": f"first {CPU_RMAT_SAMPLE} updates + 1k-pair Connected batch + forest"}
    n = 2 * BATCH
    g = O.Graph(V_DENSE, SEED)
    t = time.perf_counter()
    g.update(dense_E[:n])
    tq = time.perf_counter()
    g.query(WL.uniform_pairs(V_DENSE, 1000, WL.rng(8), distinct=False))
    tq = time.perf_counter() - tq
    dt = time.perf_counter() - t
    g.close()
    out["dense_v16384"] = {"updates_per_s": n / dt, "query_batch_ms": 1e3 * tq,
                           "sample": f"first {n} inserts + 1k-pair Connected batch"}
    g = O.Graph(1024, SEED)
    nu, lat = 0, []
    t = time.perf_counter()
    for st in plain_steps:
        if st[0] == "update":
            g.update(st[1], st[2])
            nu += len(st[2])
        else:
            t1 = time.perf_counter()
            g.query(st[1])
            lat.append(time.perf_counter() - t1)
    dt = time.perf_counter() - t
    g.close()
    out["plain_v1024"] = {"updates_per_s": nu / (dt - sum(lat)), "query_batch_ms_p50": 1e3 * float(np.median(lat)),
                          "sample": "the whole stream (start graph, 200k toggles, 20 query batches)"}
    n = 1 << 20
    g = O.Graph(131072, SEED)
    t = time.perf_counter()
    g.update(cl[:n])
    g.update(bridge_batch)
    tq = time.perf_counter()
    g.query(WL.uniform_pairs(131072, 1000, WL.rng(9), distinct=False))
    tq = time.perf_counter() - tq
    dt = time.perf_counter() - t
    g.close()
    out["cliques_v131072"] = {"updates_per_s": (n + 65536) / dt, "query_batch_ms": 1e3 * tq,
                              "sample": f"first {n} clique edges + one 64k bridge batch + 1k-pair Connected batch"}
    V, seed_i, steps, nupd = serving_one
    g = O.Graph(V, seed_i)
    t = time.perf_counter()
    for st in steps:
        if st[0] == "update":
            g.update(st[1], st[2])
        else:
            g.query(st[1])
    dt = time.perf_counter() - t
    g.close()
    out["serving_64_graphs"] = {"updates_per_s": nupd / dt,
                                "sample": f"one graph's whole stream (V={V}, {nupd} updates with its query batches)"}
    return out


# ---- reference arm ------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import torch
    if torch.cuda.is_available():
        # the headline stream itself (the generator runs on the device; no
        # library code is involved), for its first updates and its shape
        E, O, offs, _ = gen_rmat_stream(torch, torch.device("cuda", 0))
        E_h = E[:REF_RMAT_SAMPLE].cpu().numpy().astype(np.uint32)
        cfg = headline_config(int(offs[-1]), len(offs) - 1, np.diff(offs).astype(np.int64))
        del E, O
        torch.cuda.empty_cache()
    else:  # the same generator and seed on the host: its first batches
        s = WL.RmatStream(levels=RMAT_LEVELS, seed=RMAT_SEED, device="cpu")
        parts, n = [], 0
        while n < REF_RMAT_SAMPLE:
            e, _ = s.next_batch()
            parts.append(e.numpy().astype(np.uint32))
            n += len(e)
        E_h = np.concatenate(parts)
        del s
        cfg = headline_config(RMAT_UPDATES, 0, [1000, MAXB])
    cfg["sample"] = (f"per step: the oracle on the first {REF_RMAT_SAMPLE} updates of this stream, one 1k-pair "
                     "Connected batch and the spanning forest (single thread)")
    for _ in range(args.warmup):
        oracle_rmat_sample(E_h, REF_RMAT_SAMPLE)
    times, qtimes = [], []
    for _ in range(args.steps):
        dt, tq = oracle_rmat_sample(E_h, REF_RMAT_SAMPLE)
        times.append(dt)
        qtimes.append(tq)
    tot = sum(times)
    val = REF_RMAT_SAMPLE * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": cfg, "units_per_step": REF_RMAT_SAMPLE,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": cfg["sample"],
                             "query_batch_ms_p50": 1e3 * float(np.median(qtimes))},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- GPU arm ------------------------------------------------------------------

def run_gpu(args):
    import torch

    from paper_2509_14433_gb300 import autotune as AT
    from paper_2509_14433_gb300 import cupc as C

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()

    stream = torch.cuda.current_stream()
    t_gen = time.perf_counter()
    E, O, offs, fallbacks = gen_rmat_stream(torch, dev)
    t_gen = time.perf_counter() - t_gen
    n, nb = int(offs[-1]), len(offs) - 1
    sizes = np.diff(offs).astype(np.int64)
    V = V_RMAT
    st, g = C.cupc_init(V, SEED, (0, 0, 0, MAXB), None, stream)
    C.check(st, "cupc_init")
    n_buckets = AT.apply_buckets(g, V)
    prm = np.zeros(4, np.uint32)
    C.cupc_get_params(g, prm)
    L, Cc, Dd, W = (int(x) for x in prm)
    pairs = WL.uniform_pairs(V, 1000, WL.rng(77), distinct=False)
    P_d = torch.from_numpy(pairs.reshape(-1)).to(dev)
    q_out = torch.empty(1000, dtype=torch.uint8, device=dev)
    forest_d = torch.empty(V, dtype=torch.int64, device=dev)
    Eflat = E.reshape(-1)

    def step_device():
        C.check(C.cupc_reset(g, stream))
        C.check(C.cupc_update_batches(g, Eflat, O, offs, nb, stream))
        C.check(C.cupc_query(g, P_d, 1000, q_out, stream), "query", ok=(C.CUPC_OK, C.CUPC_EINCOMPLETE))
        st, nf = C.cupc_spanning_forest(g, forest_d, V, stream)
        C.check(st, "spanning_forest", ok=(C.CUPC_OK, C.CUPC_EINCOMPLETE))
        return nf

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    C.cupc_profile_enable(g, 1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        nf = step_device()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_prof = np.zeros(8)
    nl_prof = np.zeros(8, np.uint64)
    C.cupc_profile_read(g, ms_prof, nl_prof, 8)
    C.cupc_profile_enable(g, 0)
    ms = ev0.elapsed_time(ev1)
    barrier()
    ms = max_over_ranks(ms, dev)
    value = whole_job_rate(n, args.steps, world, ms)
    assert C.cupc_sync(g, stream) == C.CUPC_OK

    # ---- e2e: the same job through the C-ABI from pinned host buffers, in
    # calls of at most MAXB edges (each copy overlaps the previous launch)
    E_h = torch.empty(E.shape, dtype=torch.int32, pin_memory=True)
    E_h.copy_(E)
    O_h = torch.empty(O.shape, dtype=torch.int8, pin_memory=True)
    O_h.copy_(O)
    P_h = torch.from_numpy(pairs.reshape(-1).copy()).pin_memory()
    q_h = torch.empty(1000, dtype=torch.uint8).pin_memory()
    forest_h = torch.empty(V, dtype=torch.int64).pin_memory()
    e_ptr, o_ptr = E_h.data_ptr(), O_h.data_ptr()

    def step_host():
        C.check(C.cupc_reset(g, stream))
        for i in range(0, n, MAXB):
            k = min(MAXB, n - i)
            C.check(C.cupc_update_batch(g, e_ptr + 8 * i, o_ptr + i, k, stream))
        C.check(C.cupc_query(g, P_h, 1000, q_h, stream), "query", ok=(C.CUPC_OK, C.CUPC_EINCOMPLETE))
        st, nf = C.cupc_spanning_forest(g, forest_h, V, stream)
        C.check(st, "spanning_forest", ok=(C.CUPC_OK, C.CUPC_EINCOMPLETE))
        return nf

    step_host()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e2e_steps = 3
    for _ in range(e2e_steps):
        nf_h = step_host()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s = max_over_ranks(e2e_s, dev)
    e2e_val = whole_job_rate(n, e2e_steps, world, e2e_s * 1e3)
    assert nf_h == nf and torch.equal(forest_h[:nf], forest_d[:nf].cpu())
    assert torch.equal(q_h, q_out.cpu())
    E_cpu_sample = E_h[:max(CPU_RMAT_SAMPLE, REF_RMAT_SAMPLE)].numpy().astype(np.uint32).copy()
    del E_h, O_h

    rows, extra = {}, {}
    if rank == 0 and world == 1:
        # ---- the same stream one batch per launch (updates only, both arms)
        def upd_coalesced():
            C.check(C.cupc_update_batches(g, Eflat, O, offs, nb, stream))

        def upd_plain():
            for i in range(nb):
                a = int(offs[i])
                C.check(C.cupc_update_batch(g, E[a:].reshape(-1), O[a:], int(sizes[i]), stream))

        arms = {}
        for name, fn in (("coalesced_4M_launches", upd_coalesced), ("one_batch_per_launch", upd_plain)):
            C.check(C.cupc_reset(g, stream))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            arms[name] = n / (e0.elapsed_time(e1) / 1e3)
        extra["batched_vs_one_batch_per_launch"] = {"updates": n, "batches": nb, "updates_per_s": arms,
                                                    "fallback_uniform_inserts": int(fallbacks),
                                                    "stream_generation_s": t_gen}
        # ---- query latency on the final graph: a 1k-pair Connected batch
        # right after an update batch (a toggle of the stream's last 64k
        # updates, so the recovery runs); host submit -> answers ready
        lat = []
        tail = max(0, n - 65536)
        for k in range(QUERY_SAMPLES + 5):
            C.check(C.cupc_update_batch(g, E[tail:].reshape(-1), O[tail:], n - tail, stream))
            torch.cuda.synchronize()
            t = time.perf_counter()
            C.check(C.cupc_query(g, P_d, 1000, q_out, stream), "query", ok=(C.CUPC_OK, C.CUPC_EINCOMPLETE))
            torch.cuda.synchronize()
            if k >= 5:
                lat.append((time.perf_counter() - t) * 1e6)
        rows["rmat_v131072"] = {"updates_per_s": value, "e2e_updates_per_s": e2e_val,
                                "queries_per_s_in_query_batches": 1000 / (np.mean(lat) * 1e-6),
                                "query_after_64k_batch": pcts(lat), "forest_edges": int(nf)}

    # ---- roofline of the dominant kernel (sketch apply), measured live in
    # the timed steps: algorithmic bytes of every launch (from its chunk's
    # vertex counts) over the launches' CUDA-event time
    touched, sweep = [], []
    for i in range(0, n, MAXB):
        cnt = torch.bincount(Eflat[2 * i:2 * min(n, i + MAXB)].long(), minlength=V).cpu().numpy()
        touched.append(expected_touched_buckets(cnt, L, Cc, Dd))
        sweep.append(dense_sweep_bytes(cnt, L, W))
    apply_bytes_per_launch = 32.0 * float(np.mean(touched))
    apply_launches = int(nl_prof[2])
    assert apply_launches == args.steps * len(touched), (apply_launches, len(touched))
    apply_ms = ms_prof[2] / max(1, apply_launches)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = apply_bytes_per_launch / (apply_ms * 1e-3) / 1e9
    gpu_launches = int(nl_prof.sum())
    shares = {name: round(float(ms_prof[k]) / max(1e-9, float(ms_prof.sum())), 4)
              for k, name in enumerate(["validate", "group", "apply", "recover", "query", "sort"])}
    C.cupc_destroy(g)
    del E, O, Eflat
    torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1:
        dense_E, dense_D = make_dense_stream()
        rows["dense_v16384"], extra["batch_size_vs_query_latency"] = dense_rows(torch, C, dev, stream, dense_E,
                                                                                dense_D)
        plain_steps = WL.plain_stream(V=1024, seed=1)
        rows["plain_v1024"] = plain_rows(torch, C, dev, stream, plain_steps)
        cl, border, cpairs, comp = WL.clique_stream(V=131072, seed=7)
        rows["cliques_v131072"] = clique_rows(torch, C, dev, stream, cl, border, cpairs, comp)
        streams = WL.serving_streams(n_graphs=64, upd_range=(5e4, 5e5), seed=5)
        if not args.no_serving:
            rows["serving_64_graphs"] = serving_rows(torch, C, streams)
        if not args.no_batching:
            extra["batching_many_graphs"] = many_graphs(torch, C, dev, stream)
            extra["paper_stream_shape"] = paper_stream(torch, C, dev, stream)
        if not args.no_cpu_baseline:
            cs = cpu_samples(E_cpu_sample, dense_E, plain_steps, cl, border[0][0], streams[0])
            for k, v in cs.items():
                rows.setdefault(k, {})["cpu_oracle_1_thread"] = v
            cpu = {"value": cs["rmat_v131072"]["updates_per_s"], "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"first {CPU_RMAT_SAMPLE} updates of the headline stream + one 1k-pair "
                             "Connected batch + spanning forest (single thread)",
                   "query_batch_ms": cs["rmat_v131072"]["query_batch_ms"]}

    if rank == 0:
        cfg = headline_config(n, nb, sizes)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": cfg,
                "e2e": {"value": e2e_val, "unit": UNIT,
                        "h2d_bytes_per_step": int(9 * n + 8000), "d2h_bytes_per_step": int(1000 + 8 * nf_h)},
                "gpu_launches": gpu_launches, "apply_tuning_buckets_set": n_buckets,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": apply_traffic("rmat_v131072"),
                             "kernel": "k_apply", "algorithmic_bytes_per_launch": apply_bytes_per_launch,
                             "dense_sweep_bytes_per_launch": float(np.mean(sweep)),
                             "launches_per_step": len(touched), "avg_launch_ms": apply_ms,
                             "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy), of measured" if peaks
                             else "fallback 6800 GB/s"},
                "kernel_time_share": shares,
                "per_config": rows,
                **extra,
                "cpu_baseline": cpu, "clocks": clk}
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


# ---- the other workloads (rank 0, one GPU) -------------------------------------

def dense_rows(torch, C, dev, stream, E, D):
    """Dense V=16384: the whole job (all inserts, 10% deletes in 2^20
    batches, the forest), the query latency after a 2^20-edge batch, and the
    batch size against the latency of the next query batch."""
    V = V_DENSE
    nE, nD = len(E), len(D)
    E_d = torch.from_numpy(E.reshape(-1)).to(dev)
    D_d = torch.from_numpy(D.reshape(-1)).to(dev)
    ins_d = torch.ones(nE, dtype=torch.int8, device=dev)
    del_d = torch.full((nD,), -1, dtype=torch.int8, device=dev)
    forest_d = torch.empty(V, dtype=torch.int64, device=dev)
    st, g = C.cupc_init(V, SEED, None, None, stream)
    C.check(st)
    from paper_2509_14433_gb300 import autotune as AT
    AT.apply_buckets(g, V)

    def job():
        C.check(C.cupc_reset(g, stream))
        for i in range(0, nE, BATCH):
            C.check(C.cupc_update_batch(g, E_d[2 * i:], ins_d[i:], min(BATCH, nE - i), stream))
        for i in range(0, nD, BATCH):
            C.check(C.cupc_update_batch(g, D_d[2 * i:], del_d[i:], min(BATCH, nD - i), stream))
        st, nf = C.cupc_spanning_forest(g, forest_d, V, stream)
        C.check(st, ok=(C.CUPC_OK, C.CUPC_EINCOMPLETE))
        return nf

    job()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(2):
        nf = job()
    e1.record(stream)
    torch.cuda.synchronize()
    upd_s = 2 * (nE + nD) / (e0.elapsed_time(e1) / 1e3)
    pairs = torch.from_numpy(WL.uniform_pairs(V, 1000, WL.rng(77), distinct=False).reshape(-1)).to(dev)
    q_out = torch.empty(1000, dtype=torch.uint8, device=dev)
    lat = []
    for k in range(QUERY_SAMPLES + 5):
        i = (k % 6) * BATCH  # toggle one 2^20-edge batch, then ask
        C.check(C.cupc_update_batch(g, E_d[2 * i:], ins_d[i:], BATCH, stream))
        torch.cuda.synchronize()
        t = time.perf_counter()
        C.check(C.cupc_query(g, pairs, 1000, q_out, stream))
        torch.cuda.synchronize()
        if k >= 5:
            lat.append((time.perf_counter() - t) * 1e6)
    C.check(C.cupc_sync(g, stream))
    job()  # back to the stream's final graph (a valid stream for the sweep)
    sweep = batch_latency_sweep(torch, C, g, D_d, ins_d, del_d, pairs, q_out, stream)
    C.cupc_destroy(g)
    row = {"updates_per_s": upd_s, "updates_per_step": nE + nD, "forest_edges": int(nf),
           "query_after_2^20_batch": pcts(lat), "queries_per_s_in_query_batches": 1000 / (np.mean(lat) * 1e-6)}
    return row, sweep


def batch_latency_sweep(torch, C, g, D_d, ins_d, del_d, p_d, q_out, stream, reps=200):
    """Update batch size against the latency of the next Connected query
    batch (the trade-off the paper's update buffering makes): for each size
    b from 1 to 4M, insert then delete the first b of the deleted edges
    (absent, then present: a valid stream) and ask 1k pairs after each batch,
    `reps` times. Latency = host submit of the batch to the query's answer,
    recovery included."""
    out = {}
    for b in [4 ** k for k in range(12)]:
        upd, lat = [], []
        for k in range(reps + 2):  # the first two passes warm up
            ops = ins_d if k % 2 == 0 else del_d
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            C.check(C.cupc_update_batch(g, D_d, ops, b, stream))
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            C.check(C.cupc_query(g, p_d, 1000, q_out, stream))
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            if k >= 2:
                upd.append(t1 - t0)
                lat.append((t2 - t0) * 1e6)
        out[str(b)] = {"updates_per_s": b / statistics.median(upd), **pcts(lat)}
    return out


def plain_rows(torch, C, dev, stream, steps, reps=50):
    """Plain V=1024: ER(0.5) start graph + 200k toggles, a 1k-pair Connected
    batch every 10k updates, replayed `reps` times (20 query batches each):
    toggle updates/s and query latency (host submit -> answers ready,
    recovery included), with and without incremental labels."""
    V = 1024
    out = {}
    dsteps = []
    for s in steps:
        if s[0] == "update":
            dsteps.append(("u", torch.from_numpy(s[1].reshape(-1)).to(dev), torch.from_numpy(s[2]).to(dev), len(s[2])))
        else:
            dsteps.append(("q", torch.from_numpy(s[1].reshape(-1)).to(dev),
                           torch.empty(len(s[1]), dtype=torch.uint8, device=dev), len(s[1])))
    for mode, inc in (("recovery_per_query", 0), ("incremental_labels", 1)):
        st, g = C.cupc_init(V, SEED, None, None, stream)
        C.check(st)
        C.check(C.cupc_set_incremental(g, inc, stream))
        lat, upd_t, n_upd = [], 0.0, 0
        for rep in range(reps + 1):
            C.cupc_reset(g, stream)
            for kind, a, b, n in dsteps:
                torch.cuda.synchronize()
                t = time.perf_counter()
                if kind == "u":
                    C.check(C.cupc_update_batch(g, a, b, n, stream))
                else:
                    C.check(C.cupc_query(g, a, n, b, stream))
                torch.cuda.synchronize()
                dt = time.perf_counter() - t
                if rep == 0:
                    continue  # warm-up pass
                if kind == "u":
                    if n <= 10_000:
                        upd_t += dt
                        n_upd += n
                else:
                    lat.append(dt * 1e6)
        C.cupc_destroy(g)
        out[mode] = {"toggle_updates_per_s": n_upd / upd_t, "query": pcts(lat),
                     "queries_per_s_in_query_batches": 1000 / (np.mean(lat) * 1e-6)}
    return out


def clique_rows(torch, C, dev, stream, cl, order, pr, comp, rounds=63):
    """Adversarial V=131072: 256 cliques of 512 (33.5M edges, inserted in
    2^20 batches: the set-up, timed on its own), then `rounds` passes of 8
    bridge insert batches and 8 shuffled bridge delete batches of 64k, a
    1k-pair Connected batch after every batch (half inside one clique, half
    across two). Answers are checked against the exact components."""
    V, k = 131072, 256
    st, g = C.cupc_init(V, SEED, (0, 0, 0, BATCH), None, stream)
    C.check(st)
    from paper_2509_14433_gb300 import autotune as AT
    AT.apply_buckets(g, V)
    cl_d = torch.from_numpy(cl.reshape(-1)).to(dev)
    ones = torch.ones(len(cl), dtype=torch.int8, device=dev)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for i in range(0, len(cl), BATCH):
        C.check(C.cupc_update_batch(g, cl_d[2 * i:], ones[i:], min(BATCH, len(cl) - i), stream))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t
    dorder = [(torch.from_numpy(np.ascontiguousarray(E).reshape(-1)).to(dev),
               torch.full((len(E),), op, dtype=torch.int8, device=dev), len(E)) for E, op in order]
    P_d = torch.from_numpy(pr.reshape(-1)).to(dev)
    q_out = torch.empty(1000, dtype=torch.uint8, device=dev)
    # the exact answers after each batch of a pass: cliques joined by the
    # bridges present
    want = []
    present = np.zeros(0, np.int64)
    for E, op in order:
        ids = E[:, 0].astype(np.int64) * V + E[:, 1]
        present = np.union1d(present, ids) if op == 1 else np.setdiff1d(present, ids)
        parent = np.arange(k)

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x

        for x, y in zip(comp[present // V].tolist(), comp[present % V].tolist()):
            rx, ry = find(x), find(y)
            if rx != ry:
                parent[rx] = ry
        root = np.array([find(c) for c in range(k)])
        want.append(root[comp[pr[:, 0]]] == root[comp[pr[:, 1]]])
    lat, upd_t, n_upd, wrong = [], 0.0, 0, 0
    for rnd in range(rounds + 1):
        for j, (e, o, m) in enumerate(dorder):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            C.check(C.cupc_update_batch(g, e, o, m, stream))
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            C.check(C.cupc_query(g, P_d, 1000, q_out, stream))
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            if rnd:
                upd_t += t1 - t0
                n_upd += m
                lat.append((t2 - t1) * 1e6)
                wrong += int((q_out.cpu().numpy().astype(bool) != want[j]).sum())
    C.cupc_destroy(g)
    return {"clique_setup_updates_per_s": len(cl) / setup_s, "bridge_updates_per_s": n_upd / upd_t,
            "query_after_each_bridge_batch": pcts(lat), "wrong_answers": wrong,
            "queries_per_s_in_query_batches": 1000 / (np.mean(lat) * 1e-6)}


def many_graphs(torch, C, dev, stream, rounds=30):
    """64 graphs with V log-uniform in [2^10, 2^15], each receiving a
    1k-edge batch per round: 64 cupc_update_batch calls per round vs one
    cupc_batcher_update call (CUDA graph replay, and without the graph)."""
    rng = WL.rng(17)
    Vs = [int(2 ** x) for x in rng.uniform(10, 15, size=64)]
    graphs = []
    for i, V in enumerate(Vs):
        st, h = C.cupc_init(V, 100 + i, (0, 0, 0, 1 << 16), None, stream)
        C.check(st)
        graphs.append(h)
    m = 1000
    bat = [(torch.from_numpy(WL.uniform_pairs(V, rounds * m, rng).reshape(-1)).to(dev),
            torch.ones(rounds * m, dtype=torch.int8, device=dev)) for V in Vs]

    def plain_many():
        for r in range(rounds):
            for h, (e, o) in zip(graphs, bat):
                C.check(C.cupc_update_batch(h, e.data_ptr() + 8 * r * m, o.data_ptr() + r * m, m, stream))

    res = {}
    for name, use_graph in (("one_batch_per_launch", None), ("batcher_cuda_graph", True), ("batcher_no_graph", False)):
        if use_graph is None:
            fn = plain_many
            b = None
        else:
            st, b = C.cupc_batcher_create(64, use_graph)
            C.check(st)

            def fn(b=b):
                for r in range(rounds):
                    C.check(C.cupc_batcher_update(b, graphs, [e.data_ptr() + 8 * r * m for e, _ in bat],
                                                  [o.data_ptr() + r * m for _, o in bat], [m] * len(graphs), stream))
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = rounds * m * len(graphs) / (e0.elapsed_time(e1) / 1e3)
        if b is not None:
            C.cupc_batcher_destroy(b)
    for h in graphs:
        C.cupc_destroy(h)
    return {"graphs": len(graphs), "V_min": min(Vs), "V_max": max(Vs), "rounds": rounds, "updates_per_s": res}


def wait_until(due):
    while True:
        now = time.perf_counter()
        if now >= due:
            return
        if due - now > 2e-4:
            time.sleep(due - now - 1e-4)


def serving_rows(torch, C, streams, maxb=1 << 20):
    """Serving workload: 64 graphs, V log-uniform in [2^10, 2^15], ER(p)
    insert/delete streams with p ~ U[0.1, 0.9], batches log-uniform in
    [1k, 1M], a 1k-pair Connected batch after every 100k updates of a graph;
    requests in round-robin order over the graphs.

    closed loop: every request submitted at t = 0; cupc_server with no memory
    cap and with a cap of 25% of the graphs' total workspace, against one
    thread serving one request at a time. Latency = arrival to completion.

    open loop: requests arrive with seeded exponential gaps at a fixed
    offered rate (a fraction of the one-at-a-time arm's closed-loop request
    rate, so below its saturation), replayed until at least 1000 query
    batches were measured per point; latency is measured from each request's
    scheduled arrival, for cupc_server and for the one-at-a-time arm (a FIFO
    single server: a request starts at max(its arrival, the previous
    completion))."""
    order = WL.round_robin(streams)
    total_upd = sum(st[3] for st in streams)
    n_graphs = len(streams)
    ws = [C.cupc_workspace_bytes(st[0], (0, 0, 0, maxb)) for st in streams]
    reqs = []
    for i, stp in order:
        if stp[0] == "update":
            reqs.append((i, "u", np.ascontiguousarray(stp[1], np.uint32), np.ascontiguousarray(stp[2], np.int8)))
        else:
            reqs.append((i, "q", np.ascontiguousarray(stp[1], np.uint32), None))
    nq = sum(1 for r in reqs if r[1] == "q")
    out = {"graphs": n_graphs, "updates": int(total_upd), "requests": len(reqs), "query_batches": nq}
    last = {}
    for k, r in enumerate(reqs):
        last[r[0]] = k

    def served_run(cap_bytes, arrivals=None):
        """One pass of every request through a fresh server; arrivals: the
        scheduled arrival offsets (s) or None (all at t = 0). Returns
        (query latencies from arrival in us, makespan s, stats)."""
        st, srv = C.cupc_server_create(int(cap_bytes), n_graphs, maxb, 4, 1 << 30)
        C.check(st)
        try:
            ids = [C.cupc_server_open(srv, s_[0], s_[1])[1] for s_ in streams]
            outs, ut, qt = [], [], []
            t0 = time.perf_counter()
            for k, (i, kind, a, b) in enumerate(reqs):
                lag = 0.0
                if arrivals is not None:
                    wait_until(t0 + arrivals[k])
                    lag = time.perf_counter() - (t0 + arrivals[k])
                if kind == "u":
                    r, t = C.cupc_server_update(srv, ids[i], a, b, len(b))
                    ut.append(t)
                else:
                    ans = np.zeros(len(a), np.uint8)
                    outs.append(ans)
                    r, t = C.cupc_server_query(srv, ids[i], a, len(a), ans)
                    qt.append((t, lag))
                C.check(r, "submit")
                if k == last[i]:
                    ut.append(C.cupc_server_close(srv, ids[i])[1])
            for t in ut:
                C.check(C.cupc_server_wait(srv, t, 600000)[0], "update")
            lat = []
            for t, lag in qt:
                r, l_us = C.cupc_server_wait(srv, t, 600000)
                C.check(r, "query")
                lat.append(l_us + 1e6 * lag)
            span = time.perf_counter() - t0
            stats = np.zeros(8, np.uint64)
            C.cupc_server_stats(srv, stats)
            return lat, span, stats
        finally:
            C.cupc_server_destroy(srv)

    graphs = []
    for s_ in streams:
        r, g = C.cupc_init(s_[0], s_[1], (0, 0, 0, maxb), None, None)
        C.check(r)
        graphs.append(g)

    def plain_run(arrivals=None):
        """One thread, one request at a time, each finished before the next
        starts (FIFO); latency from the scheduled arrival."""
        for g in graphs:
            C.cupc_reset(g, None)
        torch.cuda.synchronize()
        lat = []
        t0 = time.perf_counter()
        for k, (i, kind, a, b) in enumerate(reqs):
            arr = 0.0 if arrivals is None else arrivals[k]
            if arrivals is not None:
                wait_until(t0 + arr)
            if kind == "u":
                C.check(C.cupc_update_batch(graphs[i], a, b, len(b), None))
                torch.cuda.synchronize()
            else:
                ans = np.zeros(len(a), np.uint8)
                C.check(C.cupc_query(graphs[i], a, len(a), ans, None))
                lat.append((time.perf_counter() - (t0 + arr)) * 1e6)
        return lat, time.perf_counter() - t0

    try:
        full = sum(ws) * 1.02 + (256 << 20)
        out["closed_loop"] = {}
        for name, cap in (("served_no_cap", full), ("served_cap_25pct", 0.25 * sum(ws))):
            served_run(cap)  # warm-up
            lat, span, stats = served_run(cap)
            out["closed_loop"][name] = {
                "updates_per_s": total_upd / span, "query": pcts(lat), "makespan_s": span,
                "update_launches": int(stats[2]), "update_requests": int(stats[3]),
                "admission_waits": int(stats[5])}
        plain_run()  # warm-up
        lat, span = plain_run()
        out["closed_loop"]["one_request_at_a_time"] = {"updates_per_s": total_upd / span, "query": pcts(lat),
                                                       "makespan_s": span}
        rate_plain = len(reqs) / span  # requests/s the one-at-a-time arm sustains
        rounds = max(1, -(-QUERY_SAMPLES // nq))
        g_rng = WL.rng(31)
        pts = []
        for frac in (0.25, 0.5, 0.75):
            rate = frac * rate_plain
            pt = {"offered_requests_per_s": rate, "offered_updates_per_s": rate * total_upd / len(reqs),
                  "fraction_of_one_at_a_time_capacity": frac}
            for arm in ("served", "one_request_at_a_time"):
                lat_all, upd_s = [], []
                for _ in range(rounds):
                    arrivals = np.cumsum(g_rng.exponential(1.0 / rate, size=len(reqs)))
                    if arm == "served":
                        lat, span, _ = served_run(full, arrivals)
                    else:
                        lat, span = plain_run(arrivals)
                    lat_all += lat
                    upd_s.append(total_upd / span)
                pt[arm] = {"query": pcts(lat_all), "achieved_updates_per_s": float(np.mean(upd_s))}
            pts.append(pt)
        out["open_loop"] = pts
    finally:
        for g in graphs:
            C.cupc_destroy(g)
    return out


def paper_stream(torch, C, dev, stream):
    """The paper's two stream shapes on a K13-sized dense graph (context for
    its published numbers, not the headline workload): V = 2^13, ER(0.5)
    edges (about the K13 density). The standard stream inserts every edge,
    then deletes every edge; the fixed forest stream inserts one spanning
    forest, then inserts every other edge and deletes it again (one cycle).
    Updates arrive in bursts of rho ~ U[1000, 2000], each followed by rho/9
    uniform Connected pairs (10% of the operations are queries). Each whole
    stream runs with a full recovery per query burst and with incremental
    labels (cupc_set_incremental): updates/s and queries/s over the stream,
    the recoveries it ran, and the latency of every 16th burst (its update
    batch and its queries, host submit -> answers ready)."""
    V = 1 << 13
    paper = {"standard": ("K13", 1.79e6, 3.37e6), "fixed_forest": ("K13-FF", 4.56e6, 6.92e6)}
    res = {"workload": "V=8192 ER(0.5), whole streams, query bursts of rho/9 pairs every rho ~ U[1000,2000] "
                       "updates", "paper_cupcake_48core_epyc": {}}
    st, g = C.cupc_init(V, 1, None, None, stream)
    C.check(st)
    stats = np.zeros(8, np.uint64)

    def recoveries():
        C.check(C.cupc_stats(g, stats, stream))
        return int(stats[5])

    for shape in ("standard", "fixed_forest"):
        if shape == "standard":
            E, ops = WL.standard_stream(V, 0.5, 13)
        else:
            E, ops, _ = WL.fixed_forest_stream(V, 0.5, 13, cycles=1)
        g_rng = WL.rng(17)
        bursts, i = [], 0
        while i < len(E):
            rho = int(g_rng.integers(1000, 2001))
            bursts.append((i, min(rho, len(E) - i), max(1, rho // 9)))
            i += rho
        n_q = sum(b[2] for b in bursts)
        E_d = torch.from_numpy(E.reshape(-1)).to(dev)
        ops_d = torch.from_numpy(ops).to(dev)
        P_d = torch.from_numpy(WL.uniform_pairs(V, n_q, g_rng, distinct=False).reshape(-1)).to(dev)
        out_d = torch.empty(n_q, dtype=torch.uint8, device=dev)

        def run(todo, sample_every=0):
            lat, q = [], 0
            for k, (i, n, m) in enumerate(todo):
                sample = sample_every and k % sample_every == sample_every - 1
                if sample:
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                C.check(C.cupc_update_batch(g, E_d[2 * i:], ops_d[i:], n, stream))
                C.check(C.cupc_query(g, P_d[2 * q:], m, out_d[q:], stream))
                if sample:
                    torch.cuda.synchronize()
                    lat.append((time.perf_counter() - t) * 1e6)
                q += m
            return lat

        name, pu, pq = paper[shape]
        res["paper_cupcake_48core_epyc"][name] = {"updates_per_s": pu, "queries_per_s": pq}
        out = {"updates": len(E), "inserts": int(np.sum(ops == 1)), "deletes": int(np.sum(ops == -1)),
               "queries": n_q, "bursts": len(bursts)}
        for mode, inc in (("recovery_per_burst", 0), ("incremental_labels", 1)):
            C.check(C.cupc_set_incremental(g, inc, stream))
            C.check(C.cupc_reset(g, stream))
            run(bursts[:64])  # warm-up
            C.check(C.cupc_reset(g, stream))
            r0 = recoveries()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            run(bursts)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            nrec = recoveries() - r0
            C.check(C.cupc_reset(g, stream))
            lat = run(bursts, sample_every=16)
            out[mode] = {"updates_per_s": len(E) / dt, "queries_per_s": n_q / dt, "recoveries": nrec,
                         "burst_latency": pcts(lat)}
        res[shape] = out
        del E_d, ops_d, P_d, out_d
    C.check(C.cupc_sync(g, stream), "paper stream", ok=(C.CUPC_OK, C.CUPC_EINCOMPLETE))
    C.cupc_destroy(g)
    return res


PAPER_TABLE1 = {  # CUPCaKE on a 48-core EPYC 7643 (context only): updates/s, queries/s
    13: {"standard": (1.79e6, 3.37e6), "fixed_forest": (4.56e6, 6.92e6)},
    15: {"standard": (0.84e6, 1.72e6), "fixed_forest": (2.19e6, 3.75e6)},
    16: {"standard": (0.88e6, 1.87e6), "fixed_forest": (1.75e6, 2.99e6)},
    17: {"standard": (0.61e6, 1.35e6), "fixed_forest": (1.63e6, 2.81e6)},
}


PERM_ONE = (1 << 31) - 1  # torch's device sorts (randperm) take at most this many elements
PERM_CHUNK = 1 << 30


def shuffled_parts(x, gen):
    """The elements of x in a random order, as a sequence of tensors. Up to
    PERM_ONE elements: one uniform permutation. Above: x is dealt into
    c = ceil(len / PERM_CHUNK) strided subsequences x[j::c] (each spans the
    whole id range, so every part touches every vertex region), each is
    permuted uniformly, and the parts come in a random order."""
    import torch
    m = x.numel()
    if m <= PERM_ONE:
        yield x[torch.randperm(m, generator=gen, device=x.device)]
        return
    c = -(-m // PERM_CHUNK)
    for j in torch.randperm(c, generator=gen, device=x.device).tolist():
        sub = x[j::c]
        yield sub[torch.randperm(sub.numel(), generator=gen, device=x.device)]


def run_paper_streams(args):
    """The paper's stream shapes (§5 datasets, App. C) on Kronecker-shaped
    graphs of V = 2^levels at density 0.5 (workloads.kronecker_graph): the
    standard stream (insert every edge, then delete every edge, each phase in
    a fresh random order) and the fixed forest stream (insert a spanning
    forest, then insert every other edge and delete it again), with a burst
    of rho/9 uniform Connected pairs after every rho ~ U[1000, 2000]
    updates. Each whole stream runs once with incremental labels (and, for
    the smallest graph, once with a full recovery per burst): updates/s and
    queries/s over the whole stream, the recoveries it ran. Prints one JSON
    line per (graph, stream, mode)."""
    import torch

    from paper_2509_14433_gb300 import cupc as C
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    for levels in [int(x) for x in args.kron.split(",")]:
        V = 1 << levels
        gen = torch.Generator(device=dev).manual_seed(100 + levels)
        t0 = time.perf_counter()
        ids, parent = WL.kronecker_graph(levels, 100 + levels, device=dev)
        t_gen = time.perf_counter() - t0
        m = ids.numel()
        ar = torch.arange(V, device=dev)
        fmask = parent != ar
        forest = parent[fmask] * V + ar[fmask]
        roots = int((~fmask).sum())
        st, g = C.cupc_init(V, SEED, (0, 0, 0, 1 << 16), None, stream)
        C.check(st)
        stats = np.zeros(8, np.uint64)
        fsorted = torch.sort(forest).values
        for shape in ("standard", "fixed_forest"):
            if shape == "standard":
                phases = [(ids, 1, True), (ids, -1, True)]
            else:
                keep = torch.ones(m, dtype=torch.bool, device=dev)
                keep[torch.searchsorted(ids, fsorted)] = False
                rest = torch.cat([ids[a:a + PERM_CHUNK][keep[a:a + PERM_CHUNK]] for a in range(0, m, PERM_CHUNK)])
                del keep
                phases = [(forest, 1, False), (rest, 1, True), (rest, -1, True)]
            n = sum(x.numel() for x, _, _ in phases)
            E = torch.empty((n, 2), dtype=torch.int32, device=dev)
            ops = torch.empty(n, dtype=torch.int8, device=dev)
            at = 0
            for x, op, shuffle in phases:
                for part in (shuffled_parts(x, gen) if shuffle else [x]):
                    k = part.numel()
                    E[at:at + k, 0] = (part // V).to(torch.int32)
                    E[at:at + k, 1] = (part % V).to(torch.int32)
                    ops[at:at + k] = op
                    at += k
                    del part
            del phases
            if shape == "fixed_forest":
                del rest
            rng = WL.rng(17 + levels)
            rho = rng.integers(1000, 2001, size=n // 1000 + 2)
            starts = np.concatenate([[0], np.cumsum(rho)])
            nb = int(np.searchsorted(starts, n))
            starts = np.minimum(starts[:nb + 1], n)
            qn = np.maximum(1, (starts[1:] - starts[:-1]) // 9)
            qoff = np.concatenate([[0], np.cumsum(qn)])
            P = torch.empty(2 * int(qoff[-1]), dtype=torch.int32, device=dev)
            for a in range(0, P.numel(), PERM_CHUNK):
                b = min(P.numel(), a + PERM_CHUNK)
                P[a:b] = torch.randint(0, V, (b - a,), generator=gen, device=dev, dtype=torch.int32)
            out = torch.empty(int(qoff[-1]), dtype=torch.uint8, device=dev)
            e_ptr, o_ptr, p_ptr, a_ptr = E.data_ptr(), ops.data_ptr(), P.data_ptr(), out.data_ptr()
            modes = (("incremental_labels", 1),) + ((("recovery_per_burst", 0),) if levels <= 13 else ())
            for mode, inc in modes:
                C.check(C.cupc_set_incremental(g, inc, stream))
                C.check(C.cupc_reset(g, stream))
                C.check(C.cupc_stats(g, stats, stream))
                r0 = int(stats[5])
                torch.cuda.synchronize()
                t = time.perf_counter()
                for b in range(nb):
                    a, z = int(starts[b]), int(starts[b + 1])
                    C.check(C.cupc_update_batch(g, e_ptr + 8 * a, o_ptr + a, z - a, stream))
                    q0, q1 = int(qoff[b]), int(qoff[b + 1])
                    C.check(C.cupc_query(g, p_ptr + 8 * q0, q1 - q0, a_ptr + q0, stream), "query",
                            ok=(C.CUPC_OK, C.CUPC_EINCOMPLETE))
                torch.cuda.synchronize()
                dt = time.perf_counter() - t
                C.check(C.cupc_stats(g, stats, stream))
                pu, pq = PAPER_TABLE1[levels][shape]
                print(json.dumps({"graph": f"Kronecker V=2^{levels} density 0.5", "edges": m, "forest_roots": roots,
                                  "stream": shape, "mode": mode, "updates": n, "queries": int(qoff[-1]),
                                  "bursts": nb, "seconds": dt, "updates_per_s": n / dt,
                                  "queries_per_s": int(qoff[-1]) / dt, "recoveries": int(stats[5]) - r0,
                                  "generation_s": t_gen,
                                  "paper_cupcake_48core_epyc": {"updates_per_s": pu, "queries_per_s": pq}}),
                      flush=True)
            del E, ops, P, out
            torch.cuda.empty_cache()
        C.check(C.cupc_sync(g, stream), "paper streams", ok=(C.CUPC_OK, C.CUPC_EINCOMPLETE))
        C.cupc_destroy(g)
        del ids, parent, forest
        torch.cuda.empty_cache()


def run_apply_profile(args):
    """Small cases for ncu. dense: a V=16384 graph (826 MB of sketches,
    larger than L2) receives the first 8 insert batches of the dense stream,
    then one Connected batch (one grid-wide recovery). plain: the plain
    V=1024 stream, 20 Connected batches (one-cluster recoveries).
    rmat: a V=2^15 graph (1.9 GB of sketches) receives 6 R-MAT batches of
    2^20..2^22 edges (the batched workload's generator at 15 levels)."""
    import torch

    from paper_2509_14433_gb300 import cupc as C
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    if args.profile_case == "plain":  # recoveries of the plain V=1024 stream (one-cluster kernel)
        st, g = C.cupc_init(1024, SEED, None, None, stream)
        C.check(st)
        nq = 0
        for kind, *rest in WL.plain_stream(V=1024, seed=1):
            if kind == "update":
                e, o = rest
                C.check(C.cupc_update_batch(g, torch.from_numpy(e.reshape(-1)).cuda(), torch.from_numpy(o).cuda(),
                                            len(o), stream))
            else:
                pr = rest[0]
                out = torch.empty(len(pr), dtype=torch.uint8, device="cuda")
                C.check(C.cupc_query(g, torch.from_numpy(pr.reshape(-1)).cuda(), len(pr), out, stream))
                nq += 1
        C.check(C.cupc_sync(g, stream))
        C.cupc_destroy(g)
        print("apply-profile plain done", nq, "queries")
        return
    if args.profile_case == "rmat":
        V = 1 << 15
        s = WL.RmatStream(levels=15, seed=3, batch_lo=1 << 20, batch_hi=4 << 20, device="cuda")
        bl = [s.next_batch() for _ in range(6)]
        st, g = C.cupc_init(V, SEED, (0, 0, 0, 4 << 20), None, stream)
        C.check(st)
        for e, o in bl:
            C.check(C.cupc_update_batch(g, e.reshape(-1).contiguous(), o.contiguous(), len(o), stream))
        C.check(C.cupc_sync(g, stream))
        C.cupc_destroy(g)
        print("apply-profile rmat done", [len(o) for _, o in bl])
        return
    E, _ = make_dense_stream()
    n = 8 * BATCH
    E_d = torch.from_numpy(E[:n].reshape(-1)).cuda()
    ins_d = torch.ones(n, dtype=torch.int8, device="cuda")
    st, g = C.cupc_init(V_DENSE, SEED, None, None, stream)
    C.check(st)
    from paper_2509_14433_gb300 import autotune as AT
    AT.apply(g, V_DENSE, BATCH)  # the tuned apply setting of this batch size
    for i in range(0, n, BATCH):
        C.check(C.cupc_update_batch(g, E_d[2 * i:], ins_d[i:], BATCH, stream))
    pairs = torch.from_numpy(WL.uniform_pairs(V_DENSE, 1000, WL.rng(5)).reshape(-1)).cuda()
    out = torch.empty(1000, dtype=torch.uint8, device="cuda")
    C.check(C.cupc_query(g, pairs, 1000, out, stream))
    C.check(C.cupc_sync(g, stream))
    C.cupc_destroy(g)
    print("apply-profile done")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", default="bench", choices=["bench", "apply-profile", "paper-streams"])
    ap.add_argument("--kron", default="13,15,16", help="paper-streams: Kronecker graph sizes (log2 V)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cupc", choices=["cupc", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--profile-case", default="dense", choices=["dense", "rmat", "plain"])
    args = ap.parse_args()
    if args.mode == "apply-profile":
        run_apply_profile(args)
    elif args.mode == "paper-streams":
        run_paper_streams(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
