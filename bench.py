"""Throughput benchmark of the sketch-connectivity hot path on GB300.

Workload (one step = one whole job, inputs resident in HBM before timing):
  dense V=16384: all edges of an Erdos-Renyi G(V, 0.5) graph (~67.1M) inserted
  in a seeded random order in batches of 2^20, then a uniform random 10% of
  them deleted in batches of 2^20, then the spanning forest. Sketches (826 MB)
  and the edge stream (~600 MB) are larger than L2, so no flush is needed.
value = edge updates per second over the whole job (all ranks).

Also reported: the same job end to end through the C-ABI with pinned host
buffers (e2e), Connected-query latency p50/p99 on the plain V=1024 toggle
stream and right after a dense batch, the live roofline of the dominant
kernel (the sketch apply kernel) and the CPU oracle timed on a bounded sample.

--impl reference times the CPU oracle on the same workload (bounded sample
per step) and prints the same JSON line with "impl": "reference".
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
V_DENSE, P_DENSE, BATCH, SEED = 16384, 0.5, 1 << 20, 1
CPU_SAMPLE_BATCHES = 2
REF_SAMPLE_BATCHES = 1


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


def make_dense_stream():
    E, n_del, order = WL.dense_stream(V=V_DENSE, p=P_DENSE, batch=BATCH, delete_frac=0.1, seed=SEED)
    return E, E[order[:n_del]]


def workload_config(nE, nD):
    return {"workload": f"dense ER(V={V_DENSE}, p={P_DENSE}): {nE} inserts + {nD} deletes (10%) in batches of "
                        f"{BATCH}, then spanning forest",
            "V": V_DENSE, "batch": BATCH, "updates_per_step": nE + nD, "seed": SEED,
            "apply_tuning": "autotuned table (paper_2509_14433_gb300/tuning_gb300.json) when present",
            "l2": "inputs larger than L2 (sketches 826 MB, edge stream ~600 MB): no flush"}


def expected_touched_buckets(counts, L, C, D):
    """Expected distinct buckets an update batch touches, given the number of
    batch records n_w of each vertex: per vertex and layer, the deterministic
    bucket plus, per column, sum_d 1 - (1 - p_d)^n_w with p_d = 2^-(d+1)
    (the last row takes the tail 2^-(D-1)). Hash values are uniform, so the
    sum over ~10^6 independent columns is tight around this expectation."""
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
    functions and error/counter constants of common.cuh (its other
    declarations serve other kernels and the host)."""
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
    for m in re.finditer(r"^constexpr uint32_t k(?:ErrInval|DirectItem\w*|SmemRows\w*|\w*ItemRecords) = [^;]*;|^  GC_(?:ERR|NITEMS|NEXT_ITEM) = \d+",
                         com, re.M):
        h.update(m.group(0).encode())
    return h.hexdigest()


def apply_traffic(setting):
    """DRAM bytes per k_apply launch from the committed ncu summary; None
    when the kernel's source or its launch setting changed since the
    counters were taken."""
    tp = os.path.join(ROOT, "profiles", "k_apply_traffic.json")
    try:
        rec = json.load(open(tp))
    except (OSError, ValueError):
        return None
    if rec.get("source_md5") != apply_source_digest() or list(rec.get("setting", [])) != list(setting):
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


def oracle_sample(E, batches=CPU_SAMPLE_BATCHES, seed=SEED):
    """CPU oracle on a bounded sample: the first `batches` insert batches of
    the dense stream, one 1k-pair Connected batch (which runs the recovery),
    then the spanning forest (one thread). Returns the updates, the time of
    the whole sample and the time of the query batch."""
    import oracle as O
    n = batches * BATCH
    pairs = WL.uniform_pairs(V_DENSE, 1000, WL.rng(seed + 7), distinct=False)
    g = O.Graph(V_DENSE, seed)
    t = time.perf_counter()
    for i in range(0, n, BATCH):
        assert g.update(E[i:i + BATCH]) == O.OK
    tq = time.perf_counter()
    s, a = g.query(pairs)
    tq = time.perf_counter() - tq
    assert s in (O.OK, O.EINCOMPLETE)
    s, f = g.spanning_forest()
    dt = time.perf_counter() - t
    g.close()
    return n, dt, tq


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    E, D = make_dense_stream()
    for _ in range(args.warmup):
        oracle_sample(E, REF_SAMPLE_BATCHES)
    times, qtimes, n = [], [], 0
    for _ in range(args.steps):
        n, dt, tq = oracle_sample(E, REF_SAMPLE_BATCHES)
        times.append(dt)
        qtimes.append(tq)
    tot = sum(times)
    val = n * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": workload_config(len(E), len(D)),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {n} inserts of the dense stream + one 1k-pair Connected "
                                       "batch + spanning forest per step",
                             "query_batch_ms_p50": 1e3 * float(np.median(qtimes))},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch

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

    E, D = make_dense_stream()
    nE, nD = len(E), len(D)
    stream = torch.cuda.current_stream()
    E_d = torch.from_numpy(E.reshape(-1)).to(dev)
    D_d = torch.from_numpy(D.reshape(-1)).to(dev)
    ins_d = torch.ones(nE, dtype=torch.int8, device=dev)
    del_d = torch.full((nD,), -1, dtype=torch.int8, device=dev)
    forest_d = torch.empty(V_DENSE, dtype=torch.int64, device=dev)
    st, g = C.cupc_init(V_DENSE, SEED, None, None, stream)
    C.check(st, "cupc_init")
    from paper_2509_14433_gb300 import autotune as AT
    tuned = AT.apply(g, V_DENSE, BATCH)  # tuned apply setting for 2^20-edge batches, if the table has one
    tun = np.zeros(4, np.uint32)
    C.cupc_get_tuning(g, tun)
    apply_setting = [int(x) for x in tun[:3]]
    prm = np.zeros(4, np.uint32)
    C.cupc_get_params(g, prm)
    L, Cc, Dd, W = (int(x) for x in prm)

    def step_device():
        C.check(C.cupc_reset(g, stream))
        for i in range(0, nE, BATCH):
            C.check(C.cupc_update_batch(g, E_d[2 * i:], ins_d[i:], min(BATCH, nE - i), stream))
        for i in range(0, nD, BATCH):
            C.check(C.cupc_update_batch(g, D_d[2 * i:], del_d[i:], min(BATCH, nD - i), stream))
        st, nf = C.cupc_spanning_forest(g, forest_d, V_DENSE, stream)
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
    upd_per_step = nE + nD
    value = whole_job_rate(upd_per_step, args.steps, world, ms)
    assert C.cupc_sync(g, stream) == C.CUPC_OK

    # ---- e2e: the same job through the C-ABI with pinned host buffers
    E_h = torch.from_numpy(E.reshape(-1)).pin_memory()
    D_h = torch.from_numpy(D.reshape(-1)).pin_memory()
    ins_h = torch.ones(nE, dtype=torch.int8).pin_memory()
    del_h = torch.full((nD,), -1, dtype=torch.int8).pin_memory()
    forest_h = torch.empty(V_DENSE, dtype=torch.int64).pin_memory()

    def step_host():
        C.check(C.cupc_reset(g, stream))
        for i in range(0, nE, BATCH):
            C.check(C.cupc_update_batch(g, E_h.data_ptr() + 8 * i, ins_h.data_ptr() + i, min(BATCH, nE - i), stream))
        for i in range(0, nD, BATCH):
            C.check(C.cupc_update_batch(g, D_h.data_ptr() + 8 * i, del_h.data_ptr() + i, min(BATCH, nD - i), stream))
        st, nf = C.cupc_spanning_forest(g, forest_h, V_DENSE, stream)
        C.check(st, "spanning_forest", ok=(C.CUPC_OK, C.CUPC_EINCOMPLETE))
        return nf

    step_host()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(3, min(args.steps, 5))  # at least 3: one slow step must not set the number
    for _ in range(e2e_steps):
        nf_h = step_host()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s = max_over_ranks(e2e_s, dev)
    e2e_val = whole_job_rate(upd_per_step, e2e_steps, world, e2e_s * 1e3)
    assert nf_h == nf and torch.equal(forest_h[:nf], forest_d[:nf].cpu())

    # ---- Connected-query latency right after a dense update batch
    lat_dense = []
    pairs = WL.uniform_pairs(V_DENSE, 1000, WL.rng(77), distinct=False)
    p_d = torch.from_numpy(pairs.reshape(-1)).to(dev)
    q_out = torch.empty(1000, dtype=torch.uint8, device=dev)
    for k in range(12):
        i = (k % 6) * BATCH  # toggle one 2^20-edge batch, then ask
        C.check(C.cupc_update_batch(g, E_d[2 * i:], ins_d[i:], BATCH, stream))
        torch.cuda.synchronize()
        t = time.perf_counter()
        C.check(C.cupc_query(g, p_d, 1000, q_out, stream))
        torch.cuda.synchronize()
        lat_dense.append((time.perf_counter() - t) * 1e6)
    sweep = batch_latency_sweep(torch, C, g, D_d, ins_d, del_d, p_d, q_out, stream)
    C.cupc_destroy(g)
    del E_d, D_d, ins_d, del_d

    # ---- plain V=1024 toggle stream: updates/s and query latency
    plain = plain_stream_latency(torch, C, dev, stream)
    plain.update(plain_stream_latency(torch, C, dev, stream, inc=1))
    pstream = None if args.no_batching else paper_stream(torch, C, dev, stream)
    batching = None if args.no_batching else batching_compare(torch, C, dev, stream)
    serving = None if args.no_serving else serving_compare(torch, C, dev)

    # ---- roofline of the dominant kernel (sketch apply), measured live above
    counts_per_batch = []
    for i in range(0, nE, BATCH):
        counts_per_batch.append(np.bincount(E[i:i + BATCH].reshape(-1), minlength=V_DENSE))
    for i in range(0, nD, BATCH):
        counts_per_batch.append(np.bincount(D[i:i + BATCH].reshape(-1), minlength=V_DENSE))
    touched = [expected_touched_buckets(c, L, Cc, Dd) for c in counts_per_batch]
    apply_bytes_per_launch = 32.0 * float(np.mean(touched))
    sweep_bytes_per_launch = float(np.mean([dense_sweep_bytes(c, L, W) for c in counts_per_batch]))
    apply_launches = int(nl_prof[2])
    apply_ms = ms_prof[2] / max(1, apply_launches)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = apply_bytes_per_launch / (apply_ms * 1e-3) / 1e9
    traffic = apply_traffic(apply_setting)
    gpu_launches = int(nl_prof.sum())
    shares = {name: round(float(ms_prof[k]) / max(1e-9, float(ms_prof.sum())), 4)
              for k, name in enumerate(["validate", "group", "apply", "recover", "query", "sort"])}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n, dt, tq = oracle_sample(E)
        cpu = {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {n} inserts of the dense stream + one 1k-pair Connected batch + spanning "
                         "forest (single thread)",
               "query_batch_ms": 1e3 * tq}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": workload_config(nE, nD),
                "e2e": {"value": e2e_val, "unit": UNIT,
                        "h2d_bytes_per_step": int(9 * (nE + nD)), "d2h_bytes_per_step": int(8 * nf_h)},
                "gpu_launches": gpu_launches,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic,
                             "kernel": "k_apply", "algorithmic_bytes_per_launch": apply_bytes_per_launch,
                             "dense_sweep_bytes_per_launch": sweep_bytes_per_launch,
                             "edges_per_launch": BATCH, "avg_launch_ms": apply_ms,
                             "apply_setting": apply_setting,
                             "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)" if peaks else "fallback"},
                "kernel_time_share": shares,
                "batch_size_vs_query_latency": sweep,
                "paper_stream_shape": pstream,
                "query_latency_us": {"dense_after_batch_p50": statistics.median(lat_dense),
                                     "dense_after_batch_p99": float(np.percentile(lat_dense, 99)),
                                     **plain},
                "forest_edges": int(nf),
                "batching": batching,
                "serving": serving,
                "cpu_baseline": cpu, "clocks": clk}
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def batching_compare(torch, C, dev, stream, n_batches=48, rounds=30):
    """Batched vs one-batch-per-launch (device-resident inputs, CUDA events).

    uneven: R-MAT stream on V = 2^17 (a=.57, b=c=.19, d=.05, 20% deletes of
    present edges, batch sizes log-uniform in [1k, 4M]), the first n_batches
    batches: one cupc_update_batch per batch vs cupc_update_batches over the
    back-to-back batches. many_graphs: 64 graphs with V log-uniform in
    [2^10, 2^15], each receiving a 1k-edge batch per round: 64
    cupc_update_batch calls per round vs one cupc_batcher_update call (CUDA
    graph replay, and without the graph)."""
    from paper_2509_14433_gb300 import autotune as AT
    out = {}
    # -- uneven batches of one graph
    s = WL.RmatStream(levels=17, seed=3, device=dev)
    bl = [s.next_batch() for _ in range(n_batches)]
    sizes = [len(b[1]) for b in bl]
    E = torch.cat([b[0].reshape(-1) for b in bl]).contiguous()
    O = torch.cat([b[1] for b in bl]).contiguous()
    offs = np.cumsum([0] + sizes).astype(np.uint64)
    del bl, s
    torch.cuda.empty_cache()
    V = 1 << 17
    st, g = C.cupc_init(V, 1, (0, 0, 0, 4 << 20), None, stream)
    C.check(st)
    AT.apply_buckets(g, V)  # each batch with the setting of its size

    def plain():
        for i in range(n_batches):
            C.check(C.cupc_update_batch(g, E.data_ptr() + 8 * int(offs[i]), O.data_ptr() + int(offs[i]),
                                        sizes[i], stream))

    def coalesced():
        C.check(C.cupc_update_batches(g, E, O, offs, n_batches, stream))

    res = {}
    for name, fn in (("one_batch_per_launch", plain), ("coalesced", coalesced)):
        C.cupc_reset(g, stream)
        fn()
        C.cupc_reset(g, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = int(offs[-1]) / (e0.elapsed_time(e1) / 1e3)
    C.cupc_destroy(g)
    del E, O
    torch.cuda.empty_cache()
    out["uneven_rmat_v131072"] = {"updates": int(offs[-1]), "batches": n_batches,
                                  "batch_min": int(min(sizes)), "batch_max": int(max(sizes)),
                                  "updates_per_s": res}
    # -- many graphs, one small batch each per round
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
    out["many_graphs_64x1k"] = {"graphs": len(graphs), "V_min": min(Vs), "V_max": max(Vs), "rounds": rounds,
                                "updates_per_s": res}
    return out


def serving_compare(torch, C, dev, n_graphs=64, upd_range=(5e4, 5e5), seed=5):
    """Serving workload (64 graphs, V log-uniform in [2^10, 2^15], ER(p)
    insert/delete streams, p ~ U[0.1, 0.9], batches log-uniform in [1k, 1M],
    a 1k-pair Connected batch after every 100k updates of a graph; each
    graph's stream has log-uniform[upd_range] updates). All requests arrive
    at once, round-robin over graphs. served: cupc_server (continuous
    batching, multi-graph launches, overlapped query streams) with no memory
    cap and with a cap of 25% of the graphs' total workspace (graphs wait for
    admission and close when done); plain: one thread, one request at a time
    through cupc_update_batch / cupc_query, each finished before the next.
    Latency = arrival to completion; updates/s = all updates / makespan."""
    streams = WL.serving_streams(n_graphs=n_graphs, upd_range=upd_range, seed=seed)
    order = WL.round_robin(streams)
    total_upd = sum(st[3] for st in streams)
    maxb = 1 << 20
    ws = [C.cupc_workspace_bytes(st[0], (0, 0, 0, maxb)) for st in streams]
    out = {"graphs": n_graphs, "updates": int(total_upd), "requests": len(order),
           "queries": sum(1 for _, s_ in order if s_[0] == "query")}

    def served(cap_bytes):
        st, srv = C.cupc_server_create(int(cap_bytes), n_graphs, maxb, 4)
        C.check(st)
        try:
            ids = [C.cupc_server_open(srv, s_[0], s_[1])[1] for s_ in streams]
            last = {}
            for k, (i, _) in enumerate(order):
                last[i] = k
            keep, qt, ut = [], [], []
            t0 = time.perf_counter()
            for k, (i, stp) in enumerate(order):
                if stp[0] == "update":
                    e = np.ascontiguousarray(stp[1], np.uint32)
                    o = np.ascontiguousarray(stp[2], np.int8)
                    keep.append((e, o))
                    r, t = C.cupc_server_update(srv, ids[i], e, o, len(o))
                    ut.append(t)
                else:
                    p = np.ascontiguousarray(stp[1], np.uint32)
                    ans = np.zeros(len(p), np.uint8)
                    keep.append((p, ans))
                    r, t = C.cupc_server_query(srv, ids[i], p, len(p), ans)
                    qt.append(t)
                C.check(r, "submit")
                if k == last[i]:
                    ut.append(C.cupc_server_close(srv, ids[i])[1])
            lat = []
            for t in ut:
                C.check(C.cupc_server_wait(srv, t, 600000)[0], "update")
            for t in qt:
                r, l_us = C.cupc_server_wait(srv, t, 600000)
                C.check(r, "query")
                lat.append(l_us)
            span = time.perf_counter() - t0
            stats = np.zeros(8, np.uint64)
            C.cupc_server_stats(srv, stats)
            return {"updates_per_s": total_upd / span, "query_p50_us": float(np.percentile(lat, 50)),
                    "query_p99_us": float(np.percentile(lat, 99)), "makespan_s": span,
                    "update_launches": int(stats[2]), "update_requests": int(stats[3]),
                    "admission_waits": int(stats[5])}
        finally:
            C.cupc_server_destroy(srv)

    out["served_no_cap"] = served(sum(ws) * 1.02 + (256 << 20))
    out["served_cap_25pct"] = served(0.25 * sum(ws))
    # plain: one request at a time on the caller's thread
    graphs = []
    for s_ in streams:
        r, g = C.cupc_init(s_[0], s_[1], (0, 0, 0, maxb), None, None)
        C.check(r)
        graphs.append(g)
    try:
        lat = []
        t0 = time.perf_counter()
        for i, stp in order:
            if stp[0] == "update":
                e = np.ascontiguousarray(stp[1], np.uint32)
                o = np.ascontiguousarray(stp[2], np.int8)
                C.check(C.cupc_update_batch(graphs[i], e, o, len(o), None))
                torch.cuda.synchronize()
            else:
                p = np.ascontiguousarray(stp[1], np.uint32)
                ans = np.zeros(len(p), np.uint8)
                C.check(C.cupc_query(graphs[i], p, len(p), ans, None))
                lat.append((time.perf_counter() - t0) * 1e6)
        span = time.perf_counter() - t0
        out["one_request_at_a_time"] = {"updates_per_s": total_upd / span,
                                        "query_p50_us": float(np.percentile(lat, 50)),
                                        "query_p99_us": float(np.percentile(lat, 99)), "makespan_s": span}
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
    the recoveries it ran, and the latency of every 25th burst (its update
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
            lat = run(bursts, sample_every=25)
            out[mode] = {"updates_per_s": len(E) / dt, "queries_per_s": n_q / dt, "recoveries": nrec,
                         "burst_latency_p50_us": statistics.median(lat),
                         "burst_latency_p99_us": float(np.percentile(lat, 99))}
        res[shape] = out
        del E_d, ops_d, P_d, out_d
    C.check(C.cupc_sync(g, stream), "paper stream", ok=(C.CUPC_OK, C.CUPC_EINCOMPLETE))
    C.cupc_destroy(g)
    return res


def plain_stream_latency(torch, C, dev, stream, inc=0):
    """V=1024 ER(0.5) start graph + 200k toggles, a 1k-pair Connected batch
    every 10k updates: updates/s over the toggles, query latency p50/p99
    (host submit -> answers ready, recovery included). inc: incremental
    labels (the stream is valid: a toggle inserts an absent edge or deletes
    a present one)."""
    V = 1024
    steps = WL.plain_stream(V=V, seed=1)
    st, g = C.cupc_init(V, 1, None, None, stream)
    C.check(st)
    C.check(C.cupc_set_incremental(g, inc, stream))
    dsteps = []
    for s in steps:
        if s[0] == "update":
            dsteps.append(("u", torch.from_numpy(s[1].reshape(-1)).to(dev), torch.from_numpy(s[2]).to(dev), len(s[2])))
        else:
            dsteps.append(("q", torch.from_numpy(s[1].reshape(-1)).to(dev), torch.empty(len(s[1]), dtype=torch.uint8,
                                                                                       device=dev), len(s[1])))
    lat, upd_t, n_upd = [], 0.0, 0
    for rep in range(3):
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
    sfx = "_incremental" if inc else ""
    return {f"plain_v1024{sfx}_p50": statistics.median(lat), f"plain_v1024{sfx}_p99": float(np.percentile(lat, 99)),
            f"plain_v1024{sfx}_toggle_updates_per_s": n_upd / upd_t, f"plain_v1024{sfx}_queries": len(lat)}


def batch_latency_sweep(torch, C, g, D_d, ins_d, del_d, p_d, q_out, stream):
    """Update batch size against the latency of the next Connected query
    batch (the trade-off the paper's update buffering makes): for each size
    b, insert then delete the first b of the deleted edges (absent, then
    present: a valid stream) and ask 1k pairs after each batch. Latency =
    host submit of the batch to the query's answer, recovery included."""
    out = {}
    for b in (1 << 10, 1 << 14, 1 << 17, 1 << 20, 1 << 22):
        upd, lat = [], []
        for k in range(9):  # the first pass warms up
            ops = ins_d if k % 2 == 0 else del_d
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            C.check(C.cupc_update_batch(g, D_d, ops, b, stream))
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            C.check(C.cupc_query(g, p_d, 1000, q_out, stream))
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            if k:
                upd.append(t1 - t0)
                lat.append((t2 - t0) * 1e6)
        C.check(C.cupc_update_batch(g, D_d, del_d, b, stream))  # the last pass inserted: leave the graph as it was
        out[str(b)] = {"updates_per_s": b / statistics.median(upd), "query_p50_us": statistics.median(lat),
                       "query_p99_us": float(np.percentile(lat, 99))}
    return out


def run_apply_profile(args):
    """Small cases for ncu. dense: a V=16384 graph (826 MB of sketches,
    larger than L2) receives the first 8 insert batches of the dense stream.
    rmat: a V=2^15 graph (1.9 GB of sketches) receives 6 R-MAT batches of
    2^20..2^22 edges (the batched workload's generator at 15 levels)."""
    import torch

    from paper_2509_14433_gb300 import cupc as C
    torch.cuda.set_device(0)
    if args.profile_case == "rmat":
        V = 1 << 15
        s = WL.RmatStream(levels=15, seed=3, batch_lo=1 << 20, batch_hi=4 << 20, device="cuda")
        bl = [s.next_batch() for _ in range(6)]
        stream = torch.cuda.current_stream()
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
    stream = torch.cuda.current_stream()
    st, g = C.cupc_init(V_DENSE, SEED, None, None, stream)
    C.check(st)
    from paper_2509_14433_gb300 import autotune as AT
    AT.apply(g, V_DENSE, BATCH)  # the bench's apply setting
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
    ap.add_argument("--mode", default="bench", choices=["bench", "apply-profile"])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cupc", choices=["cupc", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--profile-case", default="dense", choices=["dense", "rmat"])
    args = ap.parse_args()
    if args.mode == "apply-profile":
        run_apply_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
