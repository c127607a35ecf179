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


def make_dense_stream():
    E, n_del, order = WL.dense_stream(V=V_DENSE, p=P_DENSE, batch=BATCH, delete_frac=0.1, seed=SEED)
    return E, E[order[:n_del]]


def workload_config(nE, nD):
    return {"workload": f"dense ER(V={V_DENSE}, p={P_DENSE}): {nE} inserts + {nD} deletes (10%) in batches of "
                        f"{BATCH}, then spanning forest",
            "V": V_DENSE, "batch": BATCH, "updates_per_step": nE + nD, "seed": SEED,
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


def apply_traffic():
    """DRAM bytes per k_apply launch from the committed ncu summary, scaled
    to a 2^20-edge batch; None when the kernel source changed since the
    counters were taken."""
    import hashlib
    tp = os.path.join(ROOT, "profiles", "k_apply_traffic.json")
    src = os.path.join(ROOT, "paper_2509_14433_gb300", "csrc", "update.cu")
    try:
        rec = json.load(open(tp))
        md5 = hashlib.md5(open(src, "rb").read()).hexdigest()
    except (OSError, ValueError):
        return None
    if rec.get("update_cu_md5") != md5:
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
    the dense stream, then the spanning forest (one thread)."""
    import oracle as O
    n = batches * BATCH
    g = O.Graph(V_DENSE, seed)
    t = time.perf_counter()
    for i in range(0, n, BATCH):
        assert g.update(E[i:i + BATCH]) == O.OK
    s, f = g.spanning_forest()
    dt = time.perf_counter() - t
    g.close()
    return n, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    E, D = make_dense_stream()
    for _ in range(args.warmup):
        oracle_sample(E, REF_SAMPLE_BATCHES)
    times, n = [], 0
    for _ in range(args.steps):
        n, dt = oracle_sample(E, REF_SAMPLE_BATCHES)
        times.append(dt)
    tot = sum(times)
    val = n * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": workload_config(len(E), len(D)),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {n} inserts of the dense stream + spanning forest per step"},
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
    if pg is not None:
        t = torch.tensor([ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    upd_per_step = nE + nD
    value = upd_per_step * args.steps * world / (ms / 1e3)
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
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        nf_h = step_host()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_val = upd_per_step * e2e_steps * world / e2e_s
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
    C.cupc_destroy(g)
    del E_d, D_d, ins_d, del_d

    # ---- plain V=1024 toggle stream: updates/s and query latency
    plain = plain_stream_latency(torch, C, dev, stream)

    # ---- roofline of the dominant kernel (sketch apply), measured live above
    counts_per_batch = []
    for i in range(0, nE, BATCH):
        counts_per_batch.append(np.bincount(E[i:i + BATCH].reshape(-1), minlength=V_DENSE))
    for i in range(0, nD, BATCH):
        counts_per_batch.append(np.bincount(D[i:i + BATCH].reshape(-1), minlength=V_DENSE))
    touched = [expected_touched_buckets(c, L, Cc, Dd) for c in counts_per_batch]
    apply_bytes_per_launch = 32.0 * float(np.mean(touched))
    apply_launches = int(nl_prof[2])
    apply_ms = ms_prof[2] / max(1, apply_launches)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = apply_bytes_per_launch / (apply_ms * 1e-3) / 1e9
    traffic = apply_traffic()
    gpu_launches = int(nl_prof.sum())
    shares = {name: round(float(ms_prof[k]) / max(1e-9, float(ms_prof.sum())), 4)
              for k, name in enumerate(["validate", "group", "apply", "recover", "query", "sort"])}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n, dt = oracle_sample(E)
        cpu = {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {n} inserts of the dense stream + spanning forest (single thread)"}

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
                             "edges_per_launch": BATCH, "avg_launch_ms": apply_ms,
                             "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)" if peaks else "fallback"},
                "kernel_time_share": shares,
                "query_latency_us": {"dense_after_batch_p50": statistics.median(lat_dense),
                                     "dense_after_batch_p99": float(np.percentile(lat_dense, 99)),
                                     **plain},
                "forest_edges": int(nf),
                "cpu_baseline": cpu, "clocks": clk}
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def plain_stream_latency(torch, C, dev, stream):
    """V=1024 ER(0.5) start graph + 200k toggles, a 1k-pair Connected batch
    every 10k updates: updates/s over the toggles, query latency p50/p99
    (host submit -> answers ready, recovery included)."""
    V = 1024
    steps = WL.plain_stream(V=V, seed=1)
    st, g = C.cupc_init(V, 1, None, None, stream)
    C.check(st)
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
    return {"plain_v1024_p50": statistics.median(lat), "plain_v1024_p99": float(np.percentile(lat, 99)),
            "plain_v1024_toggle_updates_per_s": n_upd / upd_t, "plain_v1024_queries": len(lat)}


def run_apply_profile(args):
    """Small case for ncu: a V=16384 graph (826 MB of sketches, larger than
    L2) receives the first 8 insert batches of the dense stream."""
    import torch

    from paper_2509_14433_gb300 import cupc as C
    torch.cuda.set_device(0)
    E, _ = make_dense_stream()
    n = 8 * BATCH
    E_d = torch.from_numpy(E[:n].reshape(-1)).cuda()
    ins_d = torch.ones(n, dtype=torch.int8, device="cuda")
    stream = torch.cuda.current_stream()
    st, g = C.cupc_init(V_DENSE, SEED, None, None, stream)
    C.check(st)
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
    args = ap.parse_args()
    if args.mode == "apply-profile":
        run_apply_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
