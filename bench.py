#!/usr/bin/env python
"""Benchmark of the hybrid connected-components route on one GB300 per rank.

Workload (default): R-MAT scale 24, edge factor 16 (n = 16,777,216 vertices,
m = 268,435,456 undirected int32 pairs, a=0.57 b=c=0.19, ids permuted,
duplicates and self-loops kept), generated from a fixed seed. One step is
one cc_labels call (degree pass -> K-S prediction -> BFS if chosen -> SV
iterations -> labels) with the edges already resident in HBM; the metric is
m / device time (CC edges/s). The 2.15 GB edge list is larger than L2, so no
flush is done between steps.

Extra keys: roofline of the dominant kernel (algorithmic bytes per launch /
its average event-timed duration, against the measured HBM copy bandwidth),
l2_roofline (the same kernel's scattered 4-byte accesses per second against
the L2 random-op rate measured in the same run: the degree and hook passes
are bound by that rate, not by HBM),
e2e (the same metric with pinned host buffers and both copies inside the
timed region), cpu_baseline (the CPU oracle on a bounded prefix sample),
clocks sampled during the timed region, and route_compare (the forced BFS
and forced SV routes on the same graph).

`--impl reference` times the CPU oracle (sequential union-find) instead.
Under torchrun with N > 1 ranks every rank runs an independent replica
(the single-graph path does not shard); value = all ranks' pairs / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CC edges/s (m / device time to exact labels)"
UNIT = "edges/s"
WORKLOADS = {
    "rmat24": dict(kind="rmat", scale=24, edge_factor=16, seed=1),
    "rmat20": dict(kind="rmat", scale=20, edge_factor=16, seed=1),
    "rmat22": dict(kind="rmat", scale=22, edge_factor=16, seed=1),
    "planted": dict(kind="planted", seed=1),
    "grid_chains": dict(kind="grid_chains", seed=1, W=8192, nchains=10_000_000),
    "batch4096": dict(kind="batch", seed=1, G=4096, nmin=1000, nmax=1_000_000),
    "batch512": dict(kind="batch", seed=1, G=512, nmin=1000, nmax=1_000_000),
}
KERNEL_FILES = ["cc_common.cuh", "ks_math.cuh", "k_degree.cu", "k_sv.cu", "k_bfs.cu", "k_bucket.cu", "k_batch_route.cu",
                "cc_api.cu"]


def make_graph(name: str):
    import graphgen as gg

    w = dict(WORKLOADS[name])
    kind = w.pop("kind")
    if kind == "rmat":
        return gg.rmat(**w)
    if kind == "planted":
        return gg.planted(**w)
    return gg.grid_chains(**w)


def workload_config(name: str, g) -> dict:
    w = WORKLOADS[name]
    cfg = {"workload": name, "n": int(g.n), "m": int(g.m), "id_bytes": int(g.id_bytes),
           "l2": "inputs larger than L2 (no flush)" if g.m * 2 * g.id_bytes > 129e6 else "L2-resident inputs"}
    if w["kind"] == "rmat":
        cfg.update({"graph": f"R-MAT scale {w['scale']} edge factor {w['edge_factor']} (a=0.57,b=0.19,c=0.19)",
                    "seed": w["seed"]})
    else:
        cfg.update({"graph": g.name})
    return cfg


def alg_bytes(cls: str, st: dict, w: int) -> float:
    """Algorithmic bytes one call moves in a kernel class (element-size accesses)."""
    n, m = st["n"], st["m"]
    act, hooks = st["m_active"], st["sv_hooks"]
    if cls == "degree":
        return 2 * w * m + 4 * n
    if cls == "hist":
        return 4 * n
    if cls == "parent_init":
        return 4 * n
    if cls == "finalize":
        return 4 * n + w * n
    if cls == "sv_first":
        k = st.get("sv_sample_stride", 1) or 1
        if k > 1:  # front end: two passes over m/k pairs (pre-check; two gathers and a pre-check)
            return (4 * w + 16) * m / k
        return 2 * w * m + 4 * m
    if cls == "sv_gather_input":
        # read pairs, gather both parents, atomicMin per surviving pair, write survivors
        kept = act[2] if len(act) > 2 else 0
        return 2 * w * m + 8 * m + 4 * kept + 8 * kept
    if cls == "sv_gather_list":
        tot = 0
        for i in range(2, len(act)):
            mi = act[i]
            kept = act[i + 1] if i + 1 < len(act) else 0
            tot += 16 * mi + 12 * kept
        return tot
    if cls == "sv_shortcut":
        return 12 * sum(hooks)
    if cls == "csr":
        return 2 * w * m + 16 * m
    if cls in ("bfs_bottomup", "bfs_topdown"):
        return 4 * st["bfs_edges_inspected"] / 2 + n / 8 * 3
    return 0.0


def l2_ops(cls: str, st: dict) -> tuple[float, str]:
    """Scattered 4-byte accesses to L2-resident arrays one call makes in a
    kernel class, and the probe rate that bounds them. A lower bound: the
    hook atomics that follow a passing pre-check are not counted."""
    n, m = st["n"], st["m"]
    act = st["m_active"]
    if cls == "degree":
        return 2.0 * m, "red_add"            # one increment per pair endpoint
    if cls == "sv_first":
        k = st.get("sv_sample_stride", 1) or 1
        if k > 1:  # front end on m/k pairs: a pre-check, then two gathers and a pre-check
            return 4.0 * m / k, "gather"
        if 2 * m < 4 * n:  # sparse graphs: an atomicMin per pair, no pre-check read
            return 1.0 * m, "red_min"
        return 1.0 * m, "gather"             # pre-check read of parent[max(u, v)]
    if cls == "sv_gather_input":
        kept = act[2] if len(act) > 2 else 0
        return 2.0 * m + kept, "gather"      # both parents, then the pre-check of the pairs still crossing
    if cls == "sv_gather_list":
        tot = 0.0
        for i in range(2, len(act)):
            tot += 2.0 * act[i] + (act[i + 1] if i + 1 < len(act) else 0)
        return tot, "gather"
    if cls == "finalize":
        return 1.0 * n, "gather"
    return 0.0, "gather"


def sources_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_FILES:
        with open(os.path.join(ROOT, "paper_1607_06156_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_cls: str, workload: str):
    """DRAM bytes per launch of a kernel class from the committed ncu summary,
    if it matches the current sources (None otherwise)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    if d.get("sources_hash") != sources_hash():
        return None
    return d.get("traffic_per_call", {}).get(workload, {}).get(kernel_cls)


def kernel_class(name: str):
    """Kernel class (the engine's profiling scopes) of a kernel name in an ncu list.

    An SV pass is classed by its id type and mode: modes 0, 4 (the first pass
    over the caller's pairs, with or without the pre-check) and 1 (the first
    pass after the BFS, over the pairs or the list) are the first pass; mode 2
    is a gather pass, over the caller's pairs (int / long ids) or over the
    compacted list (unsigned int); mode 3 belongs to the host-input chunks."""
    sv = re.search(r"k_sv_pass<(int|long|unsigned int), (\d)", name)
    if sv:
        ids, mode = sv.group(1), int(sv.group(2))
        if mode in (0, 1, 4):
            return "sv_first"
        if mode == 2:
            return "sv_gather_list" if ids == "unsigned int" else "sv_gather_input"
        return None
    table = [("k_degree_hubs", "degree"), ("k_hub_", "degree"), ("k_degree<", "degree"), ("k_hist", "hist"),
             ("k_distinct", "ks"), ("k_ks_", "ks"), ("k_parent_init", "parent_init"), ("k_sv_sample", "sv_first"),
             ("k_shortcut_all", "sv_shortcut"), ("k_sv_shortcut", "sv_shortcut"), ("k_finalize", "finalize")]
    for key, cls in table:
        if key in name:
            return cls
    return None


def ncu_summary(csv_path: str, workload: str, scale_to: dict, command: str) -> dict:
    """DRAM bytes per cc_labels call of each kernel class from an ncu --csv
    capture of gpu__time_duration.sum, dram__bytes_read.sum and
    dram__bytes_write.sum: the class's bytes over all captured launches
    divided by the calls captured (the histogram kernel runs once per call
    on the heuristic route). The roofline divides it by the class's timed
    launches per call, like the algorithmic bytes. `scale_to` maps another
    workload to the ratio of its pairs to this one's (the streamed pairs
    dominate the traffic)."""
    import csv

    rows = list(csv.reader(open(csv_path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hi]
    ki, idi, mi, vi = h.index("Kernel Name"), h.index("ID"), h.index("Metric Name"), h.index("Metric Value")
    launches = {}
    for r in rows[hi + 1:]:
        if len(r) <= vi:
            continue
        d = launches.setdefault(int(r[idi]), {"name": r[ki]})
        d[r[mi]] = float(r[vi].replace(",", ""))
    tot, cnt = {}, {}
    for L in launches.values():
        cls = kernel_class(L["name"])
        if cls is None:
            continue
        tot[cls] = tot.get(cls, 0.0) + L.get("dram__bytes_read.sum", 0.0) + L.get("dram__bytes_write.sum", 0.0)
        cnt[cls] = cnt.get(cls, 0) + 1
    calls = cnt.get("hist", 0)
    if calls <= 0:
        raise SystemExit("no histogram launches in the capture: cannot count the calls")
    per = {k: tot[k] / calls for k in tot}
    out = {"sources_hash": sources_hash(), "command": command, "launches": cnt, "calls": calls,
           "note": f"dram__bytes_read.sum + dram__bytes_write.sum per cc_labels call and kernel class, captured on "
                   f"{workload}" + "".join(f"; {w}: scaled by the pair ratio x{f:g}" for w, f in scale_to.items()),
           "traffic_per_call": {workload: per}}
    for w, f in scale_to.items():
        out["traffic_per_call"][w] = {k: v * f for k, v in per.items()}
    return out


class ClockSampler:
    """nvidia-smi clocks/throttle sampling in the background (200 ms period)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None
        self.t_start = self.t_end = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark(self, which: str):
        setattr(self, "t_" + which, time.time())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip().lower() == "active"})
        # under load: samples at or above half the maximum clock seen
        load = [x for x in sm if sm and x >= 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(load)) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def cpu_oracle_rate(edges: np.ndarray, n: int, budget_pairs: int) -> tuple[float, int, float]:
    """The oracle's union-find on the first `budget_pairs` pairs (full n); pairs/s, pairs, seconds."""
    import oracle

    k = min(budget_pairs, edges.shape[0])
    sample = np.ascontiguousarray(edges[:k])
    t = time.perf_counter()
    oracle.labels_uf(sample, n)
    dt = time.perf_counter() - t
    return k / dt, k, dt


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time (every rank gets it); `dist` None = one rank."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, m: int, steps: int, ms_total: float) -> float:
    """Whole-job pairs/s: every rank labels its own replica of the m pairs per step."""
    return world * m * steps / (ms_total / 1e3)


def run_reference(args, world: int, rank: int):
    if rank != 0:
        return 0
    g = make_graph(args.workload)
    sample = args.ref_pairs
    cfg = workload_config(args.workload, g)
    for _ in range(args.warmup):
        cpu_oracle_rate(g.edges, g.n, sample)
    times = []
    for _ in range(args.steps):
        _, k, dt = cpu_oracle_rate(g.edges, g.n, sample)
        times.append(dt)
    tot = sum(times)
    value = k * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {k} of {g.m} pairs of the same graph, full n, sequential union-find"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args, world: int, rank: int, local: int) -> int:
    """Batched form: one cc_labels_batched call per step over G graphs, against
    a loop of per-graph cc_labels calls on the same GPU (labels compared).
    With N ranks the batch holds G x N graphs and every rank labels its own
    longest-processing-time-first shard of them (about G graphs), with no
    collective in the data path; the value is all pairs / the slowest rank."""
    import torch

    import graphgen as gg
    import paper_1607_06156_gb300 as cc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    w = dict(WORKLOADS[args.workload])
    w.pop("kind")
    if world > 1:
        from paper_1607_06156_gb300.sharding import graph_cost, lpt_shards

        w["G"] = w["G"] * world
        ng_all, mg_all = gg.batch_sizes(seed=w["seed"], G=w["G"], nmin=w["nmin"], nmax=w["nmax"])
        shard = lpt_shards(graph_cost(ng_all, mg_all), world)[rank]
        b = gg.batch(**w, graphs=shard)
        m_job = int(mg_all.sum())
    else:
        b = gg.batch(**w)
        m_job = int(b.edge_offsets[-1])
    m, n = int(b.edge_offsets[-1]), int(b.vertex_offsets[-1])
    edges_d = torch.from_numpy(b.edges).to(dev)
    eo_h = torch.from_numpy(b.edge_offsets)
    vo_h = torch.from_numpy(b.vertex_offsets)
    eo_d, vo_d = eo_h.to(dev), vo_h.to(dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    eng = cc.Engine(id_bytes=4, device=local, profile=0)  # SV loop as one captured graph
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 1)):
        eng.labels_batched_dev(edges_d, eo_d, vo_d, eo_h, vo_h, out)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    e0.record(stream)
    for _ in range(args.steps):
        eng.labels_batched_dev(edges_d, eo_d, vo_d, eo_h, vo_h, out)
        launches += eng.stats()["launches"]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    # per-kernel CUDA events in a second region (profiling on: host-driven loop)
    eng.set_options(profile=1)
    eng.labels_batched_dev(edges_d, eo_d, vo_d, eo_h, vo_h, out)
    kms, kla = {}, {}
    for _ in range(args.steps):
        eng.labels_batched_dev(edges_d, eo_d, vo_d, eo_h, vo_h, out)
        st = eng.stats()
        for k, v in st["kernel_ms"].items():
            kms[k] = kms.get(k, 0.0) + v
            kla[k] = kla.get(k, 0) + st["kernel_launches"][k]
    clocks = sampler.stop() if sampler else None
    eng.set_options(profile=0)
    if world > 1:  # the shards ran; rank 0 reports the job
        if rank == 0:
            line = {"metric": METRIC + " [batched form]", "value": m_job / (ms / 1e3), "unit": UNIT,
                    "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                    "data": "synthetic",
                    "config": {"workload": args.workload, "graphs": w["G"], "m": m_job,
                               "parallelism": f"graph shards (longest processing time first) x{world}, "
                                              "no collective",
                               "graph": "log-uniform n_g in [1K, 1M], cycling R-MAT ef 8 / grid p=0.55 / "
                                        "chain forest", "l2": "inputs larger than L2 (no flush)"},
                    "rank0_shard": {"graphs": int(b.G), "m": m, "n": n}, "gpu_launches": launches,
                    "clocks": clocks}
            print(json.dumps(line), flush=True)
        eng.close()
        dist.barrier()
        dist.destroy_process_group()
        return 0
    # the same graphs one cc_labels call at a time (each graph in its own aligned buffer)
    per = [edges_d[b.edge_offsets[g]:b.edge_offsets[g + 1]].clone() for g in range(b.G)]
    outs = [torch.empty(int(b.vertex_offsets[g + 1] - b.vertex_offsets[g]), dtype=torch.int32, device=dev)
            for g in range(b.G)]
    one = cc.Engine(id_bytes=4, device=local)
    for g in range(b.G):
        one.labels(per[g], outs[g].numel(), out=outs[g])
    torch.cuda.synchronize(dev)
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    loops = max(1, min(args.steps, 2))
    a.record(stream)
    for _ in range(loops):
        for g in range(b.G):
            one.labels(per[g], outs[g].numel(), out=outs[g])
    c.record(stream)
    torch.cuda.synchronize(dev)
    ms_loop = a.elapsed_time(c) / loops
    same = all(torch.equal(outs[g], out[b.vertex_offsets[g]:b.vertex_offsets[g + 1]]) for g in range(b.G))
    if not same:
        raise SystemExit("batched labels differ from the per-graph calls")
    dom = max(kms, key=lambda k: kms[k])
    kernels = {k: {"ms_per_step": kms[k] / args.steps, "launches_per_step": kla[k] / args.steps} for k in kms if kla[k]}
    # the same batch with the route prediction skipped (every graph SV only)
    sv = cc.Engine(id_bytes=4, device=local, route="sv")
    sv.labels_batched_dev(edges_d, eo_d, vo_d, eo_h, vo_h, out)
    torch.cuda.synchronize(dev)
    a.record(stream)
    for _ in range(loops):
        sv.labels_batched_dev(edges_d, eo_d, vo_d, eo_h, vo_h, out)
    c.record(stream)
    torch.cuda.synchronize(dev)
    ms_sv = a.elapsed_time(c) / loops
    sv.close()
    line = {"metric": METRIC + " [batched form]", "value": m / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "graphs": b.G, "n": n, "m": m,
                       "graph": "log-uniform n_g in [1K, 1M], cycling R-MAT ef 8 / grid p=0.55 / chain forest",
                       "l2": "inputs larger than L2 (no flush)"},
            "vs_per_graph_loop": {"value": m / (ms_loop / 1e3), "ms_per_step": ms_loop,
                                  "speedup": ms_loop / ms, "labels_identical": same},
            "sv_only_batched": {"value": m / (ms_sv / 1e3), "ms_per_step": ms_sv,
                                "note": "route prediction skipped (CC_ROUTE_FORCE_SV)"},
            "route_policy": "auto (a K-S fit per graph)", "graphs_routed_bfs": st["route"],
            "schedule": {"unroll": st["batch_unroll"], "grid_mult": st["batch_grid_mult"]},
            "dominant_kernel": dom, "kernels": kernels, "gpu_launches": launches, "clocks": clocks,
            "sv_iters": st["sv_iters"], "m_active": st["m_active"]}
    print(json.dumps(line), flush=True)
    eng.close()
    one.close()
    return 0


def check_labels(torch, edges_d, lab, n):
    """Cheap device-side invariants of min-id labels (outside the timed region)."""
    l = lab.long()
    e = edges_d.long()
    ok = bool((l[e[:, 0]] == l[e[:, 1]]).all())
    v = torch.arange(n, device=lab.device)
    ok = ok and bool((l <= v).all()) and bool((l[l] == l).all())
    return ok


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat24", choices=sorted(WORKLOADS))
    ap.add_argument("--route", default="auto", choices=["auto", "sv", "bfs"])
    ap.add_argument("--no-compare", action="store_true", help="skip the forced-route comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--ref-pairs", type=int, default=1 << 24, help="pairs per step of the CPU oracle")
    ap.add_argument("--cpu-pairs", type=int, default=1 << 25, help="pairs in the cpu_baseline sample")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer timing")
    ap.add_argument("--no-l2", action="store_true", help="skip the live L2 rate probe (no l2_roofline)")
    ap.add_argument("--ncu-summary", metavar="CSV",
                    help="print the DRAM traffic summary of an ncu --csv capture of --workload and exit")
    ap.add_argument("--ncu-command", default="", help="the command line of that capture (recorded)")
    args = ap.parse_args()
    if args.ncu_summary:
        w = WORKLOADS[args.workload]
        scale = {}
        if w["kind"] == "rmat" and w["scale"] < 24:
            scale["rmat24"] = float(2 ** (24 - w["scale"]))
        print(json.dumps(ncu_summary(args.ncu_summary, args.workload, scale, args.ncu_command), indent=1))
        return 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if WORKLOADS[args.workload]["kind"] == "batch":
        return run_batch(args, world, rank, local)

    import torch

    import paper_1607_06156_gb300 as cc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    g = make_graph(args.workload)
    cfg = workload_config(args.workload, g)
    w = g.id_bytes
    n, m = g.n, g.m
    edges_d = torch.from_numpy(g.edges).to(dev)
    lab = torch.empty(n, dtype=edges_d.dtype, device=dev)
    # the product path: per-kernel profiling off, so the SV loop runs as one
    # captured CUDA graph with a device-driven WHILE node
    eng = cc.Engine(id_bytes=w, route=args.route, device=local, profile=0)
    stream = torch.cuda.current_stream(dev)

    for _ in range(max(args.warmup, 1)):
        eng.labels(edges_d, n, out=lab)
    torch.cuda.synchronize(dev)
    if not check_labels(torch, edges_d, lab, n):
        raise SystemExit("label invariants violated after warm-up")

    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    e0.record(stream)
    for _ in range(args.steps):
        eng.labels(edges_d, n, out=lab)
        launches += eng.stats()["launches"]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    value = replica_value(world, m, args.steps, ms)

    # second timed region: the same calls with per-kernel CUDA events on the
    # launching stream (host-driven loop), for the kernel breakdown and roofline
    eng.set_options(profile=1)
    eng.labels(edges_d, n, out=lab)
    torch.cuda.synchronize(dev)
    kms, kla = {}, {}
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        eng.labels(edges_d, n, out=lab)
        st = eng.stats()
        for k, v in st["kernel_ms"].items():
            kms[k] = kms.get(k, 0.0) + v
            kla[k] = kla.get(k, 0) + st["kernel_launches"][k]
    p1.record(stream)
    torch.cuda.synchronize(dev)
    ms_profiled = p0.elapsed_time(p1) / args.steps
    clocks = sampler.stop() if sampler else None
    eng.set_options(profile=0)
    last = st

    # roofline of the dominant kernel class
    dom = max(kms, key=lambda k: kms[k])
    per_call_bytes = alg_bytes(dom, last, w)
    per_launch_ms = kms[dom] / max(kla[dom], 1)
    launches_per_call = kla[dom] / args.steps
    achieved = per_call_bytes / launches_per_call / (per_launch_ms / 1e3) / 1e9 if per_launch_ms > 0 else 0.0
    pk = peaks()
    peak = pk.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    if not peak:
        peak = 6800.0
    traffic = ncu_traffic(dom, args.workload)
    if traffic is not None:
        traffic /= launches_per_call
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "alg_bytes_per_launch": per_call_bytes / launches_per_call, "avg_launch_ms": per_launch_ms,
                "traffic": traffic}
    kernels = {k: {"ms_per_step": kms[k] / args.steps, "launches_per_step": kla[k] / args.steps,
                   "gbs": (alg_bytes(k, last, w) / (kms[k] / args.steps / 1e3) / 1e9) if kms[k] > 0 else None}
               for k in kms if kla[k]}
    # the scattered-access ceiling: measured L2 random-op rates of this GPU (outside the timed region)
    rates = None if args.no_l2 else eng.l2_rates()
    for k, kv in kernels.items():
        ops, op = l2_ops(k, last)
        if rates and ops > 0 and kv["ms_per_step"] > 0:
            kv["l2_gops"] = ops / (kv["ms_per_step"] / 1e3) / 1e9
            kv["l2_frac"] = kv["l2_gops"] * 1e9 / rates[op]
    ops, op = l2_ops(dom, last)
    if rates is None:
        rates = {"gather": 0.0, "red_add": 0.0, "red_min": 0.0, "atom_min": 0.0}
    l2_roofline = {"bound": "l2_random_ops", "kernel": dom, "op": op,
                   "ops_per_launch": ops / launches_per_call,
                   "achieved": ops / launches_per_call / (per_launch_ms / 1e3) / 1e9 if per_launch_ms > 0 else 0.0,
                   "peak": rates[op] / 1e9, "unit": "Gop/s",
                   "peak_source": "measured in this run: 2^28 random 4-byte ops over a 64 MiB table "
                                  "(cc_measure_l2_rates, best of 3)",
                   "rates_gops": {r: rates[r] / 1e9 for r in ("gather", "red_add", "red_min", "atom_min")}}
    l2_roofline["frac"] = l2_roofline["achieved"] / l2_roofline["peak"] if l2_roofline["peak"] else None
    if args.no_l2:
        l2_roofline = None

    # end to end through host buffers with the public host-input call
    # (cc_labels_host): the H2D copy of the pairs (chunked, overlapped with the
    # passes that stream them) and the D2H copy of the labels are inside the
    # timed region
    e2e = None
    if not args.no_e2e and (rank == 0 or world > 1):
        h_edges = torch.from_numpy(g.edges).pin_memory()
        h_lab = torch.empty(n, dtype=lab.dtype).pin_memory()
        steps_e2e = max(3, min(args.steps, 10))
        for _ in range(2):
            eng.labels_host(h_edges, n, out=h_lab)
        if not torch.equal(h_lab, lab.cpu()):
            raise SystemExit("cc_labels_host labels differ from cc_labels")
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps_e2e):
            eng.labels_host(h_edges, n, out=h_lab)
        b.record(stream)
        torch.cuda.synchronize(dev)
        t_e2e = max_over_ranks(a.elapsed_time(b) / steps_e2e, dist, dev)
        # the host link alone: the same two copies with no compute, the floor of the e2e time
        d_edges = torch.empty_like(h_edges, device=dev)
        d_lab = torch.empty_like(h_lab, device=dev)
        torch.cuda.synchronize(dev)
        a.record(stream)
        for _ in range(steps_e2e):
            d_edges.copy_(h_edges, non_blocking=True)
            h_lab.copy_(d_lab, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize(dev)
        t_link = a.elapsed_time(b) / steps_e2e
        del d_edges, d_lab
        e2e = {"value": world * m / (t_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(g.edges.nbytes),
               "d2h_bytes_per_step": int(n * lab.element_size()), "ms_per_step": t_e2e,
               "copies_alone_ms": t_link,
               "call": "cc_labels_host (pinned host buffers)"}

    # the forced routes on the same graph (the paper's dynamic-vs-opposite
    # comparison), the edge-list BFS engine, and the learned route with the
    # committed predictor weights
    route_compare = None
    if not args.no_compare and rank == 0:
        route_compare = {}
        variants = [("sv", dict(route="sv")), ("bfs", dict(route="bfs")), ("bfs_edges", dict(route="bfs", bfs_mode=1))]
        wpath = os.path.join(ROOT, "paper_1607_06156_gb300", "route_predictor.bin")
        if os.path.exists(wpath):
            variants.append(("learned", dict(route="learned")))
        ref_lab = lab.clone()
        for r, kw in variants:
            e = cc.Engine(id_bytes=w, device=local, **kw)
            if r == "learned":
                from paper_1607_06156_gb300.train_predictor import load_params

                e.set_predictor(load_params(wpath)[0])
            e.labels(edges_d, n, out=lab)
            torch.cuda.synchronize(dev)
            k = max(3, min(args.steps, 5))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(k):
                e.labels(edges_d, n, out=lab)
            b.record(stream)
            torch.cuda.synchronize(dev)
            t = a.elapsed_time(b) / k
            sd = e.stats()
            if not torch.equal(lab, ref_lab):
                raise SystemExit(f"route {r} changed the labels")
            route_compare[r] = {"value": m / (t / 1e3), "ms_per_step": t, "route": sd["route"],
                                "route_source": sd["route_source"],
                                "stage_ms": {k2: sd[k2] for k2 in ("ms_degree", "ms_predict", "ms_csr", "ms_bfs",
                                                                   "ms_sv", "ms_finalize")}}
            e.close()
        # the paper's own SV design (Algorithm 1: tuples grouped by radix sorts)
        # on the same GPU, one warm-up and one timed call (it is far slower)
        if n < (1 << 31):
            e = cc.Engine(id_bytes=w, device=local)
            e.labels_tuple_sv(edges_d, n, out=lab)
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e.labels_tuple_sv(edges_d, n, out=lab)
            b.record(stream)
            torch.cuda.synchronize(dev)
            t = a.elapsed_time(b)
            sd = e.stats()
            # one more call with the sorts timed (events around each sort)
            e.set_options(profile=1)
            e.labels_tuple_sv(edges_d, n, out=lab)
            sp = e.stats()
            e.close()
            if not torch.equal(lab, ref_lab):
                raise SystemExit("the sort-based SV changed the labels")
            route_compare["tuple_sv_alg1"] = {
                "value": m / (t / 1e3), "ms_per_step": t, "iterations": sd["sv_iters"],
                "sorts": sp["kernel_launches"]["tuple_sort"], "sort_ms": sp["kernel_ms"]["tuple_sort"],
                "sort_share": sp["kernel_ms"]["tuple_sort"] / sp["ms_total"] if sp["ms_total"] > 0 else None,
                "note": "Algorithm 1 on the device: per iteration four radix sorts of the n + 2m tuples "
                        "(plus temporaries) and segmented minima; no prediction"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, k, dt = cpu_oracle_rate(g.edges, n, args.cpu_pairs)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {k} of {m} pairs of the same graph, full n ({dt:.1f} s of sequential union-find)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32" if w == 4 else "int64", "data": "synthetic",
                "config": cfg | {"route_policy": args.route, "route_taken": "bfs+sv" if last["route"] else "sv",
                                 "ks_d": last["ks_d"], "sv_iters": last["sv_iters"],
                                 "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roofline, "l2_roofline": l2_roofline, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clocks,
                "gpu_launches": launches,
                "kernels_note": "per-kernel CUDA events from a second timed region of the same calls with "
                                "profiling on (host-driven SV loop), "
                                f"{ms_profiled:.3f} ms/step there vs {ms / args.steps:.3f} ms/step in the main region",
                "kernels": kernels, "route_compare": route_compare,
                "stage_ms": {k: last[k] for k in ("ms_degree", "ms_predict", "ms_csr", "ms_bfs", "ms_sv",
                                                  "ms_finalize", "ms_total")},
                "m_active": last["m_active"]}
        print(json.dumps(line), flush=True)
    eng.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
