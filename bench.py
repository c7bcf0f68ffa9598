#!/usr/bin/env python
"""SCC throughput benchmark on GB300.

One step = one pass of the whole hot path over one synthetic graph:
scc_graph_create (device CSR -> self-loop-free CSR + transposed CSR) ->
scc_run (trim, pivot batches, first-SCC single-reachability both ways,
multi-reachability batches, labelling, canonical labels) -> scc_graph_destroy.
Inputs are resident in HBM before the timed region; the CSR (> 1 GB) is larger
than the 129 MB L2, so no explicit flush is needed between steps.

Workload (default): R-MAT scale 24, edge factor 16 (a, b, c, d = .57, .19, .19,
.05), self-loops and duplicates removed, ids permuted, seed 0x5CC01.

Prints ONE JSON line (rank 0). `value` is whole-job edges/s: arcs of the input
times steps times replicas over the max-over-ranks time. `e2e` is the same
metric through the C ABI with HOST buffers (pinned host CSR in, host labels out,
copies inside the timed region). `roofline` reports the reachability engine
kernel (the dominant kernel) against the measured HBM copy bandwidth.
`cpu_baseline` times the CPU oracle (iterative Tarjan, one thread) on the same
graph. `--impl reference` times that oracle alone, step by step, on a bounded
sample of the workload.

Multi-GPU: the workload is one graph, which does not shard; N ranks run N
independent replicas (no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "SCC edges/s & HBM GB/s vs peak per graph"
UNIT = "edges/s"

WORKLOADS = {
    "rmat24": dict(kind="rmat", scale=24, ef=16, seed=0x5CC01),
    "torus2d256": dict(kind="torus", dims=2, side=256, p=0.5, seed=0x5CC00),
    "torus3d256": dict(kind="torus", dims=3, side=256, p=0.3, seed=0x5CC02),
    "knn8m": dict(kind="knn", n=8_000_000, k=5, seed=0x5CC03),
    # batched SCC: 4,096 graphs, vertex counts log-uniform in [1e3, 1e6], half 2D
    # tori (side ceil(sqrt n), p = 0.5), half R-MAT (scale round(log2 n), edge
    # factor 8); one packed int32 CSR with int64 bases
    "batch4096": dict(kind="batch", G=4096, n_lo=1000, n_hi=1_000_000, seed=0x5CC04),
    "batch256": dict(kind="batch", G=256, n_lo=1000, n_hi=100_000, seed=0x5CC05),
    # served SCC and reachability: Poisson arrivals, SCC requests on graphs
    # log-uniform in [1e4, 4e6] vertices (R-MAT edge factor 16, 2D tori p = 0.5,
    # 3D tori p = 0.3) and reach_multi queries of 1-64 sources on resident graphs
    "serve": dict(kind="serve", rate=2000.0, seconds=4.0, scc_frac=0.25, n_lo=10_000, n_hi=4_000_000, pool=24,
                  resident=8, cap=120e9, seed=0x5CC06),
}


def make_graph(spec, scale_override=None):
    from paper_2303_04934_gb300 import graphgen as gg
    if spec["kind"] == "rmat":
        return gg.rmat(scale_override or spec["scale"], spec["ef"], seed=spec["seed"])
    if spec["kind"] == "torus":
        return gg.torus(spec["dims"], spec["side"], spec["p"], seed=spec["seed"])
    if spec["kind"] == "knn":
        return gg.knn(spec["n"], spec["k"], seed=spec["seed"])
    raise ValueError(spec)


def workload_name(spec, g):
    if spec["kind"] == "rmat":
        return f"rmat_s{spec['scale']}_ef{spec['ef']}"
    if spec["kind"] == "torus":
        return f"torus{spec['dims']}d_{spec['side']}_p{spec['p']}"
    return f"knn_n{spec['n']}_k{spec['k']}"


# ---------------------------------------------------------------- replicas --
def max_over_ranks(x: float, dist, device) -> float:
    """The largest of every rank's x (the job's time is its slowest replica's)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Replicas of the same workload: units of all ranks over the slowest rank's time."""
    return world * units_per_rank / seconds


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # nvidia-smi initialises the management library when it starts; wait
        # for its first sample so that start-up does not fall in a timed region
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                break
            time.sleep(0.01)

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        out["sm_mhz"] = statistics.median(sm) if sm else None
        out["sm_max_mhz"] = max(mx) if mx else None
        out["reasons"] = sorted(reasons)
        out["samples"] = len(rows)
        return out


# ------------------------------------------------------------- CPU oracle --
def time_oracle(g, reps=1):
    import oracle
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.scc_labels(g.n, g.offsets, g.targets)
    return (time.perf_counter() - t0) / reps


def run_reference(args, spec):
    """--impl reference: the CPU oracle (iterative Tarjan, 1 thread) timed per
    step on a bounded sample of the workload (same generator, smaller scale)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    sample_spec = dict(spec)
    if spec["kind"] == "rmat":
        sample_scale = 20
        g = make_graph(spec, scale_override=sample_scale)
        sample = f"rmat_s{sample_scale}_ef{spec['ef']} (same generator and parameters, 1/16 of the vertices)"
    else:
        g = make_graph(sample_spec)
        sample = "the whole workload"
    for _ in range(args.warmup):
        time_oracle(g)
    ts = [time_oracle(g) for _ in range(args.steps)]
    t = sum(ts)
    value = g.m * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": workload_name(spec, g), "sample": sample,
                                            "n": g.n, "m": g.m},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- batches --
def _stratified(order, k):
    """k graphs spread evenly over a size order."""
    k = max(1, min(k, len(order)))
    return [int(order[int(i * len(order) / k)]) for i in range(k)]


def _oracle_all_cores(p, graphs):
    """Seconds for the CPU oracle on `graphs` of batch p, one graph per thread on
    every host core (the oracle's C code runs without the interpreter lock)."""
    import concurrent.futures as cf
    import oracle
    cores = os.cpu_count() or 1

    def one(gi):
        h = p.graph(gi)
        oracle.scc_labels(h.n, h.offsets, h.targets)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(one, graphs))
    return time.perf_counter() - t0, cores


def run_batch(args, spec):
    """Batched SCC: one step = scc_batch_run over the whole packed batch (the
    input resident on the device; the per-graph transposes are inside the run).
    Beside it: the plain per-graph path (scc_graph_create + scc_run + destroy
    for each graph) timed on a sample of graphs spread over the size range and
    scaled to the batch, and the CPU oracle on all host cores."""
    from paper_2303_04934_gb300 import graphgen as gg
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    t_gen = time.perf_counter()
    p = gg.mixed_batch(spec["G"], spec["n_lo"], spec["n_hi"], seed=spec["seed"])
    t_gen = time.perf_counter() - t_gen
    G, nv, na = p.G, int(p.vbase[-1]), int(p.ebase[-1])
    sizes = np.diff(p.ebase) + np.diff(p.vbase)
    order = np.argsort(-sizes, kind="stable")
    wname = f"batch_G{G}_n{spec['n_lo']}-{spec['n_hi']}_torus2d-rmat8"
    # a replay reads the packed CSR and writes (then reads) its G^T, as large again
    csr_bytes = 4 * (nv + G) + 4 * na
    l2_note = (f"inputs larger than L2 (packed CSR {csr_bytes / 1e9:.2f} GB and its G^T as much again, "
               f"against a 129 MB L2)" if 2 * csr_bytes > 129e6 else
               f"inputs smaller than L2 (packed CSR {csr_bytes / 1e6:.0f} MB): replays may find them in L2")
    config = {"workload": wname, "graphs": G, "vertices": nv, "arcs": na, "seed": spec["seed"],
              "parallelism": f"replicas{world}", "l2": l2_note}

    if args.impl == "reference":
        if rank != 0:
            return 0
        sample = _stratified(order, max(16, G // 16))
        ms_ = na_s = 0
        for _ in range(args.warmup):
            _oracle_all_cores(p, sample[:8])
        ts = []
        for _ in range(args.steps):
            t, cores = _oracle_all_cores(p, sample)
            ts.append(t)
        na_s = int(sum(p.ebase[g + 1] - p.ebase[g] for g in sample))
        value = na_s * args.steps / sum(ts)
        smp = f"{len(sample)} of the {G} graphs, spread over the size range, one graph per thread"
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic", "config": {**config, "sample": smp},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": smp},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch
    from paper_2303_04934_gb300 import build as libbuild
    from paper_2303_04934_gb300 import scc
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()

    if not os.path.exists(libbuild.SO_PATH):
        raise RuntimeError("CUDA library not built: run python -c 'import __graft_entry__ as g; g.build()'")
    scc.load()
    stream = torch.cuda.Stream()
    d = [torch.from_numpy(a).to("cuda") for a in (p.vbase, p.ebase, p.offsets, p.targets)]
    torch.cuda.synchronize()
    h = scc.scc_batch_create(G, d[0], d[1], d[2], d[3], stream)
    tuned = None
    if args.batch_block or args.batch_bps is not None or args.tau:
        c = scc.scc_batch_get_config(h)
        if args.batch_block:
            c.block = args.batch_block
        if args.batch_bps is not None:
            c.blocks_per_sm = args.batch_bps
        if args.tau:
            c.tau = args.tau
        scc.scc_batch_set_config(h, c)
    if args.autotune:
        best, ms_t = scc.scc_batch_autotune(h, sample=min(64, G), stream=stream)
        tuned = {"tau": best.tau, "block": best.block, "lambda": best.lambda_, "sample_ms": ms_t}
    cfg = scc.scc_batch_get_config(h)
    labels_d = torch.empty(max(nv, 1), dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            scc.scc_batch_run(h, labels_d, stream)
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    launches0 = scc.scc_debug_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            scc.scc_batch_run(h, labels_d, stream)
        ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = scc.scc_debug_launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    st = scc.scc_batch_get_stats(h)
    per_graph = None
    if args.verbose:
        tm = scc.scc_debug_batch_times(h, G).astype(np.int64)
        dur = (tm[:, 5] - tm[:, 0]) / 1e6
        span = (tm[:, 5].max() - tm[:, 0].min()) / 1e6
        busy = np.bincount(tm[:, 6], weights=dur, minlength=st["blocks"])
        top = np.argsort(-dur)[:8]
        phase = np.diff(tm[:, :6], axis=1).sum(axis=0) / 1e6
        names = ["transpose", "trim_and_first_scc", "class_trim", "batches", "labels"]
        per_graph = {"span_ms": span, "busiest_block_ms": float(busy.max()), "mean_block_ms": float(busy.mean()),
                     "block_ms_by_phase": {k: float(v) for k, v in zip(names, phase)},
                     "longest": [{"graph": p.names[i], "n": int(p.vbase[i + 1] - p.vbase[i]),
                                  "m": int(p.ebase[i + 1] - p.ebase[i]), "ms": float(dur[i]),
                                  "phases_ms": [float(x) for x in np.diff(tm[i, :6]) / 1e6],
                                  "rounds_searches_reruns_batches": [int(x) for x in tm[i, 7:11]]} for i in top],
                     "totals_rounds_searches_reruns_batches": [int(x) for x in tm[:, 7:11].sum(axis=0)]}
    value = whole_job_rate(na * args.steps, world, ms / 1e3)
    graphs_per_s = whole_job_rate(G * args.steps, world, ms / 1e3)
    # roofline of a whole replay (the persistent kernel, after the G^T passes of
    # the graph groups and a one-thread reset): algorithmic bytes per graph =
    # building G^T (read the targets twice, write them once, 12 B per arc, + 12 B
    # per vertex of offsets) + reading G and G^T once and writing the labels
    # (8 B per arc + 12 B per vertex)
    peaks = _read_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    alg = 20 * na + 24 * nv
    achieved = alg / (ms / args.steps / 1e3) / 1e9
    roofline = {"bound": "hbm",
                "kernel": "k_batch_scc (persistent, one block per graph; whole replay with the G^T passes)",
                "achieved": achieved,
                "peak": hbm_peak, "peak_source": "measured" if "hbm_gbs" in peaks else "fallback", "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "algorithmic_bytes_per_launch": alg,
                "ms_per_launch": ms / args.steps}

    # ---- the plain per-graph path on a sample spread over the sizes, scaled
    plain = None
    if not args.no_plain:
        sample = _stratified(order, 64)
        tot = 0.0
        for gi in sample:
            gph = p.graph(gi)
            if gph.n == 0:
                continue
            od = torch.from_numpy(np.ascontiguousarray(gph.offsets)).to("cuda")
            ad = torch.from_numpy(np.ascontiguousarray(gph.targets)).to("cuda")
            lab = torch.empty(gph.n, dtype=torch.int32, device="cuda")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                for rep in range(2):  # the first call warms this size up
                    if rep == 1:
                        e0.record(stream)
                    hh = scc.scc_graph_create(gph.n, gph.m, od, ad, stream)
                    scc.scc_run(hh, lab, stream)
                    scc.scc_graph_destroy(hh)
                e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        est_ms = tot * G / len(sample)
        plain = {"graphs_per_s": G / (est_ms / 1e3), "edges_per_s": na / (est_ms / 1e3),
                 "ms_per_batch_est": est_ms, "sample_graphs": len(sample),
                 "how": "scc_graph_create + scc_run + scc_graph_destroy per graph on a sample spread over the "
                        "size range, time scaled by G / sample"}

    # ---- end to end: host packed arrays in, host labels out
    e2e = None
    if not args.no_e2e:
        hp = [torch.from_numpy(a).pin_memory() for a in (p.vbase, p.ebase, p.offsets, p.targets)]
        lab_h = torch.empty(max(nv, 1), dtype=torch.int32).pin_memory()
        k2 = max(1, min(args.steps, 2))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k2):
            hh = scc.scc_batch_create(G, hp[0], hp[1], hp[2], hp[3], stream)
            scc.scc_batch_set_config(hh, cfg)
            scc.scc_batch_run(hh, lab_h, stream)
            scc.scc_batch_destroy(hh)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        h2d = sum(int(a.numel()) * a.element_size() for a in hp)
        e2e = {"value": world * na * k2 / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 4 * nv, "steps": k2,
               "includes": "scc_batch_create (copy + validation) + scc_batch_run + scc_batch_destroy"}

    # ---- the CPU oracle on all host cores, on a sample of the batch
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        sample = _stratified(order, max(16, G // 16))
        t, cores = _oracle_all_cores(p, sample)
        na_s = int(sum(p.ebase[g + 1] - p.ebase[g] for g in sample))
        cpu = {"value": na_s / t, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{len(sample)} of the {G} graphs spread over the size range, one graph per thread",
               "seconds": t}
    scc.scc_batch_destroy(h)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {**config, "tau": cfg.tau, "block": cfg.block, "lambda": cfg.lambda_,
                           "beta": cfg.beta, "blocks": st["blocks"], "workspace_gb": st["workspace_bytes"] / 2**30,
                           "step": "scc_batch_run (CUDA graph replay of the persistent launch)",
                           "autotuned": tuned},
                "graphs_per_s": graphs_per_s, "plain_per_graph": plain,
                "speedup_vs_plain": (graphs_per_s / plain["graphs_per_s"]) if plain else None,
                "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clk,
                "gen_seconds": t_gen}
        if per_graph:
            line["per_graph"] = per_graph
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ serving --
def _serve_pool(count, n_lo, n_hi, seed):
    """Graphs log-uniform in [n_lo, n_hi] vertices, cycling R-MAT (edge factor
    16), 2D tori (p = 0.5) and 3D tori (p = 0.3)."""
    from paper_2303_04934_gb300 import graphgen as gg
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), count))):
        s = (seed * 7919 + i) & (2**63 - 1)
        kind = i % 3
        if kind == 0:
            out.append(gg.rmat(max(1, int(round(np.log2(n)))), 16, seed=s))
        elif kind == 1:
            out.append(gg.torus(2, int(np.ceil(np.sqrt(n))), 0.5, seed=s))
        else:
            out.append(gg.torus(3, int(np.ceil(n ** (1 / 3))), 0.3, seed=s))
    return out


def _serve_trace(spec, pool, resident, seed):
    rng = np.random.default_rng(seed)
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / spec["rate"])
        if t >= spec["seconds"]:
            break
        if rng.random() < spec["scc_frac"]:
            reqs.append((t, 0, int(rng.integers(0, len(pool))), None, 0))
        else:
            r = int(rng.integers(0, len(resident)))
            k = int(rng.integers(1, 65))
            reqs.append((t, 1, r, rng.integers(0, resident[r].n, k).astype(np.int32), int(rng.integers(0, 2))))
    return reqs


def _serve_once(scc, cfg, pool_h, res_h, resident, trace):
    """Replay the trace open-loop against a fresh server; returns its stats and
    the wall time from the first arrival to the last completion."""
    srv = scc.SccServer(cfg)
    try:
        gids = [srv.add_graph(g.n, off, adj) for g, (off, adj) in zip(resident, res_h)]
        lab = [np.empty(g.n, np.int32) for g, _ in pool_h]
        outs = [np.empty(g.n, np.uint64) for g in resident]
        srv.reset_stats()
        t0 = time.perf_counter()
        for (ta, kind, idx, src, d) in trace:
            while time.perf_counter() - t0 < ta:
                pass
            if kind == 0:
                g, (off, adj) = pool_h[idx]
                srv.submit_scc(g.n, off, adj, lab[idx])
            else:
                srv.submit_reach(gids[idx], src, d, outs[idx])
        t_sub = time.perf_counter() - t0
        srv.drain()
        wall = time.perf_counter() - t0
        st = srv.stats()
    finally:
        srv.close()
    return st, wall, t_sub


def run_serve(args, spec):
    """Served SCC and reachability (one step = one replay of the arrival trace):
    the continuous-batching server against the same trace served one request at
    a time on the plain path (no batching, no merging, no upload ahead)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    import torch
    from paper_2303_04934_gb300 import scc
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "metric": METRIC,
                              "unavailable": "the served workload has no CPU form; the oracle arm covers the graph "
                                             "workloads"}), flush=True)
        return 0
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    scc.load()
    t_gen = time.perf_counter()
    pool = _serve_pool(spec["pool"], spec["n_lo"], spec["n_hi"], spec["seed"])
    resident = _serve_pool(spec["resident"], spec["n_lo"], spec["n_hi"], spec["seed"] + 1)
    t_gen = time.perf_counter() - t_gen
    if args.serve_seconds:
        spec["seconds"] = args.serve_seconds
    if args.serve_rate:
        spec["rate"] = args.serve_rate
    trace = _serve_trace(spec, pool, resident, spec["seed"] + 2)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    pool_h = [(g, (pin(g.offsets), pin(g.targets))) for g in pool]
    res_h = [(pin(g.offsets), pin(g.targets)) for g in resident]
    n_scc = sum(1 for r in trace if r[1] == 0)
    arcs_scc = sum(pool[r[2]].m for r in trace if r[1] == 0)
    cfg = scc.scc_server_config_default()
    cfg.mem_cap_bytes = int(spec["cap"])
    plain_cfg = scc.scc_server_config_default()
    plain_cfg.mem_cap_bytes = int(spec["cap"])
    plain_cfg.batch_vertices = 0
    plain_cfg.merge_reach = 0
    plain_cfg.prefetch = 0
    launches0 = scc.scc_debug_launch_count()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    st, wall, t_sub = _serve_once(scc, cfg, pool_h, res_h, resident, trace)
    clk = clocks.stop()
    launches = scc.scc_debug_launch_count() - launches0
    plain = None
    if not args.no_plain:
        pst, pwall, _ = _serve_once(scc, plain_cfg, pool_h, res_h, resident, trace)
        plain = {"graphs_per_s": n_scc / pwall, "requests_per_s": len(trace) / pwall, "p50_ms": pst["p50_ms"],
                 "p99_ms": pst["p99_ms"], "scc_p99_ms": pst["scc_p99_ms"], "reach_p99_ms": pst["reach_p99_ms"],
                 "wall_s": pwall, "failed": pst["failed"],
                 "how": "same trace; every request alone on the plain path (scc_graph_create + scc_run, or one "
                        "reach_multi), no batching, no merging, no upload ahead"}
    if rank == 0:
        value = arcs_scc / wall
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 0,
                "ms_per_step": 1e3 * wall, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": "synthetic",
                "config": {"workload": f"serve_poisson{int(spec['rate'])}_{spec['seconds']}s_scc{spec['scc_frac']}",
                           "requests": len(trace), "scc_requests": n_scc, "reach_requests": len(trace) - n_scc,
                           "scc_pool": [f"{g.name} (n={g.n}, m={g.m})" for g in pool],
                           "resident": [f"{g.name} (n={g.n}, m={g.m})" for g in resident],
                           "mem_cap_gb": spec["cap"] / 1e9, "parallelism": f"replicas{world}",
                           "step": "one open-loop replay of the arrival trace, drained"},
                "graphs_per_s": n_scc / wall, "requests_per_s": len(trace) / wall, "submit_s": t_sub,
                "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "scc_p50_ms": st["scc_p50_ms"],
                "scc_p99_ms": st["scc_p99_ms"], "reach_p50_ms": st["reach_p50_ms"], "reach_p99_ms": st["reach_p99_ms"],
                "server": {k: st[k] for k in ("units", "batched_launches", "batched_graphs", "plain_scc",
                                              "reach_launches", "reach_shared", "mem_peak", "max_admitted",
                                              "failed", "busy_reach_ms", "busy_batched_ms", "busy_plain_ms")},
                "plain_per_graph": plain,
                "speedup_vs_plain": {"graphs_per_s": (n_scc / wall) / plain["graphs_per_s"],
                                     "p99": plain["p99_ms"] / max(st["p99_ms"], 1e-9)} if plain else None,
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                        "note": "every request is host in, host out: the served numbers are end to end"},
                "roofline": None, "cpu_baseline": None, "gpu_launches": launches, "clocks": clk,
                "gen_seconds": t_gen}
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ extras --
# The default run (R-MAT 24 headline, one GPU) also measures the other
# configurations in compact form, each beside its CPU oracle: the 3D torus,
# the k-NN graph and the small 2D torus (plain per-graph SCC), the batch of
# 4,096 graphs, and the served trace at its offered rate and at loads the
# server sustains.
def _read_peaks():
    """The measured peaks of this machine (MEASURED_PEAKS.json), or {}."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _extra_graph(name, scc, torch, stream, steps, warmup, cpu):
    spec = WORKLOADS[name]
    t_gen = time.perf_counter()
    g = make_graph(spec)
    t_gen = time.perf_counter() - t_gen
    off_d = torch.from_numpy(g.offsets).to("cuda")
    adj_d = torch.from_numpy(g.targets).to("cuda")
    lab = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()

    def step():
        h = scc.scc_graph_create(g.n, g.m, off_d, adj_d, stream)
        try:
            scc.scc_run(h, lab, stream)
            return scc.scc_get_stats(h)
        finally:
            scc.scc_graph_destroy(h)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    sts = []
    with torch.cuda.stream(stream):
        evs[0].record(stream)
        for i in range(steps):
            sts.append(step())
            evs[i + 1].record(stream)
    torch.cuda.synchronize()
    ms = evs[0].elapsed_time(evs[-1]) / steps
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
    mean = lambda k: sum(st[k] for st in sts) / len(sts)
    out = {"workload": workload_name(spec, g), "n": g.n, "m": g.m, "seed": spec["seed"], "steps": steps,
           "warmup": warmup, "ms_per_step": ms, "edges_per_s": g.m / (ms / 1e3),
           "create_ms": mean("ms_create"), "step_ms": step_ms,
           "run_ms": {k: mean(k) for k in ("ms_trim", "ms_first_scc", "ms_class_trim", "ms_multi_search", "ms_label")},
           "rounds": sts[-1]["search_rounds"], "batches": sts[-1]["batches"], "tau": sts[-1]["tau"],
           "step": "scc_graph_create + scc_run + scc_graph_destroy, inputs resident in device memory",
           "gen_seconds": t_gen}
    if spec["kind"] == "torus" and spec["dims"] == 2:
        out["note"] = "L2-resident (about 1.3 MB of CSR): a bandwidth fraction is not meaningful"
    # the run's algorithmic bytes, counted as for the benchmark graph (8 B per
    # arc examined, 8 B per item expanded, 16 B per pair inserted, 20 B per
    # active vertex per labelling), over the run's mean time (create excluded)
    last = sts[-1]
    E = last["engine_arcs"] + last["multi_arcs"]
    P = last["engine_items"] + last["multi_items"]
    I = last["pairs"]
    act = (g.n - last["n_trimmed"]) + last["multi_active_sum"]
    run_bytes = 8 * E + 8 * P + 16 * I + 20 * act
    run_ms = sum(out["run_ms"].values())
    peak = float(_read_peaks().get("hbm_gbs", 6800.0))
    out["run_roofline"] = {"bound": "hbm", "bytes_formula": "8 E + 8 P + 16 I + 20 sum(active per labelling)",
                           "E_arcs": E, "P_items": P, "I_pairs": I, "active_labelled": act,
                           "algorithmic_bytes": run_bytes, "run_ms": run_ms,
                           "achieved_gbs": run_bytes / (run_ms / 1e3) / 1e9 if run_ms > 0 else None,
                           "frac": run_bytes / (run_ms / 1e3) / 1e9 / peak if run_ms > 0 else None, "peak": peak,
                           "rounds": last["search_rounds"],
                           "note": "latency-bound rounds: the time follows the rounds, not the bytes"}
    out["connectivity"] = _measure_cc(g, off_d, adj_d, scc, torch, stream, 5, 2, cpu)
    if spec["kind"] == "knn":
        # the hash bag of Sec. 3.3 (sampled, sigma = 50) against a reservation bag
        # (sigma = 0: one counter hands out segments), on the multi-reachability
        # heavy graph; scc_run alone on a built graph
        abl = {}
        h = scc.scc_graph_create(g.n, g.m, off_d, adj_d, stream)
        try:
            for name, sig in (("sampled_sigma50", 50), ("reservation", 0)):
                c = scc.scc_config_default()
                c.sigma = sig
                scc.scc_set_config(h, c)
                ts = []
                for rep in range(3):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    with torch.cuda.stream(stream):
                        e0.record(stream)
                        scc.scc_run(h, lab, stream)
                        e1.record(stream)
                    torch.cuda.synchronize()
                    if rep:
                        ts.append(e0.elapsed_time(e1))
                st = scc.scc_get_stats(h)
                abl[name] = {"scc_run_ms": sum(ts) / len(ts), "rounds": st["search_rounds"],
                             "ms_multi_search": st["ms_multi_search"], "pairs": st["pairs"]}
        finally:
            scc.scc_graph_destroy(h)
        out["bag_ablation"] = abl
    if cpu:
        tc = time_oracle(g)
        out["cpu_baseline"] = {"value": g.m / tc, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": "the whole graph, 1 run", "seconds": tc}
        out["gpu_over_oracle"] = (g.m / (ms / 1e3)) / (g.m / tc)
    del off_d, adj_d, lab
    return out


def _measure_cc(g, off_d, adj_d, scc, torch, stream, steps, warmup, cpu):
    """Connected components (cc_run: LDD-UF-JTB with VGC and the hash bag,
    Sec. 5.1) of the undirected graph under the arcs, on a built graph: the
    labels checked against the oracle's union-find, both timed."""
    import oracle
    lab = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")
    h = scc.scc_graph_create(g.n, g.m, off_d, adj_d, stream)
    try:
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                scc.cc_run(h, lab, stream)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(steps):
                scc.cc_run(h, lab, stream)
            ev1.record(stream)
        torch.cuda.synchronize()
        st = scc.cc_get_stats(h)
    finally:
        scc.scc_graph_destroy(h)
    ms = ev0.elapsed_time(ev1) / steps
    out = {"ms_per_run": ms, "edges_per_s": g.m / (ms / 1e3), "steps": steps, "warmup": warmup,
           "components": st["components"], "clusters": st["clusters"], "ldd_rounds": st["ldd_rounds"],
           "ldd_batches": st["ldd_batches"], "cross_arcs": st["cross_arcs"],
           "ms_split": {k: st[k] for k in ("ms_ldd", "ms_union", "ms_label")},
           "step": "cc_run on a built graph (symmetric CSR kept from the warm-up)"}
    if cpu:
        t0 = time.perf_counter()
        want, ncc = oracle.cc_labels(g.n, g.offsets, g.targets)
        tc = time.perf_counter() - t0
        out["labels_equal_oracle"] = bool(np.array_equal(lab.cpu().numpy()[:g.n], want))
        out["cpu_baseline"] = {"value": g.m / tc, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": "the whole graph, 1 run (sequential union-find)", "seconds": tc}
    del lab
    return out


def _measure_le(g, scc, torch, stream, steps, cpu):
    """Least-element lists (le_lists_run: Alg. 5, Sec. 5.2) of the undirected
    graph under the arcs for the handle's seeded order, timed on a built graph;
    the lists checked against the oracle's sequential pruned BFS (same order)."""
    import oracle
    off_d = torch.from_numpy(g.offsets).to("cuda")
    adj_d = torch.from_numpy(g.targets).to("cuda")
    h = scc.scc_graph_create(g.n, g.m, off_d, adj_d, stream)
    try:
        total = scc.le_lists_run(h, stream)  # warm-up (and the symmetric CSR)
        ts = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                total = scc.le_lists_run(h, stream)
                e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        st = scc.le_get_stats(h)
        order = np.empty(g.n, np.int32)
        off = np.empty(g.n + 1, np.int64)
        src = np.empty(max(total, 1), np.int32)
        dist = np.empty(max(total, 1), np.int32)
        scc.le_lists_get(h, order, off, src, dist, total, stream)
    finally:
        scc.scc_graph_destroy(h)
    ms = sum(ts) / len(ts)
    out = {"workload": g.name, "n": g.n, "m": g.m, "ms_per_run": ms, "edges_per_s": g.m / (ms / 1e3),
           "entries": total, "mean_list_length": total / max(g.n, 1), "candidates": st["candidates"],
           "bfs_levels": st["levels"], "arcs_examined": st["arcs"], "launches": st["launches"], "steps": steps,
           "step": "le_lists_run on a built graph (symmetric CSR kept from the warm-up)"}
    if cpu:
        t0 = time.perf_counter()
        w_off, w_src, w_dist = oracle.le_lists(g.n, g.offsets, g.targets, order)
        tc = time.perf_counter() - t0
        out["lists_equal_oracle"] = bool(np.array_equal(off, w_off) and np.array_equal(src[:total], w_src)
                                         and np.array_equal(dist[:total], w_dist))
        out["cpu_baseline"] = {"value": g.m / tc, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": "the whole graph, 1 run (sequential pruned BFS, same order)", "seconds": tc}
    del off_d, adj_d
    return out


def _extra_batch(scc, torch, stream, steps, warmup, cpu):
    from paper_2303_04934_gb300 import graphgen as gg
    import oracle
    spec = WORKLOADS["batch4096"]
    t_gen = time.perf_counter()
    p = gg.mixed_batch(spec["G"], spec["n_lo"], spec["n_hi"], seed=spec["seed"])
    t_gen = time.perf_counter() - t_gen
    G, nv, na = p.G, int(p.vbase[-1]), int(p.ebase[-1])
    sizes = np.diff(p.ebase) + np.diff(p.vbase)
    order = np.argsort(-sizes, kind="stable")
    d = [torch.from_numpy(a).to("cuda") for a in (p.vbase, p.ebase, p.offsets, p.targets)]
    torch.cuda.synchronize()
    h = scc.scc_batch_create(G, d[0], d[1], d[2], d[3], stream)
    try:
        t_tune = time.perf_counter()
        best, ms_t = scc.scc_batch_autotune(h, sample=min(16, G), stream=stream)
        t_tune = time.perf_counter() - t_tune
        tuned = {"tau": best.tau, "block": best.block, "lambda": best.lambda_, "sample_ms": ms_t,
                 "seconds": t_tune}
        cfg = scc.scc_batch_get_config(h)
        labels_d = torch.empty(max(nv, 1), dtype=torch.int32, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                scc.scc_batch_run(h, labels_d, stream)
        torch.cuda.synchronize()
        launches0 = scc.scc_debug_launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(steps):
                scc.scc_batch_run(h, labels_d, stream)
            ev1.record(stream)
        torch.cuda.synchronize()
        launches = scc.scc_debug_launch_count() - launches0
        ms = ev0.elapsed_time(ev1) / steps
        st = scc.scc_batch_get_stats(h)
        tm = scc.scc_debug_batch_times(h, G).astype(np.int64)
        dur = (tm[:, 5] - tm[:, 0]) / 1e6
        span = (tm[:, 5].max() - tm[:, 0].min()) / 1e6
        busy = np.bincount(tm[:, 6], weights=dur, minlength=st["blocks"])
        labels_h = labels_d.cpu().numpy()
    finally:
        scc.scc_batch_destroy(h)
    peaks = _read_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    alg = 20 * na + 24 * nv
    out = {"workload": f"batch_G{G}_n{spec['n_lo']}-{spec['n_hi']}_torus2d-rmat8", "graphs": G, "vertices": nv,
           "arcs": na, "seed": spec["seed"], "steps": steps, "warmup": warmup, "ms_per_step": ms,
           "graphs_per_s": G / (ms / 1e3), "edges_per_s": na / (ms / 1e3), "gpu_launches_per_step": launches / steps,
           "config": {"tau": cfg.tau, "block": cfg.block, "lambda": cfg.lambda_, "beta": cfg.beta,
                      "blocks": st["blocks"], "workspace_gb": st["workspace_bytes"] / 2**30},
           "autotuned": tuned,
           "roofline": {"bound": "hbm", "kernel": "k_batch_scc (whole replay with the G^T passes)",
                        "achieved": alg / (ms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                        "frac": alg / (ms / 1e3) / 1e9 / hbm_peak, "algorithmic_bytes_per_launch": alg,
                        "bytes_formula": "20 B per arc + 24 B per vertex (build G^T, read G and G^T once, write labels)"},
           "span_ms": span, "mean_block_ms": float(busy.mean()), "busiest_block_ms": float(busy.max()),
           "span_over_mean_block": span / max(float(busy.mean()), 1e-9),
           "step": "scc_batch_run (CUDA graph replay of the persistent launch), inputs resident in device memory",
           "gen_seconds": t_gen}
    # the plain per-graph path on a sample spread over the sizes, scaled
    sample = _stratified(order, 64)
    tot = 0.0
    for gi in sample:
        gph = p.graph(gi)
        if gph.n == 0:
            continue
        od = torch.from_numpy(np.ascontiguousarray(gph.offsets)).to("cuda")
        ad = torch.from_numpy(np.ascontiguousarray(gph.targets)).to("cuda")
        lab = torch.empty(gph.n, dtype=torch.int32, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for rep in range(2):  # the first call warms this size up
                if rep == 1:
                    e0.record(stream)
                hh = scc.scc_graph_create(gph.n, gph.m, od, ad, stream)
                scc.scc_run(hh, lab, stream)
                scc.scc_graph_destroy(hh)
            e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    est_ms = tot * G / len(sample)
    out["plain_per_graph"] = {"graphs_per_s": G / (est_ms / 1e3), "edges_per_s": na / (est_ms / 1e3),
                              "ms_per_batch_est": est_ms, "sample_graphs": len(sample)}
    out["speedup_vs_plain"] = out["graphs_per_s"] / out["plain_per_graph"]["graphs_per_s"]
    if cpu:
        import concurrent.futures as cf
        csample = _stratified(order, max(16, G // 16))
        cores = os.cpu_count() or 1
        res = {}

        def one(gi):
            hg = p.graph(gi)
            res[gi] = oracle.scc_labels(hg.n, hg.offsets, hg.targets)[0]

        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=cores) as ex:
            list(ex.map(one, csample))
        tc = time.perf_counter() - t0
        na_s = int(sum(p.ebase[g + 1] - p.ebase[g] for g in csample))
        out["cpu_baseline"] = {"value": na_s / tc, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{len(csample)} of the {G} graphs spread over the size range, one graph "
                                         "per thread", "seconds": tc}
        out["gpu_over_oracle"] = out["edges_per_s"] / out["cpu_baseline"]["value"]
        # the same sampled graphs' labels from the timed replays against the oracle's
        out["labels_checked_graphs"] = len(csample)
        out["labels_equal_oracle"] = bool(all(np.array_equal(p.labels_of(labels_h, g), res[g]) for g in csample))
    del d
    return out


def _extra_serve(scc, torch, sweep=(0.25, 0.5, 0.9), sweep_seconds=2.0):
    spec = dict(WORKLOADS["serve"])
    t_gen = time.perf_counter()
    pool = _serve_pool(spec["pool"], spec["n_lo"], spec["n_hi"], spec["seed"])
    resident = _serve_pool(spec["resident"], spec["n_lo"], spec["n_hi"], spec["seed"] + 1)
    t_gen = time.perf_counter() - t_gen
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    pool_h = [(g, (pin(g.offsets), pin(g.targets))) for g in pool]
    res_h = [(pin(g.offsets), pin(g.targets)) for g in resident]
    cfg = scc.scc_server_config_default()
    cfg.mem_cap_bytes = int(spec["cap"])
    plain_cfg = scc.scc_server_config_default()
    plain_cfg.mem_cap_bytes = int(spec["cap"])
    plain_cfg.batch_vertices = 0
    plain_cfg.merge_reach = 0
    plain_cfg.prefetch = 0

    def both(trace):
        r = {}
        for name, c in (("server", cfg), ("plain", plain_cfg)):
            st, wall, _ = _serve_once(scc, c, pool_h, res_h, resident, trace)
            n_scc = sum(1 for q in trace if q[1] == 0)
            r[name] = {"wall_s": wall, "requests_per_s": len(trace) / wall, "graphs_per_s": n_scc / wall,
                       "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "scc_p99_ms": st["scc_p99_ms"],
                       "reach_p99_ms": st["reach_p99_ms"], "failed": st["failed"]}
        return r

    trace = _serve_trace(spec, pool, resident, spec["seed"] + 2)
    full = both(trace)
    out = {"workload": f"serve_poisson{int(spec['rate'])}_{spec['seconds']}s_scc{spec['scc_frac']}",
           "requests": len(trace), "scc_requests": sum(1 for q in trace if q[1] == 0),
           "mem_cap_gb": spec["cap"] / 1e9, "offered_rate": spec["rate"], "at_offered_rate": full,
           "speedup_vs_plain": {"graphs_per_s": full["server"]["graphs_per_s"] / full["plain"]["graphs_per_s"],
                                "p99": full["plain"]["p99_ms"] / max(full["server"]["p99_ms"], 1e-9)},
           "gen_seconds": t_gen}
    sat = full["server"]["requests_per_s"]  # what the server completes when offered more than it can take
    out["saturation_requests_per_s"] = sat
    loads = []
    for i, frac in enumerate(sweep):
        sp = dict(spec)
        sp["rate"] = frac * sat
        sp["seconds"] = sweep_seconds
        tr = _serve_trace(sp, pool, resident, spec["seed"] + 10 + i)
        r = both(tr)
        loads.append({"fraction_of_saturation": frac, "offered_rate": sp["rate"], "requests": len(tr), **r})
    out["below_saturation"] = loads
    out["note"] = ("every request is host in, host out; at the offered 2,000 requests/s both servers are "
                   "overloaded, so their latencies there are queueing delays; the loads below saturation are "
                   "fractions of the rate the continuous-batching server completes when overloaded")
    return out


# ------------------------------------------------------------------- ours --
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat24", choices=sorted(WORKLOADS))
    ap.add_argument("--rmat-scale", type=int, default=None,
                    help="profiling aid: R-MAT scale instead of the workload's (not a bench line)")
    ap.add_argument("--rmat-ef", type=int, default=None,
                    help="profiling aid: R-MAT edge factor instead of the workload's (not a bench line)")
    ap.add_argument("--tau", type=int, default=None)
    ap.add_argument("--seeds", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--autotune", action="store_true", help="batch workloads: run the autotuner first")
    ap.add_argument("--no-plain", action="store_true", help="batch workloads: skip the per-graph comparison")
    ap.add_argument("--batch-block", type=int, default=None, help="batch workloads: threads per block")
    ap.add_argument("--batch-bps", type=int, default=None, help="batch workloads: blocks per SM (0 = auto)")
    ap.add_argument("--serve-seconds", type=float, default=None, help="serve workload: trace length")
    ap.add_argument("--serve-rate", type=float, default=None, help="serve workload: arrivals per second")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the other configurations measured beside the headline")
    args = ap.parse_args()
    spec = dict(WORKLOADS[args.workload])
    if spec["kind"] == "batch":
        return run_batch(args, spec)
    if spec["kind"] == "serve":
        return run_serve(args, spec)
    if args.rmat_scale and spec["kind"] == "rmat":
        spec["scale"] = args.rmat_scale
    if args.rmat_ef and spec["kind"] == "rmat":
        spec["ef"] = args.rmat_ef
    if args.impl == "reference":
        return run_reference(args, spec)

    import torch
    from paper_2303_04934_gb300 import build as libbuild
    from paper_2303_04934_gb300 import scc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()

    if not os.path.exists(libbuild.SO_PATH):
        raise RuntimeError("CUDA library not built: run python -c 'import __graft_entry__ as g; g.build()'")
    scc.load()

    t_gen = time.perf_counter()
    g = make_graph(spec)
    t_gen = time.perf_counter() - t_gen
    n, m = g.n, g.m
    stream = torch.cuda.Stream()
    off_d = torch.from_numpy(g.offsets).to("cuda")
    adj_d = torch.from_numpy(g.targets).to("cuda")
    labels_d = torch.empty(n, dtype=torch.int32, device="cuda")
    cfg = scc.scc_config_default()
    if args.tau:
        cfg.tau = args.tau
    if args.seeds:
        cfg.seeds = args.seeds
    torch.cuda.synchronize()

    def step(offp, adjp, labp):
        h = scc.scc_graph_create(n, m, offp, adjp, stream)
        try:
            scc.scc_set_config(h, cfg)
            scc.scc_run(h, labp, stream)
            st = scc.scc_get_stats(h)
        finally:
            scc.scc_graph_destroy(h)
        return st

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(off_d, adj_d, labels_d)
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    launches0 = scc.scc_debug_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            stats.append(step(off_d, adj_d, labels_d))
        ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = scc.scc_debug_launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    value = whole_job_rate(m * args.steps, world, ms / 1e3)

    # ---- roofline of the dominant kernel. Candidates, each timed live with CUDA
    # events on its launching stream inside the library, with its algorithmic
    # bytes per launch (the data the algorithm must move):
    #   first-SCC engine (2 launches): 4 B arc target + 4 B visited word per arc
    #     examined, 8 B row offsets per item expanded;
    #   transpose rows pass: read the 2 B local target twice and the 4 B source
    #     once, write the source and the row offset: 12 B per arc + 4 B per vertex;
    #   transpose split pass: read and write (u, local target): 12 B per arc;
    #   transpose partition pass: read the arc, write (u, local target): 10 B per
    #     arc + 4 B per vertex (row offsets of the tiles);
    #   intake pass (copy + range check + bucket histogram of the targets):
    #     read and write 4 B per arc;
    #   multi-reachability batch loop: 8 B per arc examined (target + label),
    #     8 B row offsets per item expanded, 16 B per pair inserted (table
    #     slot + bag slot).
    peaks = _read_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    mt = m  # generated graphs have no self-loops
    cands = {
        "engine_kernel<PolSingle> (first-SCC VGC reachability)": (
            sum(s["ms_engine"] for s in stats), sum(s["engine_launches"] for s in stats),
            sum(8 * s["engine_arcs"] + 8 * s["engine_items"] for s in stats)),
        "k_sub_rows (transpose, per-sub-bucket rows)": (
            sum(s["ms_transpose_rows"] for s in stats), len(stats), len(stats) * (12 * mt + 4 * n)),
        "k_bucket_split (transpose, buckets into sub-buckets)": (
            sum(s["ms_transpose_split"] for s in stats), len(stats), len(stats) * (12 * mt)),
        "k_bucket_part (transpose, bucket partition)": (
            sum(s["ms_transpose_part"] for s in stats), len(stats), len(stats) * (10 * m + 4 * n)),
        "k_copy_check_hist (intake: copy, range check, bucket histogram)": (
            sum(s["ms_transpose_hist"] for s in stats), len(stats), len(stats) * (8 * m)),
        "bgss_kernel (multi-reachability batch loop)": (
            sum(s["ms_multi_search"] for s in stats), sum(s["multi_launches"] for s in stats),
            sum(8 * s["multi_arcs"] + 8 * s["multi_items"] + 16 * s["pairs"] for s in stats)),
    }
    kname, (kms, klaunch, kbytes) = max(cands.items(), key=lambda kv: kv[1][0])
    achieved = kbytes / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    # measured DRAM bytes per launch of this kernel (profiles/traffic.json, an ncu
    # capture scaled to this workload), only while the kernel source is unchanged
    traffic = None
    try:
        import hashlib
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json"))).get(kname)
        if rec and spec["kind"] == "rmat" and spec["scale"] == 24:
            cur = hashlib.sha256(open(os.path.join(ROOT, rec["source"]), "rb").read()).hexdigest()
            if cur == rec["source_sha256"]:
                traffic = rec["bytes_per_launch"]
    except Exception:
        traffic = None
    # the transpose build (a1) as one unit: G read twice and G^T written once,
    # 2 (4m + 4n) + (4m + 4n) = 12m + 12n bytes, over the four passes' time
    a1_ms = sum(s["ms_transpose_hist"] + s["ms_transpose_part"] + s["ms_transpose_split"] + s["ms_transpose_rows"]
                for s in stats) / len(stats)
    a1_bytes = 12 * m + 12 * n
    a1 = {"ms_per_step": a1_ms, "algorithmic_bytes": a1_bytes, "bytes_formula": "12m + 12n (G read twice, G^T written once)",
          "achieved_gbs": a1_bytes / (a1_ms / 1e3) / 1e9 if a1_ms > 0 else None,
          "frac": (a1_bytes / (a1_ms / 1e3) / 1e9 / hbm_peak) if a1_ms > 0 else None,
          "passes_ms": {k: sum(s[k] for s in stats) / len(stats) for k in
                        ("ms_transpose_hist", "ms_transpose_part", "ms_transpose_split", "ms_transpose_rows")}}
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm_peak,
                "peak_source": peak_src, "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": traffic,
                "algorithmic_bytes_per_launch": kbytes / max(1, klaunch),
                "ms_per_launch": kms / max(1, klaunch), "share_of_step": (kms / ms) if ms > 0 else None,
                "others": {k: {"ms_per_step": v[0] / max(1, len(stats)),
                               "achieved_gbs": (v[2] / (v[0] / 1e3) / 1e9) if v[0] > 0 else None}
                           for k, v in cands.items() if k != kname}}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        off_h = torch.from_numpy(g.offsets).pin_memory()
        adj_h = torch.from_numpy(g.targets).pin_memory()
        lab_h = torch.empty(n, dtype=torch.int32).pin_memory()
        k2 = max(1, min(args.steps, 10))  # whole-step wall time over up to 10 steps: one host hiccup moves it less
        with torch.cuda.stream(stream):
            step(off_h, adj_h, lab_h)
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            for _ in range(k2):
                st_e2e = step(off_h, adj_h, lab_h)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
        barrier()
        te = max_over_ranks(t1 - t0, dist, "cuda")
        e2e = {"value": whole_job_rate(m * k2, world, te), "unit": UNIT, "h2d_bytes_per_step": 4 * (n + 1) + 4 * m,
               "d2h_bytes_per_step": 4 * n, "steps": k2, "ms_per_step": 1e3 * te / k2,
               "create_ms_last_step": {k: st_e2e[k] for k in ("ms_create", "ms_transpose_hist", "ms_transpose_part",
                                                              "ms_transpose_split", "ms_transpose_rows")}}

    # ---- CPU oracle on the host cores (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if m > 400_000_000:
            sample_scale = 22
            gs = make_graph(spec, scale_override=sample_scale)
            sample = f"rmat_s{sample_scale}_ef{spec['ef']} (same generator and parameters, 1/4 of the vertices), 1 run"
        else:
            gs, sample = g, "the whole workload, 1 run"
        tcpu = time_oracle(gs)
        cpu = {"value": gs.m / tcpu, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
               "host_cores": os.cpu_count(), "seconds": tcpu}

    last = stats[-1]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload_name(spec, g), "n": n, "m": m, "seed": spec["seed"],
                       "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (CSR + transpose > 2 GB)",
                       "tau": cfg.tau or last["tau"], "tau_auto": cfg.tau == 0, "seeds": cfg.seeds,
                       "beta": cfg.beta, "lambda": cfg.lambda_,
                       "step": "scc_graph_create + scc_run + scc_graph_destroy"},
            "e2e": e2e, "roofline": roofline, "a1_transpose": a1, "cpu_baseline": cpu, "gpu_launches": launches,
            "clocks": clk}
    # one extra step with the three calls timed separately (outside the timed
    # region): the SCC computation alone (scc_run on a built graph) as a rate too
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(2):  # the second one is reported
        with torch.cuda.stream(stream):
            evs[0].record(stream)
            h = scc.scc_graph_create(n, m, off_d, adj_d, stream)
            evs[1].record(stream)
            scc.scc_set_config(h, cfg)
            scc.scc_run(h, labels_d, stream)
            evs[2].record(stream)
            scc.scc_graph_destroy(h)
            evs[3].record(stream)
        torch.cuda.synchronize()
    t_run = evs[1].elapsed_time(evs[2])
    line["split_ms"] = {"create": evs[0].elapsed_time(evs[1]), "run": t_run, "destroy": evs[2].elapsed_time(evs[3])}
    # the whole run's algorithmic bytes (counted from the run's own counters):
    # 4 B target + 4 B label or visited word per arc examined, 8 B row offsets
    # per item expanded, 16 B per pair inserted (table slot + bag slot), 20 B per
    # active vertex per labelling (the first SCC's over the untrimmed vertices,
    # then one per multi-reachability batch); the step adds the transpose
    # build's 12m + 12n
    E = last["engine_arcs"] + last["multi_arcs"]
    P = last["engine_items"] + last["multi_items"]
    I = last["pairs"]
    act = (n - last["n_trimmed"]) + last["multi_active_sum"]
    run_bytes = 8 * E + 8 * P + 16 * I + 20 * act
    line["run_roofline"] = {
        "bound": "hbm", "bytes_formula": "8 E + 8 P + 16 I + 20 sum(active per labelling)",
        "E_arcs": E, "P_items": P, "I_pairs": I, "active_labelled": act, "algorithmic_bytes": run_bytes,
        "scc_run_ms": t_run, "achieved_gbs": run_bytes / (t_run / 1e3) / 1e9 if t_run > 0 else None,
        "frac": run_bytes / (t_run / 1e3) / 1e9 / hbm_peak if t_run > 0 else None, "peak": hbm_peak,
        "step_bytes": run_bytes + a1_bytes, "step_ms": ms / args.steps,
        "step_achieved_gbs": (run_bytes + a1_bytes) / (ms / args.steps / 1e3) / 1e9,
        "step_frac": (run_bytes + a1_bytes) / (ms / args.steps / 1e3) / 1e9 / hbm_peak,
        "lower_bound_bytes": 8 * m + 12 * n,
        "lower_bound_note": "read G and G^T once and write the labels: no SCC method moves fewer bytes"}
    line["scc_run_only"] = {"ms": t_run, "edges_per_s": m / (t_run / 1e3) if t_run > 0 else None,
                            "note": "one scc_run on a built graph (the step also builds and frees it)"}
    if args.verbose:
        line["breakdown_last_step"] = last
        line["gen_seconds"] = t_gen
    if (rank == 0 and world == 1 and not args.no_extras and args.workload == "rmat24" and not args.rmat_scale
            and not args.rmat_ef):
        t_x = time.perf_counter()
        line["connectivity"] = _measure_cc(g, off_d, adj_d, scc, torch, stream, 5, 2, not args.no_cpu_baseline)
        del off_d, adj_d, labels_d
        torch.cuda.synchronize()
        cpu_x = not args.no_cpu_baseline
        line["workloads"] = {nm: _extra_graph(nm, scc, torch, stream, 5, 3, cpu_x)
                             for nm in ("torus3d256", "knn8m", "torus2d256")}
        from paper_2303_04934_gb300 import graphgen as gg
        line["lelists"] = [_measure_le(gx, scc, torch, stream, 3, cpu_x)
                           for gx in (gg.rmat(20, 16, seed=0x5CC01), gg.torus(3, 64, 0.3, seed=0x5CC02))]
        torch.cuda.empty_cache()
        line["batched"] = _extra_batch(scc, torch, stream, 3, 3, cpu_x)
        torch.cuda.empty_cache()
        line["served"] = _extra_serve(scc, torch)
        line["extras_seconds"] = time.perf_counter() - t_x
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
