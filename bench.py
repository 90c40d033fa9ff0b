#!/usr/bin/env python
"""Benchmark of the GiLA k-hop Fruchterman-Reingold layout on GB300.

One step = one whole layout of the workload graph with its placement
resident in HBM: rebuild the k-hop lists N_v(k) (the lists are dropped
before every step), run every FR iteration, then take the FP64 quality
reductions of the result. `value` is pair interactions per second over the
timed steps, P = nnz(N(k)) + nnz(A) directed pairs per iteration (each
k-hop pair gives a repulsion, each edge also an attraction).

Default workload: the 1M-edge power-law graph, Chung-Lu gamma = 2.3,
n = 250,000, E = 1,000,000 (seed 3), k = 3, 300 iterations, linear cooling
from 0.1 sqrt(n), d = 1, FP32 with compensated sums, placement uniform in
[0, sqrt n]^2. The k-hop lists (about 45 GB) are far larger than L2, so no
explicit flush is needed between steps.

On one GPU the same line also carries secondary figures: the triangulated
1000 x 1000 mesh (k = 3), the Barabasi-Albert graphs of 1M edges (k = 2)
and 300k edges (k = 3, k = 2), the batch of 4096 small graphs in one
persistent launch against one-at-a-time launches (FP32 and FP64), and a
short Poisson serving stream against a FIFO one-at-a-time server.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gila|reference]
                       [--workload NAME] [--no-secondary]
Under torchrun each rank lays out its own copy of the workload (replicas).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "ba100k_k3": dict(graph="ba100k", k=3, iters=500, precision="fp32",
                      desc="Barabasi-Albert n=100000 m=3 (299,994 edges), k=3, 500 iterations, "
                           "linear cooling from 0.1*sqrt(n), d=1, FP32"),
    "ba100k_k2": dict(graph="ba100k", k=2, iters=500, precision="fp32",
                      desc="Barabasi-Albert n=100000 m=3 (299,994 edges), k=2, 500 iterations, "
                           "linear cooling from 0.1*sqrt(n), d=1, FP32"),
    "grid32": dict(graph="grid32", k=2, iters=100, precision="fp64",
                   desc="32x32 grid, k=2, 100 iterations, linear cooling from 3.2, d=1, FP64"),
    "mesh1000_k3": dict(graph="mesh1000", k=3, iters=300, precision="fp32c",
                        desc="1000x1000 triangulated mesh, k=3, 300 iterations, FP32 compensated"),
    "chunglu250k_k3": dict(graph="chunglu250k", k=3, iters=300, precision="fp32c",
                           oracle_sample=2048,
                           desc="Chung-Lu gamma=2.3, n=250000, E=1000000, k=3, 300 iterations, "
                                "FP32 compensated"),
    "chunglu40k_k3": dict(graph="chunglu40k", k=3, iters=300, precision="fp32c",
                          oracle_sample=2048,
                          desc="Chung-Lu gamma=2.3, n=40000, E=160000, k=3, 300 iterations, "
                               "FP32 compensated (the default workload's shape at a size a full "
                               "profiler capture handles)"),
    "ba1m_k2": dict(graph="ba1m", k=2, iters=500, precision="fp32", oracle_sample=4096,
                    desc="Barabasi-Albert n=333,334 m=3 (999,996 edges), k=2, 500 iterations, "
                         "linear cooling from 0.1*sqrt(n), d=1, FP32"),
    "ba1m_k3": dict(graph="ba1m", k=3, iters=500, precision="fp32", oracle_sample=2048,
                    desc="Barabasi-Albert n=333,334 m=3 (999,996 edges), k=3, 500 iterations, "
                         "linear cooling from 0.1*sqrt(n), d=1, FP32"),
    "batch4096": dict(k=2, iters=200, precision="fp32",
                      desc="4096 graphs, n log-uniform in [50, 5000] (random trees, near-square "
                           "grids, G(n, 4/(n-1))), k=2, 200 iterations each, one persistent launch"),
    "serve": dict(iters=300, precision="fp32",
                  desc="Poisson stream of Barabasi-Albert layout requests, E log-uniform in "
                       "[1e3, 1e6], k in {2, 3}, 300 iterations, FP32"),
}
PREC = {"fp32": 0, "fp64": 1, "fp32c": 2}

# DRAM traffic of one iteration (ncu dram__bytes_read.sum +
# dram__bytes_write.sum of its blocked_kernel launch and, in tile mode, its
# combine_kernel launch) on a workload, with the SHA-256 of the kernel
# sources it was measured on: reported only while those sources are
# unchanged, else null.
KERNEL_SOURCES = ("paper_1606_02162_gb300/csrc/blocked.cu",
                  "paper_1606_02162_gb300/csrc/force.cuh",
                  "paper_1606_02162_gb300/csrc/device_util.cuh")
NCU_TRAFFIC = {
    "chunglu250k_k3": {"bytes": 22770000000 + 96030000 + 52050000 + 512,
                       "kernels": "blocked_kernel + combine_kernel (one iteration)",
                       "profile": "profiles/launches_chunglu250k_k3.md",
                       "sources_sha256": "ef1358f5c4f89edf74c85712a3ee31cc3b3757f3ada5517093e71b6c4fcefe66"},
}


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(workload: str):
    rec = NCU_TRAFFIC.get(workload)
    if rec is None or rec["sources_sha256"] != kernel_sources_sha256():
        return None
    return rec
DTYPE_NAME = {"fp32": "f32", "fp64": "f64", "fp32c": "f32"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        try:
            os.unlink(self.file.name)
        except OSError:
            pass
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist, device) -> float:
    """The sum of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def init_dist(ws, local):
    """NCCL process group for torchrun replicas (None on one GPU)."""
    if ws <= 1:
        return None
    import torch
    import torch.distributed as dist
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return dist


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(O, g, pos, k, S):
    """The oracle on a systematic sample of S vertices (for graphs whose full
    k-hop lists do not fit the oracle): their k-hop rows (timed), then their
    forces from a k-hop CSR holding only those rows. Returns (pairs of the
    sample per iteration, build seconds, a function timing one force pass)."""
    sel = np.arange(0, g.n, max(1, g.n // S), dtype=np.int64)[:S]
    t = time.perf_counter()
    counts, rows = O.khop_rows(g.n, g.row_ptr, g.col_idx, k, sel)
    t_build = time.perf_counter() - t
    c = np.zeros(g.n, dtype=np.int64)
    c[sel] = counts
    krow = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(c, out=krow[1:])
    deg = np.diff(g.row_ptr)
    pairs = int(counts.sum() + deg[sel].sum())

    def force_pass():
        t0 = time.perf_counter()
        O.forces(g.n, g.row_ptr, g.col_idx, krow, rows, pos, sel=sel)
        return time.perf_counter() - t0

    return pairs, t_build, force_pass, len(sel)


def reference_arm(args, wl, ws, rank):
    """The oracle, as it stands, on the host cores: each step is one FP64 FR
    iteration over the whole workload graph plus 1/iters of the oracle's
    k-hop build (timed once), i.e. the per-iteration share of one layout."""
    if rank != 0:
        return 0
    import oracle as O
    from paper_1606_02162_gb300 import inputs as I
    g, pos = I.workload(wl["graph"])
    k, iters = wl["k"], wl["iters"]
    if wl.get("oracle_sample"):
        pairs, t_build, force_pass, S = oracle_sample(O, g, pos, k, wl["oracle_sample"])
        for _ in range(args.warmup):
            force_pass()
        times = [force_pass() for _ in range(args.steps)]
        t_step = sum(times) / len(times) + t_build / iters
        value = pairs / t_step
        sample = (f"FP64 C oracle on a systematic sample of {S} of {g.n} vertices: their "
                  f"k-hop rows ({t_build:.2f} s, 1/{iters} per step) and one force pass "
                  f"over them per step ({pairs} pairs)")
        line = {
            "impl": "reference", "metric": "pair-interactions/s", "value": value,
            "unit": "pairs/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "n": g.n, "edges": g.num_edges, "k": k,
                       "sample_pairs_per_iter": pairs},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": O.threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return 0
    t = time.perf_counter()
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    t_build = time.perf_counter() - t
    P = int(krow[-1]) + g.nnz
    t0 = 0.1 * math.sqrt(g.n)
    cur = pos
    for i in range(args.warmup):
        cur, _ = O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, cur, O.temperature(0, t0, i, iters))
    times = []
    for i in range(args.steps):
        t = time.perf_counter()
        cur, _ = O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, cur,
                        O.temperature(0, t0, args.warmup + i, iters))
        times.append(time.perf_counter() - t)
    t_step = sum(times) / len(times) + t_build / iters
    value = P / t_step
    cores = O.threads()
    line = {
        "impl": "reference", "metric": "pair-interactions/s", "value": value, "unit": "pairs/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "n": g.n, "edges": g.num_edges, "k": k,
                   "pairs_per_iter": P},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                         "sample": f"FP64 C oracle, one FR iteration over the whole graph per "
                                   f"step plus 1/{iters} of its k-hop build ({t_build:.2f} s)"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(wl, g, pos, budget_s=20.0):
    """The FP64 oracle on the host cores on a bounded sample of the workload:
    its own k-hop build plus as many whole-graph iterations as fit in about
    budget_s seconds, scaled to one whole layout (build + all iterations)."""
    import oracle as O
    k, iters = wl["k"], wl["iters"]
    if wl.get("oracle_sample"):
        pairs, t_build, force_pass, S = oracle_sample(O, g, pos, k, wl["oracle_sample"])
        done, t_it = 0, 0.0
        while done < iters and (done < 2 or t_build + t_it < budget_s):
            t_it += force_pass()
            done += 1
        t_layout = t_build + t_it / done * iters
        cores = O.threads()
        O.set_threads(1)
        try:
            t_one = force_pass()
        finally:
            O.set_threads(cores)
        return {"value": pairs * iters / t_layout, "unit": "pairs/s", "cores": cores,
                "kind": "oracle", "single_thread_pairs_per_s": pairs / t_one,
                "sample": f"FP64 C oracle on a systematic sample of {S} of {g.n} vertices: "
                          f"their k-hop rows ({t_build:.2f} s) + {done} force passes over them "
                          f"({t_it:.2f} s), scaled to one whole layout of the sample"}
    t = time.perf_counter()
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    t_build = time.perf_counter() - t
    P = int(krow[-1]) + g.nnz
    t0 = 0.1 * math.sqrt(g.n)
    cur = pos
    done, t_it = 0, 0.0
    while done < iters and (done < 2 or t_build + t_it < budget_s):
        t = time.perf_counter()
        cur, _ = O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, cur,
                        O.temperature(0, t0, done, iters))
        t_it += time.perf_counter() - t
        done += 1
    t_layout = t_build + t_it / done * iters
    cores = O.threads()
    # the same iteration on one thread (one step, for the per-core figure)
    O.set_threads(1)
    try:
        t = time.perf_counter()
        O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, cur, O.temperature(0, t0, done, iters))
        t_one = time.perf_counter() - t
    finally:
        O.set_threads(cores)
    return {"value": P * iters / t_layout, "unit": "pairs/s", "cores": cores,
            "kind": "oracle",
            "single_thread_pairs_per_s": P / t_one,
            "sample": f"FP64 C oracle: k-hop build ({t_build:.2f} s) + {done} of {iters} "
                      f"iterations ({t_it:.2f} s), scaled to one whole layout; one more "
                      f"iteration on 1 thread ({t_one:.2f} s) for the per-core figure"}


def _timed_region(torch, stream, fn, steps):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def bench_batch(steps, warmup, ws, local, dist, count=4096, plain_every=16):
    """Many small graphs: all `count` layouts per step in one persistent,
    graph-captured launch (plus the one k-hop build of the union), FP32 and
    FP64, against laying every `plain_every`-th graph out one at a time with
    the single-graph kernels. Returns the figures (rank-local layouts/s
    scaled by ws)."""
    import torch

    from paper_1606_02162_gb300 import gila as G
    from paper_1606_02162_gb300 import inputs as I
    wl = WORKLOADS["batch4096"]
    graphs = I.batch_mix(count, 50, 5000, 4)
    pos = [I.uniform_positions(g.n, 400000 + i) for i, g in enumerate(graphs)]
    k, iters = wl["k"], wl["iters"]
    out = {}
    stream = torch.cuda.current_stream()
    for name, prec, dt in (("fp32", G.GILA_FP32, torch.float32), ("fp64", G.GILA_FP64, torch.float64)):
        prm = G.params(k=k, iters=iters, precision=prec)
        b = G.Batch(graphs)
        x0 = torch.tensor(np.concatenate(pos), dtype=dt, device="cuda")
        x = torch.empty_like(x0)
        # launch shape and lane thresholds picked by the library's autotuner
        # on this batch (10 probe iterations per candidate; one-time setup)
        t_tune = time.perf_counter()
        tuning = G.gila_batch_autotune(b.handle, prm, x0, 10)
        t_tune = time.perf_counter() - t_tune

        def step():
            G.gila_batch_khop_reset(b.handle)
            G.gila_batch_build_khop(b.handle, k)
            x.copy_(x0)
            G.gila_layout_batch_device(b.handle, prm, x)

        for _ in range(max(warmup, 1)):
            step()
        clocks = ClockSampler(local)
        clocks.start()
        l0 = G.gila_kernel_launches()
        if dist is not None:
            dist.barrier()
        ms = _timed_region(torch, stream, step, steps)
        if dist is not None:
            dist.barrier()
        ms = max_over_ranks(ms, dist, "cuda")
        launches = G.gila_kernel_launches() - l0
        clk = clocks.stop()
        nnz = G.gila_batch_info(b.handle)["nnz_khop"]
        P = nnz + sum(g.nnz for g in graphs)
        b.close()
        out[name] = {"layouts_per_s": ws * len(graphs) * steps / (ms / 1e3),
                     "ms_per_step": ms / steps,
                     "pairs_per_s": ws * P * iters * steps / (ms / 1e3),
                     "gpu_launches": launches, "clocks": clk,
                     "tuning": tuning, "autotune_s": round(t_tune, 3)}
    # one graph at a time (same kernels of the single-graph path), on a
    # systematic sample of every plain_every-th graph
    sample = graphs[::plain_every]
    spos = pos[::plain_every]
    plain = {}
    for name, prec, dt in (("fp32", G.GILA_FP32, torch.float32), ("fp64", G.GILA_FP64, torch.float64)):
        prm = G.params(k=k, iters=iters, precision=prec)
        hs = [G.Graph.from_inputs(g) for g in sample]
        xs0 = [torch.tensor(p, dtype=dt, device="cuda") for p in spos]
        xs = [torch.empty_like(t) for t in xs0]

        def one_at_a_time():
            for h, a0, a in zip(hs, xs0, xs):
                G.gila_khop_reset(h.handle)
                G.gila_build_khop(h.handle, k)
                a.copy_(a0)
                G.gila_layout_run_device(h.handle, prm, a)

        one_at_a_time()
        pms = _timed_region(torch, stream, one_at_a_time, 1)
        for h in hs:
            h.close()
        plain[name] = ws * len(sample) / (pms / 1e3)
    return {"workload": wl["desc"], "graphs": len(graphs),
            "vertices": int(sum(g.n for g in graphs)),
            "fp32": out["fp32"], "fp64": out["fp64"],
            "plain_one_at_a_time": {"fp32_layouts_per_s": plain["fp32"],
                                    "fp64_layouts_per_s": plain["fp64"],
                                    "sample": f"every {plain_every}th graph ({len(sample)})"},
            "speedup_vs_plain": {"fp32": out["fp32"]["layouts_per_s"] / plain["fp32"],
                                 "fp64": out["fp64"]["layouts_per_s"] / plain["fp64"]}}


def run_batch(args, wl, ws, rank, local):
    """The batch workload as its own JSON line."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local)
    dist = init_dist(ws, local)
    res = bench_batch(args.steps, args.warmup, ws, local, dist)
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {
        "metric": "layouts/s", "value": res["fp32"]["layouts_per_s"], "unit": "layouts/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": res["fp32"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": res,
        "gpu_launches": res["fp32"]["gpu_launches"], "clocks": res["fp32"]["clocks"],
    }
    print(json.dumps(line), flush=True)
    return 0


def bench_serve(ws, local, dist, count=48, emax=1e6, mults=(0.9, 2.0, 4.0), seed=5):
    """Serving stream: layout requests arriving as a Poisson process, served
    by the continuous-batching server, against one-at-a-time service of the
    same requests (a FIFO single server fed by the same arrivals, with each
    request's measured service time). Returns the figures per arrival rate."""
    import torch

    from paper_1606_02162_gb300 import gila as G
    from paper_1606_02162_gb300 import inputs as I
    wl = WORKLOADS["serve"]
    reqs = I.serving_requests(count, seed, emax=emax)
    graphs = [I.barabasi_albert_fast(r["n"], 3, r["seed"]) for r in reqs]
    pos = [I.uniform_positions(g.n, r["seed"]) for g, r in zip(graphs, reqs)]
    prms = [G.params(k=r["k"], iters=wl["iters"], precision=G.GILA_FP32) for r in reqs]
    # one at a time: service time of each request alone
    service = []
    for g, p, prm in zip(graphs[:2], pos[:2], prms[:2]):  # warm-up
        with G.Graph.from_inputs(g) as h:
            G.gila_layout_run(h.handle, prm, p)
    for g, p, prm in zip(graphs, pos, prms):
        t = time.perf_counter()
        with G.Graph.from_inputs(g) as h:
            G.gila_layout_run(h.handle, prm, p)
        service.append(time.perf_counter() - t)
    service = np.array(service)
    capacity = 1.0 / service.mean()  # one-at-a-time layouts/s
    # device time of each request alone (k-hop build and iterations between
    # CUDA events on the stream): with every request's GPU work back to back
    # and no host time at all, the stream could run at most at
    # count / sum(device) layouts/s
    device = []
    stream = torch.cuda.current_stream()
    for g, p, prm in zip(graphs, pos, prms):
        with G.Graph.from_inputs(g) as h:
            x = torch.tensor(p, dtype=torch.float32, device="cuda")
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G.gila_build_khop(h.handle, prm.k)
            G.gila_layout_run_device(h.handle, prm, x)
            e1.record(stream)
            torch.cuda.synchronize()
            device.append(e0.elapsed_time(e1) / 1e3)
    device_bound = len(device) / sum(device)
    free_b, _ = torch.cuda.mem_get_info()
    budget = int(free_b * 0.6)
    runs = []
    for mult in mults:
        rate = mult * capacity
        arrivals = I.poisson_arrivals(count, rate, 55)
        # FIFO single server with the measured service times
        done, plain_lat = 0.0, []
        for a, sv in zip(arrivals, service):
            start = max(a, done)
            done = start + sv
            plain_lat.append(done - a)
        lat = []
        if dist is not None:
            dist.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        l0 = G.gila_kernel_launches()
        with G.Server(budget, 16) as s:
            t0 = time.perf_counter()
            tickets = []
            for a, g, p, prm in zip(arrivals, graphs, pos, prms):
                now = time.perf_counter() - t0
                if a > now:
                    time.sleep(a - now)
                tickets.append(s.submit(g, p, prm))
            for tk in tickets:
                _, info = s.wait(tk)
                lat.append(info["latency_ms"] / 1e3)
            makespan = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
            st = s.stats()
        launches = G.gila_kernel_launches() - l0
        clk = clocks.stop()
        lat = np.array(lat)
        plain_lat = np.array(plain_lat)
        runs.append({"arrival_rate_per_s": rate, "rate_vs_plain_capacity": mult,
                     "gpu_launches": launches, "clocks": clk,
                     "server": {"layouts_per_s": ws * count / makespan,
                                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                                "bytes_peak": st["bytes_peak"]},
                     "plain_one_at_a_time": {"layouts_per_s": ws * count / done,
                                             "p50_ms": float(np.percentile(plain_lat, 50) * 1e3),
                                             "p99_ms": float(np.percentile(plain_lat, 99) * 1e3)}})
    return {"workload": "Poisson stream of Barabasi-Albert layout requests, E log-uniform in "
                        "[1e3, %.0f], k in {2, 3}, 300 iterations, FP32" % emax,
            "requests": count,
            "budget": budget, "plain_capacity_layouts_per_s": capacity,
            "mean_service_ms": float(service.mean() * 1e3),
            "device_bound_layouts_per_s": device_bound,
            "mean_device_ms": float(np.mean(device) * 1e3), "runs": runs}


def run_serve(args, wl, ws, rank, local, count=48, emax=1e6):
    """The serving workload as its own JSON line."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local)
    dist = init_dist(ws, local)
    res = bench_serve(ws, local, dist, count=count, emax=emax)
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    top = res["runs"][-1]
    line = {
        "metric": "layouts/s", "value": top["server"]["layouts_per_s"], "unit": "layouts/s",
        "n_gpus": ws, "steps": 1, "warmup": 2,
        "ms_per_step": ws * count / top["server"]["layouts_per_s"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": res,
        "gpu_launches": top["gpu_launches"], "clocks": top["clocks"],
    }
    print(json.dumps(line), flush=True)
    return 0


def roofline_of(g, P, nnzk, elem, iter_ms, kern, hbm, peak_kind, tr):
    """Roofline record of one FR iteration. The bound is HBM: the only
    compulsory DRAM traffic of an iteration is the id stream of the k-hop
    lists as the kernel reads them (2 B per entry on the blocked path, whose
    ids are 16-bit and relative to a position tile; 4 B on the plain path),
    the adjacency ids of the attraction pass (4 B per directed edge), and per
    vertex the row offset (8 B) and the own position read and written
    (2 x elem); the gathered positions are served on chip (shared-memory
    tiles on the blocked path, L2 otherwise). `frac` is that compulsory
    traffic over the measured iteration time against the measured HBM copy
    bandwidth. The 12 B/pair gather model (a 4 B id and a float2 position per
    pair, every gather counted as HBM traffic) is kept as a second figure;
    it exceeds 1 wherever positions come from shared memory."""
    blocked = bool(kern) and kern.get("name", "").startswith("blocked_kernel")
    id_bytes = 2 if blocked else 4
    nnza = P - nnzk
    comp = id_bytes * nnzk + 4 * nnza + 8 * (g.n + 1) + 2 * elem * g.n
    gather = (4 + elem) * P + 8 * (g.n + 1) + 2 * elem * g.n
    achieved = comp / (iter_ms / 1e3) / 1e9
    rec = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
           "frac": achieved / hbm, "traffic": tr["bytes"] if tr else None,
           "kernel": "one FR iteration (all kernels of an iteration; dominant below)",
           "bytes_model": "compulsory: %d B per k-hop entry (ids as stored) + 4 B per adjacency "
                          "entry + 8 B offset + 2 x %d B position per vertex" % (id_bytes, elem),
           "alg_bytes_per_launch": comp, "iter_ms": iter_ms,
           "peak_source": peak_kind,
           "traffic_source": tr["profile"] if tr else None,
           "gather_model": {"bytes_per_iter": gather,
                            "gbs": gather / (iter_ms / 1e3) / 1e9,
                            "frac": gather / (iter_ms / 1e3) / 1e9 / hbm}}
    if kern and kern["launches"] > 0:
        kms = kern["ms"] / kern["launches"]
        # the repulsion kernel streams the k-hop ids once
        kb = id_bytes * nnzk
        rec["dominant_kernel"] = {"name": kern["name"], "ms_per_launch": kms,
                                  "share_of_iteration": kms / iter_ms,
                                  "compulsory_bytes": kb,
                                  "gbs": kb / (kms / 1e3) / 1e9,
                                  "frac": kb / (kms / 1e3) / 1e9 / hbm}
    return rec


def run_graph(args, name, steps, warmup, with_e2e, with_cpu, ws, rank, dist, local):
    """One single-graph workload: `steps` whole layouts timed with CUDA
    events on the launching stream after `warmup` untimed ones; per-iteration
    and repulsion-kernel times from the library's own events on the same
    stream. Returns a dict of figures."""
    import torch

    from paper_1606_02162_gb300 import gila as G
    from paper_1606_02162_gb300 import inputs as I
    wl = WORKLOADS[name]

    def barrier():
        if dist is not None:
            dist.barrier()

    g, pos0 = I.workload(wl["graph"])
    prec = PREC[wl["precision"]]
    k, iters = wl["k"], wl["iters"]
    prm = G.params(k=k, iters=iters, precision=prec)
    dt = torch.float64 if prec == G.GILA_FP64 else torch.float32
    stream = torch.cuda.current_stream()

    # ------------------------------------------------ device-resident steps
    h = G.Graph.from_inputs(g)
    pos_init = torch.tensor(pos0, dtype=dt, device="cuda")
    pos = torch.empty_like(pos_init)

    def step():
        G.gila_khop_reset(h.handle)
        G.gila_build_khop(h.handle, k)
        pos.copy_(pos_init)
        G.gila_layout_run_device(h.handle, prm, pos)
        return G.gila_layout_metrics(h.handle, prm, pos)

    for _ in range(max(warmup, 0)):
        step()
    torch.cuda.synchronize()
    G.gila_profile_read(h.handle)  # clear
    G.gila_profile_read_kernel(h.handle)
    G.gila_profile_enable(h.handle, 2)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = G.gila_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev0.record(stream)
    marks[0].record(stream)
    last = None
    for i in range(steps):
        last = step()
        marks[i + 1].record(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    step_ms = [marks[i].elapsed_time(marks[i + 1]) for i in range(steps)]
    nnzk = G.gila_graph_info(h.handle)["nnz_khop"]
    P = nnzk + g.nnz
    launches = G.gila_kernel_launches() - launches0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = G.gila_profile_read(h.handle)
    kern = G.gila_profile_read_kernel(h.handle)
    G.gila_profile_enable(h.handle, False)
    ms = max_over_ranks(ms, dist, "cuda")
    value = P * iters * steps * ws / (ms / 1e3)
    iter_ms = prof["iter_ms"] / max(prof["iter_launches"], 1)
    build_ms = prof["build_ms"] / max(prof["builds"], 1)
    h.close()
    del pos, pos_init
    torch.cuda.empty_cache()

    elem = 16 if prec == G.GILA_FP64 else 8
    hbm, peak_kind = peaks()
    roof = roofline_of(g, P, nnzk, elem, iter_ms, kern, hbm, peak_kind, measured_traffic(name))

    # ------------------------------------------------ end to end (host buffers)
    e2e = None
    if with_e2e:
        row = torch.from_numpy(g.row_ptr).pin_memory().numpy()
        col = torch.from_numpy(g.col_idx).pin_memory().numpy()
        pin_in = torch.from_numpy(np.ascontiguousarray(pos0)).pin_memory().numpy()
        pin_out = torch.empty(pin_in.shape, dtype=torch.float64).pin_memory().numpy()
        e2e_steps = min(steps, 10)

        def e2e_step():
            # CSR and placement uploads, k-hop build, iterations, FP64
            # quality reductions and the placement download, all inside
            # the public host-buffer calls
            hh = G.Graph(g.n, row, col)
            try:
                G.gila_layout_run(hh.handle, prm, pin_in, pin_out, metrics=True)
            finally:
                hh.close()

        e2e_step()
        barrier()
        t = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t, dist, "cuda")
        e2e = {"value": P * iters * e2e_steps * ws / e2e_s, "unit": "pairs/s",
               "h2d_bytes_per_step": int(row.nbytes + col.nbytes + pin_in.nbytes),
               "d2h_bytes_per_step": int(pin_out.nbytes) + 2 * 32,
               "ms_per_step": e2e_s / e2e_steps * 1e3, "steps": e2e_steps}

    cpu = None
    if with_cpu and rank == 0 and ws == 1:
        cpu = cpu_baseline(wl, g, pos0)
    return {"name": name, "wl": wl, "g": g, "value": value, "ms": ms, "steps": steps,
            "ms_per_step": ms / steps, "step_ms": step_ms, "nnzk": nnzk, "P": P,
            "iter_ms": iter_ms, "build_ms": build_ms, "launches": launches, "clocks": clk,
            "roofline": roof, "e2e": e2e, "cpu": cpu, "last": last}


def secondary_record(r):
    """Short summary of a secondary workload for the main line."""
    roof = r["roofline"]
    rec = {"workload": r["wl"]["desc"], "pairs_per_iter": r["P"], "ms_per_iter": r["iter_ms"],
           "pairs_per_s": r["value"], "khop_build_and_plan_ms": r["build_ms"],
           "compulsory_frac": roof["frac"], "gather_model_frac": roof["gather_model"]["frac"],
           "steps": r["steps"]}
    dk = roof.get("dominant_kernel")
    if dk:
        rec["dominant_kernel"] = {"name": dk["name"], "ms_per_launch": dk["ms_per_launch"],
                                  "frac": dk["frac"]}
    return rec


SECONDARY = ("mesh1000_k3", "ba1m_k2", "ba1m_k3", "ba100k_k3", "ba100k_k2")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gila", choices=["gila", "reference"])
    ap.add_argument("--workload", default="chunglu250k_k3", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary graphs, the batch and the serving figures")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    ws, rank, local = dist_env()

    if args.impl == "reference":
        if args.workload in ("batch4096", "serve"):
            print(json.dumps({"impl": "reference", "unavailable":
                              "the CPU oracle arm is defined for the single-graph workloads"}))
            return 0
        return reference_arm(args, wl, ws, rank)
    if args.workload == "batch4096":
        return run_batch(args, wl, ws, rank, local)
    if args.workload == "serve":
        return run_serve(args, wl, ws, rank, local)

    import torch

    import __graft_entry__
    __graft_entry__.build()

    torch.cuda.set_device(local)
    dist = init_dist(ws, local)
    r = run_graph(args, args.workload, args.steps, args.warmup, not args.no_e2e,
                  not args.no_cpu_baseline, ws, rank, dist, local)
    # secondary figures, one GPU only: the short-row graphs (mesh, k = 2),
    # the default-sized BA graph, the batch and a short serving stream
    secondary = None
    if ws == 1 and not args.no_secondary:
        secondary = {}
        for name in SECONDARY:
            if name == args.workload:
                continue
            s = run_graph(args, name, 3, 1, False, False, ws, rank, dist, local)
            secondary[name] = secondary_record(s)
        secondary["batch4096"] = bench_batch(1, 1, ws, local, dist)
        secondary["serve"] = bench_serve(ws, local, dist, count=48, emax=1e6, mults=(2.0, 4.0))

    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    g, last = r["g"], r["last"]
    line = {
        "metric": "pair-interactions/s", "value": r["value"], "unit": "pairs/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_NAME[wl["precision"]], "data": "synthetic",
        "config": {"workload": wl["desc"], "n": g.n, "edges": g.num_edges, "k": wl["k"],
                   "iters": wl["iters"], "nnz_khop": r["nnzk"], "pairs_per_iter": r["P"],
                   "ms_per_iter": r["iter_ms"], "khop_build_and_plan_ms": r["build_ms"],
                   "step_ms": [round(x, 3) for x in r["step_ms"]],
                   "layouts_per_s": ws * args.steps / (r["ms"] / 1e3),
                   "l2": "inputs larger than L2 (k-hop lists %.2f GB)" % (4 * r["nnzk"] / 1e9),
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "quality_last": {"edge_cv": last["edge_cv"],
                                    "rep_att_ratio": last["rep_att_ratio"]} if last else None,
                   "secondary": secondary},
        "roofline": r["roofline"], "cpu_baseline": r["cpu"], "e2e": r["e2e"],
        "gpu_launches": r["launches"], "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
