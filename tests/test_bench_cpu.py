"""CPU checks of bench.py's host logic: the reference arm (the oracle on the
host cores) at one rank and under a two-rank torchrun launch, the
max/sum-over-ranks reductions on a world-size-2 gloo process group, and the
roofline record's arithmetic."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_reference_arm_one_rank():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "grid32",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    ln = lines[0]
    assert ln["impl"] == "reference" and ln["unit"] == "pairs/s" and ln["value"] > 0
    assert ln["n_gpus"] == 1 and ln["steps"] == 2 and ln["warmup"] == 1
    assert ln["higher_is_better"] is True
    assert ln["cpu_baseline"]["kind"] == "oracle" and ln["cpu_baseline"]["cores"] >= 1
    assert ln["cpu_baseline"]["value"] == ln["value"]
    assert ln["e2e"] == {"value": ln["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0,
                         "d2h_bytes_per_step": 0}
    # P = nnz(N(2)) + 2E for the 32 x 32 grid
    assert ln["config"]["pairs_per_iter"] == 11652 + 2 * 1984


def test_reference_arm_two_ranks_prints_one_line():
    port = _free_port()
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1", "--master-port",
                        str(port), "bench.py", "--impl", "reference", "--workload", "grid32",
                        "--steps", "1", "--warmup", "0", "--gpus", "2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference"


def test_unavailable_reference_workloads():
    for wl in ("batch4096", "serve"):
        r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", wl],
                           cwd=ROOT, capture_output=True, text=True, timeout=120)
        assert r.returncode == 0
        ln = _json_lines(r.stdout)[0]
        assert ln["impl"] == "reference" and "unavailable" in ln


def _reduce_worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mx = bench.max_over_ranks(10.0 + 5 * rank, dist, "cpu")
    sm = bench.sum_over_ranks(1.5 + rank, dist, "cpu")
    dist.destroy_process_group()
    q.put((rank, mx, sm))


def test_rank_reductions_gloo_world_size_two():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_reduce_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 15.0, 4.0), (1, 15.0, 4.0)]


def test_reductions_without_process_group():
    import bench
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.sum_over_ranks(3.0, None, "cpu") == 3.0


def test_roofline_record_arithmetic():
    """The roofline record's compulsory bytes (2 B per k-hop entry on the
    blocked path, 4 B on the plain path, 4 B per adjacency entry, 8 B offset
    and two positions per vertex), the achieved bandwidth and fraction, and
    the dominant kernel's own figures, on made-up sizes."""
    import types
    import bench
    g = types.SimpleNamespace(n=1000)
    nnzk, nnza = 50_000, 6_000
    kern = {"name": "blocked_kernel", "ms": 2.0, "launches": 4}
    r = bench.roofline_of(g, nnzk + nnza, nnzk, 8, 0.01, kern, 1000.0, "measured", None)
    comp = 2 * nnzk + 4 * nnza + 8 * 1001 + 16 * 1000
    assert r["alg_bytes_per_launch"] == comp
    assert abs(r["achieved"] - comp / 1e-5 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1000.0) < 1e-12
    assert r["traffic"] is None
    dk = r["dominant_kernel"]
    assert dk["ms_per_launch"] == 0.5 and dk["compulsory_bytes"] == 2 * nnzk
    assert abs(dk["frac"] - 2 * nnzk / 0.5e-3 / 1e9 / 1000.0) < 1e-12
    plain = bench.roofline_of(g, nnzk + nnza, nnzk, 8, 0.01,
                              {"name": "iteration_kernel", "ms": 1.0, "launches": 1},
                              1000.0, "measured", None)
    assert plain["alg_bytes_per_launch"] == comp + 2 * nnzk


def test_traffic_record_follows_the_kernel_sources():
    """A recorded ncu traffic figure is reported only while the kernel
    sources hash to the value recorded with it."""
    import bench
    rec = dict(bench.NCU_TRAFFIC["chunglu250k_k3"])
    saved = bench.NCU_TRAFFIC["chunglu250k_k3"]
    try:
        bench.NCU_TRAFFIC["chunglu250k_k3"] = dict(rec, sources_sha256=bench.kernel_sources_sha256())
        assert bench.measured_traffic("chunglu250k_k3")["bytes"] == rec["bytes"]
        bench.NCU_TRAFFIC["chunglu250k_k3"] = dict(rec, sources_sha256="0" * 64)
        assert bench.measured_traffic("chunglu250k_k3") is None
    finally:
        bench.NCU_TRAFFIC["chunglu250k_k3"] = saved
    assert bench.measured_traffic("no_such_workload") is None
