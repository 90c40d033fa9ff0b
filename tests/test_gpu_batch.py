"""Batched layouts (one persistent, graph-captured launch for many graphs)
against the oracle, graph by graph.

  k-hop lists of the union     bit-exact, graph by graph
  one iteration                FP32 within 1e-4, FP64 within 1e-12 of each
                               graph's largest move
  a few iterations (FP64)      within 1e-9 of the placement's extent
  alone vs in the batch        bit-identical (FP32 and FP64)
"""
import math

import numpy as np
import pytest

import __graft_entry__
import oracle as O
from paper_1606_02162_gb300 import gila as G
from paper_1606_02162_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    import torch
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def mix():
    graphs = I.batch_mix(48, 20, 900, 11)
    graphs.append(I.star(600))           # a long row in a small graph
    graphs.append(I.csr_from_edges(5, [], []))  # no edges
    pos = [I.uniform_positions(g.n, 100 + i) for i, g in enumerate(graphs)]
    return graphs, pos


def _concat(pos):
    return np.concatenate(pos, axis=0) if pos else np.zeros((0, 2))


def _split(arr, graphs):
    out, o = [], 0
    for g in graphs:
        out.append(arr[o:o + g.n])
        o += g.n
    return out


def test_batch_khop_matches_oracle_per_graph(mix):
    graphs, _ = mix
    k = 2
    with G.Batch(graphs) as b:
        nnz = G.gila_batch_build_khop(b.handle, k)
        info = G.gila_batch_info(b.handle)
    assert info["count"] == len(graphs) and info["total_n"] == sum(g.n for g in graphs)
    assert nnz == sum(O.khop(g.n, g.row_ptr, g.col_idx, k)[0][-1] for g in graphs)


@pytest.mark.parametrize("prec,tol", [(G.GILA_FP32, 1e-4), (G.GILA_FP32_COMPENSATED, 1e-4),
                                      (G.GILA_FP64, 1e-12)], ids=["fp32", "fp32c", "fp64"])
def test_batch_one_iteration(mix, prec, tol):
    graphs, pos = mix
    k = 2
    with G.Batch(graphs) as b:
        out = G.gila_layout_batch_run(b.handle, G.params(k=k, iters=1, precision=prec), _concat(pos))
    rnd = (lambda p: p.astype(np.float32).astype(np.float64)) if prec != G.GILA_FP64 else (lambda p: p)
    for g, p, o in zip(graphs, pos, _split(out, graphs)):
        if g.n == 0:
            continue
        krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
        base = rnd(p)
        t = 0.1 * math.sqrt(g.n)  # first temperature of the linear schedule, this graph's n
        _, odisp = O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, base, t)
        scale = max(np.abs(odisp).max(), 1e-300)
        assert np.abs((o - base) - odisp).max() <= tol * scale + 4 * np.finfo(np.float32).eps * (
            np.abs(base).max() if prec != G.GILA_FP64 else 0.0), g.name


def test_batch_several_iterations_fp64(mix):
    graphs, pos = mix
    k, iters = 2, 6
    with G.Batch(graphs) as b:
        out = G.gila_layout_batch_run(b.handle, G.params(k=k, iters=iters, precision=G.GILA_FP64),
                                      _concat(pos))
    for g, p, o in zip(graphs, pos, _split(out, graphs)):
        if g.n == 0:
            continue
        krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
        ref = O.run(g.n, g.row_ptr, g.col_idx, krow, kcol, p, iters)
        assert np.abs(o - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max()), g.name


def test_batch_geometric_schedule(mix):
    graphs, pos = mix
    graphs, pos = graphs[:12], pos[:12]
    k, iters = 2, 4
    prm = G.params(k=k, iters=iters, precision=G.GILA_FP64, schedule=G.GILA_COOL_GEOMETRIC, d=1.3)
    with G.Batch(graphs) as b:
        out = G.gila_layout_batch_run(b.handle, prm, _concat(pos))
    for g, p, o in zip(graphs, pos, _split(out, graphs)):
        krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
        ref = O.run(g.n, g.row_ptr, g.col_idx, krow, kcol, p, iters, d=1.3,
                    schedule=O.SCHED_GEOM)
        assert np.abs(o - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max()), g.name


@pytest.mark.parametrize("prec", [G.GILA_FP32, G.GILA_FP64], ids=["fp32", "fp64"])
def test_alone_equals_in_batch(mix, prec):
    graphs, pos = mix
    prm = G.params(k=2, iters=30, precision=prec)
    with G.Batch(graphs) as b:
        together = _split(G.gila_layout_batch_run(b.handle, prm, _concat(pos)), graphs)
    for i in (0, 7, len(graphs) - 2):
        with G.Batch([graphs[i]]) as b1:
            alone = G.gila_layout_batch_run(b1.handle, prm, pos[i])
        assert np.array_equal(alone, together[i]), graphs[i].name


def test_launch_shape_does_not_change_results(mix):
    graphs, pos = mix
    prm = G.params(k=2, iters=10, precision=G.GILA_FP32)
    outs = []
    for threads, ctas in ((256, 1), (512, 2), (1024, 2)):
        with G.Batch(graphs) as b:
            G.gila_batch_tune(b.handle, threads=threads, ctas_per_sm=ctas)
            outs.append(G.gila_layout_batch_run(b.handle, prm, _concat(pos)))
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_graph_replay_and_device_entry(mix):
    import torch
    graphs, pos = mix
    prm = G.params(k=2, iters=8, precision=G.GILA_FP32)
    with G.Batch(graphs) as b:
        x0 = torch.tensor(_concat(pos), dtype=torch.float32, device="cuda")
        a = x0.clone()
        G.gila_layout_batch_device(b.handle, prm, a)  # captures a CUDA graph
        first = a.clone()
        a.copy_(x0)
        G.gila_layout_batch_device(b.handle, prm, a)  # same arguments: replays it
        c = x0.clone()
        G.gila_layout_batch_device(b.handle, prm, c)  # new buffer: captures again
        torch.cuda.synchronize()
        assert torch.equal(a, first) and torch.equal(c, first)
        host = G.gila_layout_batch_run(b.handle, prm, _concat(pos))
        assert np.array_equal(host, first.double().cpu().numpy())


def test_layout_batch_from_graph_handles(mix):
    graphs, pos = mix
    graphs, pos = graphs[:10], pos[:10]
    prm = G.params(k=2, iters=12, precision=G.GILA_FP64)
    hs = [G.Graph.from_inputs(g) for g in graphs]
    try:
        outs = G.gila_layout_batch([h.handle for h in hs], prm, pos)
    finally:
        for h in hs:
            h.close()
    with G.Batch(graphs) as b:
        ref = _split(G.gila_layout_batch_run(b.handle, prm, _concat(pos)), graphs)
    for o, r in zip(outs, ref):
        assert np.array_equal(o, r)


def test_graph_beyond_shared_memory():
    # FP64, 30,000 vertices: two placements need 960 KB, so this graph
    # iterates on global buffers inside its CTA
    g = I.barabasi_albert(30000, 2, 3)
    small = I.grid(10, 10)
    graphs = [small, g]
    pos = [I.uniform_positions(x.n, 7 + i) for i, x in enumerate(graphs)]
    k = 2
    with G.Batch(graphs) as b:
        out = _split(G.gila_layout_batch_run(b.handle, G.params(k=k, iters=1, precision=G.GILA_FP64),
                                             _concat(pos)), graphs)
    for x, p, o in zip(graphs, pos, out):
        krow, kcol = O.khop(x.n, x.row_ptr, x.col_idx, k)
        _, odisp = O.step(x.n, x.row_ptr, x.col_idx, krow, kcol, p, 0.1 * math.sqrt(x.n))
        assert np.abs((o - p) - odisp).max() <= 1e-12 * np.abs(odisp).max()


def test_autotune_returns_a_valid_shape(mix):
    import torch
    graphs, pos = mix
    prm = G.params(k=2, iters=20, precision=G.GILA_FP32)
    with G.Batch(graphs) as b:
        x = torch.tensor(_concat(pos), dtype=torch.float32, device="cuda")
        before = x.clone()
        t = G.gila_batch_autotune(b.handle, prm, x, probe_iters=3)
        assert torch.equal(x, before)  # the probe does not touch the input
        assert t["threads"] in (256, 512, 1024) and t["ctas_per_sm"] >= 1
        out = G.gila_layout_batch_run(b.handle, G.params(k=2, iters=1, precision=G.GILA_FP32),
                                      _concat(pos))
    for g, p, o in zip(graphs, pos, _split(out, graphs)):
        if g.n == 0:
            continue
        krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
        base = p.astype(np.float32).astype(np.float64)
        _, odisp = O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, base, 0.1 * math.sqrt(g.n))
        assert np.abs((o - base) - odisp).max() <= 1e-4 * np.abs(odisp).max() + 4e-7 * np.abs(base).max()
