"""GPU parity of degree-one pruning, weighted repulsion and reinsertion
(Sections 4.3 and 4.6) against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1606_02162_gb300 import gila as G
from paper_1606_02162_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _leafy_graphs():
    return [
        ("tree", I.random_tree(3000, 21)),
        ("ba1", I.barabasi_albert(4000, 1, 22)),
        ("ba2", I.barabasi_albert(5000, 2, 23)),
        ("chunglu", I.chung_lu(6000, 2.3, 3.0, 9000, 24)),
        ("star", I.star(40)),
        ("edge", I.path(2)),
        ("path", I.path(9)),
        ("cycle", I.cycle(30)),
    ]


@pytest.mark.parametrize("name,g", _leafy_graphs(), ids=[n for n, _ in _leafy_graphs()])
def test_prune_structure_matches_oracle(name, g):
    _torch()
    anchor, w, newid, kept = O.prune(g.n, g.row_ptr, g.col_idx)
    prow, pcol = O.pruned_csr(g.n, g.row_ptr, g.col_idx, newid, kept)
    with G.Graph.from_inputs(g) as h, G.Pruned(h) as p:
        assert p.kept == kept and p.removed == g.n - kept
        a2, w2, i2 = G.gila_pruned_export(p.handle, g.n)
        assert np.array_equal(a2, anchor) and np.array_equal(w2, w) and np.array_equal(i2, newid)
        pg = p.pruned_graph
        info = G.gila_graph_info(pg)
        assert info["n"] == kept and info["nnz_adj"] == len(pcol)
        # the pruned adjacency, read back as its 1-hop lists
        G.gila_build_khop(pg, 1)
        krow, kcol = G.gila_khop_export(pg)
        assert np.array_equal(krow, prow) and np.array_equal(kcol, pcol)


@pytest.mark.parametrize("prec,tol", [(G.GILA_FP32, 1e-4), (G.GILA_FP32_COMPENSATED, 1e-4),
                                      (G.GILA_FP64, 1e-12)], ids=["fp32", "fp32c", "fp64"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_weighted_step_matches_oracle(prec, tol, k):
    torch = _torch()
    g = I.barabasi_albert(3000, 2, 31)
    pos = I.uniform_positions(g.n, 32)
    wt = 1.0 + (np.arange(g.n) * 7919 % 5).astype(np.float64)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    t = 0.8
    ref, rdisp = O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, t, wt=wt)
    dt = torch.float64 if prec == G.GILA_FP64 else torch.float32
    with G.Graph.from_inputs(g) as h:
        G.gila_graph_set_repulsion_weights(h.handle, wt)
        x = torch.tensor(pos, dtype=dt, device="cuda")
        y = torch.empty_like(x)
        disp = torch.empty_like(x)
        G.gila_layout_step(h.handle, G.params(k=k, precision=prec), t, x, y, disp)
        got = disp.double().cpu().numpy()
    scale = np.abs(rdisp).max()
    assert np.abs(got - rdisp).max() <= tol * scale
    # the weights matter: the unweighted step differs by far more
    _, udisp = O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, t)
    assert np.abs(udisp - rdisp).max() > 100 * tol * scale


def test_weights_clear_and_validate():
    torch = _torch()
    g = I.barabasi_albert(500, 2, 33)
    pos = I.uniform_positions(g.n, 34)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
    _, rdisp = O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, 1.0)
    with G.Graph.from_inputs(g) as h:
        G.gila_graph_set_repulsion_weights(h.handle, np.full(g.n, 2.0))
        G.gila_graph_set_repulsion_weights(h.handle, None)
        x = torch.tensor(pos, dtype=torch.float64, device="cuda")
        y, disp = torch.empty_like(x), torch.empty_like(x)
        G.gila_layout_step(h.handle, G.params(k=2, precision=G.GILA_FP64), 1.0, x, y, disp)
        assert np.abs(disp.cpu().numpy() - rdisp).max() <= 1e-12 * np.abs(rdisp).max()
        bad = np.ones(g.n)
        bad[3] = -1.0
        with pytest.raises(G.GilaError):
            G.gila_graph_set_repulsion_weights(h.handle, bad)
        G.gila_graph_set_repulsion_weights(h.handle, np.ones(g.n))
        with pytest.raises(G.GilaError):
            G.gila_layout_step(h.handle, G.params(k=2, precision=G.GILA_FP64_ORDERED), 1.0, x, y)


def _rotation_scores(ppos, pv, nb, m):
    s = 2 * math.pi / m
    theta = s * (np.arange(64) + 0.5) / 64
    if len(nb) == 0:
        return np.full(64, np.inf), s
    vec = ppos[nb] - ppos[pv]
    a = np.mod(np.arctan2(vec[:, 1], vec[:, 0]), s)
    diff = np.abs(a[None, :] - theta[:, None])
    return np.minimum(diff, s - diff).min(axis=1), s


@pytest.mark.parametrize("prec", [G.GILA_FP64, G.GILA_FP32], ids=["fp64", "fp32"])
def test_reinsert_matches_oracle(prec):
    torch = _torch()
    g = I.barabasi_albert(6000, 1, 41)
    anchor, w, newid, kept = O.prune(g.n, g.row_ptr, g.col_idx)
    prow, pcol = O.pruned_csr(g.n, g.row_ptr, g.col_idx, newid, kept)
    ppos = I.uniform_positions(kept, 42) * 2.0
    if prec == G.GILA_FP32:
        ppos = ppos.astype(np.float32).astype(np.float64)
    ref = O.reinsert(g.n, g.row_ptr, g.col_idx, newid, anchor, w, prow, pcol, ppos, d=1.0)
    dt = torch.float64 if prec == G.GILA_FP64 else torch.float32
    with G.Graph.from_inputs(g) as h, G.Pruned(h) as p:
        pp = torch.tensor(ppos, dtype=dt, device="cuda")
        full = torch.zeros((g.n, 2), dtype=dt, device="cuda")
        G.gila_reinsert_degree_one(p.handle, G.params(precision=prec), pp, full)
        got = full.double().cpu().numpy()
    keep = newid >= 0
    assert np.array_equal(got[keep], ppos)
    # FP64: a few ulps of cos/sin; FP32: the rounding of the stored coordinates
    tol = (1e-12 if prec == G.GILA_FP64 else 1e-6) * max(1.0, np.abs(ref).max())
    bad = np.nonzero(np.abs(got - ref).max(axis=1) > tol)[0]
    # a differing leaf is allowed only where the rotation was a near-tie
    # (atan2 of the two sides may differ in the last bit): the device's choice
    # must then score as well as the best
    for u in bad:
        v = anchor[u]
        assert v >= 0
        pv = newid[v]
        nb = pcol[prow[pv]:prow[pv + 1]]
        score, s = _rotation_scores(ppos, pv, nb, w[v])
        r = got[u] - ppos[pv]
        ang = math.atan2(r[1], r[0]) % s
        c = int(round(ang / s * 64 - 0.5)) % 64
        assert score[c] >= score.max() - 1e-9
    assert len(bad) <= max(2, g.n // 1000)


@pytest.mark.parametrize("prec", [G.GILA_FP64, G.GILA_FP32], ids=["fp64", "fp32"])
def test_pipeline_one_iteration_matches_oracle(prec):
    """Gather, one weighted iteration, reinsert: the whole pipeline for one
    iteration against the oracle's."""
    _torch()
    g = I.barabasi_albert(3000, 1, 51)
    pos0 = I.uniform_positions(g.n, 52)
    prm = G.params(k=2, iters=1, precision=prec)
    ref = O.pipeline(g.n, g.row_ptr, g.col_idx, pos0, k=2, iters=1)
    with G.Graph.from_inputs(g) as h, G.Pruned(h) as p:
        got = G.gila_layout_pruned_run(p.handle, prm, pos0)
    anchor, w, newid, kept = O.prune(g.n, g.row_ptr, g.col_idx)
    keep = newid >= 0
    move = np.abs(ref[keep] - pos0[keep]).max()  # largest displacement
    big = np.abs(ref).max()
    tol = 1e-12 * (move + big) if prec == G.GILA_FP64 else 1e-4 * move + 1e-6 * big
    err = np.abs(got - ref).max(axis=1)
    assert err[keep].max() <= tol
    # leaves may differ only where a rotation was a near-tie
    assert np.quantile(err, 0.999) <= tol


@pytest.mark.parametrize("prec", [G.GILA_FP32, G.GILA_FP64], ids=["fp32", "fp64"])
def test_pipeline_whole_run_quality(prec):
    """A whole pruned layout: edge-length CV and the repulsive/attractive
    ratio of the final full drawing within 2% of the oracle's pipeline."""
    _torch()
    g = I.barabasi_albert(20000, 1, 61)
    pos0 = I.uniform_positions(g.n, 62)
    k, iters = 3, 200
    prm = G.params(k=k, iters=iters, precision=prec)
    ref = O.pipeline(g.n, g.row_ptr, g.col_idx, pos0, k=k, iters=iters)
    with G.Graph.from_inputs(g) as h, G.Pruned(h) as p:
        got = G.gila_layout_pruned_run(p.handle, prm, pos0)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    mo = O.metrics(g.n, g.row_ptr, g.col_idx, krow, kcol, ref)
    torch = _torch()
    dt = torch.float64 if prec == G.GILA_FP64 else torch.float32
    with G.Graph.from_inputs(g) as h:
        mg = G.gila_layout_metrics(h.handle, prm, torch.tensor(got, dtype=dt, device="cuda"))
    for key in ("edge_cv", "rep_att_ratio"):
        assert abs(mg[key] - mo[key]) <= 0.02 * abs(mo[key]), (key, mg[key], mo[key])


def test_pipeline_without_leaves_equals_plain_run():
    """No degree-one vertex: weights are all 1, and the pipeline gives the
    plain layout bit for bit."""
    _torch()
    g = I.tri_mesh(30, 30)
    pos0 = I.uniform_positions(g.n, 71)
    prm = G.params(k=2, iters=20, precision=G.GILA_FP64)
    with G.Graph.from_inputs(g) as h:
        plain = G.gila_layout_run(h.handle, prm, pos0)
    with G.Graph.from_inputs(g) as h, G.Pruned(h) as p:
        assert p.removed == 0
        piped = G.gila_layout_pruned_run(p.handle, prm, pos0)
    assert np.array_equal(plain, piped)


def test_pipeline_star_and_edge():
    _torch()
    g = I.star(12)
    pos0 = I.uniform_positions(g.n, 81)
    with G.Graph.from_inputs(g) as h, G.Pruned(h) as p:
        out = G.gila_layout_pruned_run(p.handle, G.params(k=2, iters=30, d=2.0,
                                                          precision=G.GILA_FP64), pos0)
    assert np.array_equal(out[0], pos0[0])
    r = out[1:] - out[0]
    assert np.allclose(np.hypot(r[:, 0], r[:, 1]), 0.4, rtol=1e-14)
    g = I.path(2)
    with G.Graph.from_inputs(g) as h, G.Pruned(h) as p:
        assert p.kept == 1
        out = G.gila_layout_pruned_run(p.handle, G.params(k=1, iters=5, precision=G.GILA_FP64),
                                       np.array([[1.0, 2.0], [5.0, 5.0]]))
    a = 2 * math.pi * 0.5 / 64
    assert np.allclose(out, [[1.0, 2.0], [1.0 + 0.2 * math.cos(a), 2.0 + 0.2 * math.sin(a)]],
                       rtol=0, atol=1e-15)


def test_pipeline_device_entry_and_empty_graph():
    torch = _torch()
    g = I.random_tree(2000, 91)
    pos0 = I.uniform_positions(g.n, 92)
    prm = G.params(k=2, iters=10, precision=G.GILA_FP32)
    with G.Graph.from_inputs(g) as h, G.Pruned(h) as p:
        host = G.gila_layout_pruned_run(p.handle, prm, pos0)
        x = torch.tensor(pos0, dtype=torch.float32, device="cuda")
        G.gila_layout_pruned_run_device(p.handle, prm, x)
        torch.cuda.synchronize()
        assert np.array_equal(x.double().cpu().numpy(), host)
    e = I.csr_from_edges(0, [], [])
    with G.Graph.from_inputs(e) as h, G.Pruned(h) as p:
        assert p.kept == 0 and p.removed == 0
        out = G.gila_layout_pruned_run(p.handle, prm, np.zeros((0, 2)))
        assert out.shape == (0, 2)
