"""Parity on the two large graphs at full size, k = 3, through the calls the
benchmark times.

Triangulated mesh 1000 x 1000 (n = 1,000,000, 2,996,001 edges): k-hop lists
bit-exact, one step of all vertices against the oracle, and whole 300-
iteration layouts within 2% of the oracle's in edge-length CV and the
repulsive/attractive ratio.

Chung-Lu, gamma = 2.3, n = 250,000, 1,000,000 edges: about 1.1e10 k-hop
entries (45 GB of ids), beyond what the oracle can build for every vertex.
Checked on sampled outputs the oracle computes one by one (k-hop rows of hubs,
ordinary and isolated vertices; the resultant force of sampled vertices; the
capped moves of a systematic sample of 2,048 vertices and the hubs, in every
precision, in the benchmark's launch configuration) and through properties
that hold at any size (the forces sum to zero; FP32, compensated FP32 and
FP64 layouts agree). The FP64 mode is validated over the first 10 iterations
on a Chung-Lu graph of the same shape that the oracle lays out whole
(n = 20,000, 80,000 edges, k = 3, 1.4e8 k-hop entries), with the position
tiles of the blocked path cut to 2,000 vertices so that it runs in 10 tiles
as the full-size graph does: each GPU step from the oracle's placement of
that iteration within 1e-12 of the largest move.
"""
import math

import numpy as np
import pytest

import __graft_entry__
import oracle as O
from paper_1606_02162_gb300 import gila as G
from paper_1606_02162_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


# --------------------------------------------------------------------- mesh

@pytest.fixture(scope="module")
def mesh():
    _torch()
    __graft_entry__.build()
    g, pos = I.workload("mesh1000")
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 3)
    return g, pos, krow, kcol


def test_mesh_khop_bit_exact(mesh):
    g, _, okrow, okcol = mesh
    with G.Graph.from_inputs(g) as h:
        assert G.gila_build_khop(h.handle, 3) == okrow[-1]
        krow, kcol = G.gila_khop_export(h.handle)
    assert np.array_equal(krow, okrow) and np.array_equal(kcol, okcol)


@pytest.mark.parametrize("prec,tol", [(G.GILA_FP32_COMPENSATED, 1e-4), (G.GILA_FP32, 1e-4),
                                      (G.GILA_FP64, 1e-12)], ids=["fp32c", "fp32", "fp64"])
def test_mesh_step_all_vertices(mesh, prec, tol):
    torch = _torch()
    g, pos, okrow, okcol = mesh
    t = 0.1 * math.sqrt(g.n)
    dt = torch.float64 if prec == G.GILA_FP64 else torch.float32
    with G.Graph.from_inputs(g) as h:
        x = torch.tensor(pos, dtype=dt, device="cuda")
        y, disp = torch.empty_like(x), torch.empty_like(x)
        G.gila_layout_step(h.handle, G.params(k=3, precision=prec), t, x, y, disp)
        base = x.double().cpu().numpy()
        got = disp.double().cpu().numpy()
    _, odisp = O.step(g.n, g.row_ptr, g.col_idx, okrow, okcol, base, t)
    assert np.abs(got - odisp).max() <= tol * np.abs(odisp).max()


def test_mesh_whole_layout_quality(mesh):
    torch = _torch()
    g, pos, okrow, okcol = mesh
    iters = 300
    ref = O.run(g.n, g.row_ptr, g.col_idx, okrow, okcol, pos, iters)
    mo = O.metrics(g.n, g.row_ptr, g.col_idx, okrow, okcol, ref)
    for prec in (G.GILA_FP32_COMPENSATED, G.GILA_FP32):
        with G.Graph.from_inputs(g) as h:
            x = torch.tensor(pos, dtype=torch.float32, device="cuda")
            prm = G.params(k=3, iters=iters, precision=prec)
            G.gila_layout_run_device(h.handle, prm, x)
            m = G.gila_layout_metrics(h.handle, prm, x)
        for key in ("edge_cv", "rep_att_ratio"):
            assert abs(m[key] - mo[key]) <= 0.02 * abs(mo[key]), (prec, key, m[key], mo[key])


# ----------------------------------------------------------------- Chung-Lu

@pytest.fixture(scope="module")
def chunglu():
    _torch()
    __graft_entry__.build()
    g, pos = I.workload("chunglu250k")
    h = G.Graph.from_inputs(g)
    nnz = G.gila_build_khop(h.handle, 3)
    deg = np.diff(g.row_ptr)
    rng = np.random.default_rng(7)
    hubs = np.argsort(-deg, kind="stable")[:6]
    isolated = np.nonzero(deg == 0)[0][:3]
    leaves = np.nonzero(deg == 1)[0][:3]
    rest = rng.choice(g.n, 36, replace=False)
    sel = np.unique(np.concatenate([hubs, isolated, leaves, rest]))
    yield g, pos, h, nnz, sel
    h.close()


def _partial_khop(g, sel, counts, rows):
    """A k-hop CSR holding only the rows of sel (ascending), for the oracle's
    forces of the selected vertices."""
    c = np.zeros(g.n, dtype=np.int64)
    c[sel] = counts
    krow = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(c, out=krow[1:])
    return krow, rows


def test_chunglu_khop_sampled_rows(chunglu):
    g, _, h, nnz, sel = chunglu
    counts, rows = G.gila_khop_export_rows(h.handle, sel)
    ocounts, orows = O.khop_rows(g.n, g.row_ptr, g.col_idx, 3, sel)
    assert np.array_equal(counts, ocounts) and np.array_equal(rows, orows)
    assert nnz > 1e10  # about 1.5e10 entries
    # membership is symmetric: u in N(v) <=> v in N(u), checked on sampled pairs
    off = np.concatenate([[0], np.cumsum(counts)])
    row_of = {int(v): rows[off[i]:off[i + 1]] for i, v in enumerate(sel)}
    for i, v in enumerate(sel):
        for u in sel:
            if u == v:
                continue
            assert (np.searchsorted(row_of[int(v)], u) < len(row_of[int(v)]) and
                    row_of[int(v)][np.searchsorted(row_of[int(v)], u)] == u) == \
                   (np.searchsorted(row_of[int(u)], v) < len(row_of[int(u)]) and
                    row_of[int(u)][np.searchsorted(row_of[int(u)], v)] == v)


@pytest.mark.parametrize("prec,tol", [(G.GILA_FP32_COMPENSATED, 1e-4), (G.GILA_FP32, 1e-4)],
                         ids=["fp32c", "fp32"])
def test_chunglu_forces_sampled_and_sum(chunglu, prec, tol):
    """Uncapped step (t = 1e30, so the move is the force itself) in the
    benchmark's launch configuration (blocked path): sampled forces against
    the oracle, and the sum of all forces against zero."""
    torch = _torch()
    g, pos, h, _, sel = chunglu
    x = torch.tensor(pos, dtype=torch.float32, device="cuda")
    y, disp = torch.empty_like(x), torch.empty_like(x)
    G.gila_layout_step(h.handle, G.params(k=3, precision=prec), 1e30, x, y, disp)
    F = disp.double().cpu().numpy()
    base = x.double().cpu().numpy()
    counts, rows = O.khop_rows(g.n, g.row_ptr, g.col_idx, 3, sel)
    krow, kcol = _partial_khop(g, sel, counts, rows)
    OF = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, base, sel=sel)
    assert np.abs(F[sel] - OF).max() <= tol * np.abs(OF).max()
    # pairwise forces cancel: the total is tiny against the total magnitude
    total = np.abs(F.sum(axis=0)).max()
    assert total <= 1e-5 * np.abs(F).sum()


def test_chunglu_whole_layouts_agree_across_precisions(chunglu):
    """300 iterations (the configuration) in FP32 compensated and FP32, and
    the first 10 in FP64 against FP32 compensated: edge-length CV and the
    repulsive/attractive ratio within 2%."""
    torch = _torch()
    g, pos, h, _, _ = chunglu
    res = {}
    for name, prec, iters in (("fp32c", G.GILA_FP32_COMPENSATED, 300), ("fp32", G.GILA_FP32, 300),
                              ("fp32c10", G.GILA_FP32_COMPENSATED, 10),
                              ("fp64_10", G.GILA_FP64, 10)):
        dt = torch.float64 if prec == G.GILA_FP64 else torch.float32
        x = torch.tensor(pos, dtype=dt, device="cuda")
        prm = G.params(k=3, iters=iters, precision=prec)
        G.gila_layout_run_device(h.handle, prm, x)
        res[name] = G.gila_layout_metrics(h.handle, prm, x)
        assert np.isfinite(x.double().cpu().numpy()).all()
    for a, b in (("fp32", "fp32c"), ("fp64_10", "fp32c10")):
        for key in ("edge_cv", "rep_att_ratio"):
            assert abs(res[a][key] - res[b][key]) <= 0.02 * abs(res[b][key]), \
                (a, b, key, res[a][key], res[b][key])


@pytest.fixture(scope="module")
def chunglu_sample(chunglu):
    """A systematic sample of 2,048 vertices and the 16 largest hubs, with the
    oracle's k-hop rows of exactly those vertices."""
    g, _, _, _, _ = chunglu
    deg = np.diff(g.row_ptr)
    sys_sel = np.arange(0, g.n, g.n // 2048, dtype=np.int64)[:2048]
    hubs = np.argsort(-deg, kind="stable")[:16]
    sel = np.unique(np.concatenate([sys_sel, hubs]))
    counts, rows = O.khop_rows(g.n, g.row_ptr, g.col_idx, 3, sel)
    krow, kcol = _partial_khop(g, sel, counts, rows)
    return sel, krow, kcol


@pytest.mark.parametrize("prec,tol", [(G.GILA_FP32_COMPENSATED, 1e-4), (G.GILA_FP32, 1e-4),
                                      (G.GILA_FP64, 1e-12)], ids=["fp32c", "fp32", "fp64"])
def test_chunglu_capped_moves_sample(chunglu, chunglu_sample, prec, tol):
    """One iteration at the linear schedule's first temperature (0.1 sqrt(n)
    = 50, which caps the hubs) in the benchmark's launch configuration: the
    capped moves of the sample against the oracle's. The oracle's step runs
    on a k-hop CSR that holds only the sample's rows, so only those moves are
    complete and compared."""
    torch = _torch()
    g, pos, h, _, _ = chunglu
    sel, krow, kcol = chunglu_sample
    t = 0.1 * math.sqrt(g.n)
    dt = torch.float64 if prec == G.GILA_FP64 else torch.float32
    x = torch.tensor(pos, dtype=dt, device="cuda")
    y, disp = torch.empty_like(x), torch.empty_like(x)
    G.gila_profile_enable(h.handle, 2)
    G.gila_layout_step(h.handle, G.params(k=3, precision=prec), t, x, y, disp)
    G.gila_profile_read(h.handle)
    assert G.gila_profile_read_kernel(h.handle)["name"].startswith("blocked_kernel")
    G.gila_profile_enable(h.handle, 0)
    got = disp.double().cpu().numpy()[sel]
    base = x.double().cpu().numpy()
    _, odisp = O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, base, t)
    odisp = odisp[sel]
    assert np.abs(got - odisp).max() <= tol * np.abs(odisp).max()
    # the hubs are capped: their move has length t
    capped = np.linalg.norm(odisp, axis=1) > 0.999 * t
    assert capped.sum() >= 8


def test_chunglu_shape_fp64_first_ten_iterations():
    """FP64 mode over the first 10 iterations of a 300-iteration linear
    schedule on a Chung-Lu graph of the configuration's shape, blocked path
    in 10 tiles: every GPU step from the oracle's placement of that
    iteration within 1e-12 of the largest move."""
    torch = _torch()
    __graft_entry__.build()
    g = I.chung_lu(20000, 2.3, 8.0, 80000, 31)
    pos = I.uniform_positions(g.n, 32)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, 3)
    prm = G.params(k=3, iters=300, precision=G.GILA_FP64)
    t0 = 0.1 * math.sqrt(g.n)
    with G.Graph.from_inputs(g) as h:
        G.gila_graph_tune(h.handle, tiled=1, tile_vertices=2000)
        G.gila_profile_enable(h.handle, 2)
        x = pos.copy()
        for i in range(10):
            t = O.temperature(O.SCHED_LINEAR, t0, i, 300)
            assert t == pytest.approx(G.gila_temperature(prm, t0, i), rel=1e-15)
            xin = torch.tensor(x, dtype=torch.float64, device="cuda")
            y, disp = torch.empty_like(xin), torch.empty_like(xin)
            G.gila_layout_step(h.handle, prm, t, xin, y, disp)
            xnext, odisp = O.step(g.n, g.row_ptr, g.col_idx, okrow, okcol, x, t)
            got = disp.cpu().numpy()
            assert np.abs(got - odisp).max() <= 1e-12 * np.abs(odisp).max(), i
            x = xnext
        G.gila_profile_read(h.handle)
        assert G.gila_profile_read_kernel(h.handle)["name"].startswith("blocked_kernel")
