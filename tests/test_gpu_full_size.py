"""Parity at full size on the benchmark workload: Barabasi-Albert graph,
n = 100,000, m = 3 (299,994 edges), seed 2, placement uniform in
[0, sqrt n]^2, k = 2 and k = 3, driven through the same C-ABI calls the
benchmark times (gila_build_khop, gila_layout_run_device, gila_layout_metrics).

  k-hop lists      bit-exact against the oracle's BFS
  one step         all 100,000 moves, FP32 within 1e-4 and FP64 within 1e-12
                   of the largest move
  whole layout     500 iterations; edge-length CV and repulsive/attractive
                   ratio of the FP32 layout within 2% of the oracle's FP64
                   layout and of the GPU's FP64 layout
"""
import math

import numpy as np
import pytest

import __graft_entry__
import oracle as O
from paper_1606_02162_gb300 import gila as G
from paper_1606_02162_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ba():
    __graft_entry__.build()
    import torch
    torch.cuda.set_device(0)
    g, pos = I.workload("ba100k")
    lists = {k: O.khop(g.n, g.row_ptr, g.col_idx, k) for k in (2, 3)}
    return g, pos, lists


@pytest.mark.parametrize("k", [2, 3])
def test_khop_bit_exact(ba, k):
    g, _, lists = ba
    with G.Graph.from_inputs(g) as h:
        nnz = G.gila_build_khop(h.handle, k)
        krow, kcol = G.gila_khop_export(h.handle)
    okrow, okcol = lists[k]
    assert nnz == okrow[-1]
    assert np.array_equal(krow, okrow)
    assert np.array_equal(kcol, okcol)


@pytest.mark.parametrize("prec,tol", [(G.GILA_FP32, 1e-4), (G.GILA_FP32_COMPENSATED, 1e-4),
                                      (G.GILA_FP64, 1e-12)], ids=["fp32", "fp32c", "fp64"])
@pytest.mark.parametrize("k", [2, 3])
def test_step_all_vertices(ba, k, prec, tol):
    import torch
    g, pos, lists = ba
    okrow, okcol = lists[k]
    t = 0.1 * math.sqrt(g.n)
    dt = torch.float64 if prec == G.GILA_FP64 else torch.float32
    with G.Graph.from_inputs(g) as h:
        p_in = torch.tensor(pos, dtype=dt, device="cuda")
        p_out = torch.empty_like(p_in)
        disp = torch.empty_like(p_in)
        G.gila_layout_step(h.handle, G.params(k=k, precision=prec), t, p_in, p_out, disp)
        torch.cuda.synchronize()
        base = p_in.double().cpu().numpy()
        got = disp.double().cpu().numpy()
    _, odisp = O.step(g.n, g.row_ptr, g.col_idx, okrow, okcol, base, t)
    assert np.abs(got - odisp).max() <= tol * np.abs(odisp).max()


@pytest.mark.parametrize("k", [2, 3])
def test_whole_layout_quality(ba, k):
    import torch
    g, pos, lists = ba
    okrow, okcol = lists[k]
    iters = 500
    res = {}
    for prec in (G.GILA_FP32, G.GILA_FP64):
        dt = torch.float64 if prec == G.GILA_FP64 else torch.float32
        prm = G.params(k=k, iters=iters, precision=prec)
        with G.Graph.from_inputs(g) as h:
            x = torch.tensor(pos, dtype=dt, device="cuda")
            G.gila_layout_run_device(h.handle, prm, x)
            res[prec] = (G.gila_layout_metrics(h.handle, prm, x), x.double().cpu().numpy())
    ref = O.run(g.n, g.row_ptr, g.col_idx, okrow, okcol, pos, iters)
    mo = O.metrics(g.n, g.row_ptr, g.col_idx, okrow, okcol, ref)
    m32, _ = res[G.GILA_FP32]
    m64, _ = res[G.GILA_FP64]
    # the device reductions agree with the oracle's on the same seeded
    # FP32-rounded placement (FP32 placements: edge figures in FP64, k-hop
    # terms in double-float arithmetic, all summed in FP64)
    p0 = pos.astype(np.float32).astype(np.float64)
    mo0 = O.metrics(g.n, g.row_ptr, g.col_idx, okrow, okcol, p0)
    with G.Graph.from_inputs(g) as h:
        m0 = G.gila_layout_metrics(h.handle, G.params(k=k, precision=G.GILA_FP32),
                                   torch.tensor(p0, dtype=torch.float32, device="cuda"))
    for key in mo0:
        assert m0[key] == pytest.approx(mo0[key], rel=1e-11), key
    for key in ("edge_cv", "rep_att_ratio"):
        assert abs(m32[key] - mo[key]) <= 0.02 * abs(mo[key]), (key, m32[key], mo[key])
        assert abs(m32[key] - m64[key]) <= 0.02 * abs(m64[key]), (key, m32[key], m64[key])


@pytest.mark.parametrize("k", [2, 3])
def test_ba_1m_edges_sampled(k):
    """The 1M-edge Barabasi-Albert graph (n = 333,334; the serving stream's
    largest requests), on the blocked path in 14 tiles with short segments:
    sampled k-hop rows exact, and the capped moves (first temperature) of a
    systematic sample of 2,048 vertices and the 16 largest hubs within 1e-4
    of the largest move, against the oracle's step over a k-hop CSR that
    holds only the sample's rows."""
    import torch
    g, pos = I.workload("ba1m")
    deg = np.diff(g.row_ptr)
    sel = np.unique(np.concatenate([np.arange(0, g.n, g.n // 2048, dtype=np.int64)[:2048],
                                    np.argsort(-deg, kind="stable")[:16]]))
    counts, rows = O.khop_rows(g.n, g.row_ptr, g.col_idx, k, sel)
    c = np.zeros(g.n, dtype=np.int64)
    c[sel] = counts
    krow = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(c, out=krow[1:])
    t = 0.1 * np.sqrt(g.n)
    with G.Graph.from_inputs(g) as h:
        G.gila_build_khop(h.handle, k)
        gc, grows = G.gila_khop_export_rows(h.handle, sel)
        assert np.array_equal(gc, counts) and np.array_equal(grows, rows)
        x = torch.tensor(pos, dtype=torch.float32, device="cuda")
        y, disp = torch.empty_like(x), torch.empty_like(x)
        G.gila_profile_enable(h.handle, 2)
        G.gila_layout_step(h.handle, G.params(k=k), t, x, y, disp)
        G.gila_profile_read(h.handle)
        assert G.gila_profile_read_kernel(h.handle)["name"].startswith("blocked_kernel")
        base = x.double().cpu().numpy()
        got = disp.double().cpu().numpy()[sel]
    _, odisp = O.step(g.n, g.row_ptr, g.col_idx, krow, rows, base, t)
    odisp = odisp[sel]
    assert np.abs(got - odisp).max() <= 1e-4 * np.abs(odisp).max()
