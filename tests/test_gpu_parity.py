"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (element by element on the same seeded inputs):
  k-hop lists        bit-exact (sorted rows, same offsets)
  one step, FP32     max |disp_gpu - disp_oracle| <= 1e-4 max |disp_oracle|
  one step, FP64     max |disp_gpu - disp_oracle| <= 1e-12 max |disp_oracle|
  whole runs         edge-length CV and repulsive/attractive ratio within 2%
The FP32 step is compared from the FP32-rounded placement, so both sides
start from identical coordinates.
"""
import math

import numpy as np
import pytest

import __graft_entry__
import oracle as O
from paper_1606_02162_gb300 import gila as G
from paper_1606_02162_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {G.GILA_FP32: 1e-4, G.GILA_FP32_COMPENSATED: 1e-4, G.GILA_FP64: 1e-12}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    import torch
    torch.cuda.set_device(0)


def _torch():
    import torch
    return torch


def _dt(prec):
    t = _torch()
    return t.float64 if prec in (G.GILA_FP64, G.GILA_FP64_ORDERED) else t.float32


def gpu_quality(g, k, placement, prec, d=1.0, p=2, q=1):
    """Edge-length CV and repulsive/attractive ratio of a placement by the
    library's own FP64 reductions: the GPU's figure of a GPU layout, set
    against the oracle's figure of the oracle's layout."""
    import torch
    dt = torch.float64 if prec in (G.GILA_FP64, G.GILA_FP64_ORDERED) else torch.float32
    with G.Graph.from_inputs(g) as h:
        x = torch.tensor(placement, dtype=dt, device="cuda")
        return G.gila_layout_metrics(h.handle, G.params(k=k, d=d, p=p, q=q, precision=prec), x)


def gpu_khop(g, k):
    with G.Graph.from_inputs(g) as h:
        nnz = G.gila_build_khop(h.handle, k)
        krow, kcol = G.gila_khop_export(h.handle)
    assert nnz == krow[-1]
    return krow, kcol


def gpu_step(g, k, pos, t, prec, d=1.0, p=2, q=1, tune=None):
    torch = _torch()
    with G.Graph.from_inputs(g) as h:
        if tune:
            G.gila_graph_tune(h.handle, **tune)
        p_in = torch.tensor(pos, dtype=_dt(prec), device="cuda")
        p_out = torch.empty_like(p_in)
        disp = torch.empty_like(p_in)
        G.gila_layout_step(h.handle, G.params(k=k, d=d, p=p, q=q, precision=prec), t, p_in, p_out,
                           disp)
        torch.cuda.synchronize()
        return (p_in.double().cpu().numpy(), p_out.double().cpu().numpy(),
                disp.double().cpu().numpy())


KHOP_CASES = [
    ("grid32", lambda: I.grid(32, 32), 2),
    ("mesh60", lambda: I.tri_mesh(60, 60), 3),
    ("ba5k_k2", lambda: I.barabasi_albert(5000, 3, 1), 2),
    ("ba5k_k3", lambda: I.barabasi_albert(5000, 3, 1), 3),
    ("er3k_k4", lambda: I.erdos_renyi(3000, 4.0, 2), 4),
    ("tree2k_k5", lambda: I.random_tree(2000, 3), 5),
    ("cl5k_k2", lambda: I.chung_lu(5000, 2.3, 8.0, 20000, 4), 2),
    ("star2k_k1", lambda: I.star(2000), 1),
    ("star2k_k2", lambda: I.star(2000), 2),
    ("k700_k1", lambda: I.complete(700), 1),
    ("path1k_k7", lambda: I.path(1000), 7),
    ("isolated", lambda: I.csr_from_edges(50, [0, 3, 7], [1, 4, 8]), 3),
    ("noedges", lambda: I.csr_from_edges(10, [], []), 2),
]


@pytest.mark.parametrize("name,maker,k", KHOP_CASES, ids=[c[0] for c in KHOP_CASES])
def test_khop_bit_exact(name, maker, k):
    g = maker()
    krow, kcol = gpu_khop(g, k)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    assert np.array_equal(krow, okrow)
    assert np.array_equal(kcol, okcol)


def test_golden_grid_count():
    krow, _ = gpu_khop(I.grid(32, 32), 2)
    assert krow[-1] == 11652


def test_khop_cache_and_rebuild():
    g = I.barabasi_albert(3000, 3, 5)
    with G.Graph.from_inputs(g) as h:
        n2 = G.gila_build_khop(h.handle, 2)
        a = G.gila_khop_export(h.handle)
        assert G.gila_build_khop(h.handle, 2) == n2
        n3 = G.gila_build_khop(h.handle, 3)
        assert n3 > n2
        assert G.gila_build_khop(h.handle, 2) == n2
        b = G.gila_khop_export(h.handle)
        G.gila_khop_reset(h.handle)
        assert G.gila_graph_info(h.handle)["k_built"] == 0
        assert G.gila_build_khop(h.handle, 2) == n2
        c = G.gila_khop_export(h.handle)
    for x, y in ((a, b), (a, c)):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])


STEP_CASES = [
    ("grid32_k2", lambda: I.grid(32, 32), 2),
    ("ba20k_k2", lambda: I.barabasi_albert(20000, 3, 7), 2),
    ("ba5k_k3", lambda: I.barabasi_albert(5000, 3, 1), 3),
    ("cl20k_k2", lambda: I.chung_lu(20000, 2.3, 8.0, 80000, 3), 2),
    ("mesh100_k3", lambda: I.tri_mesh(100, 100), 3),
    ("star70k_k1", lambda: I.star(70000), 1),
    ("k700_k1", lambda: I.complete(700), 1),
]


@pytest.mark.parametrize("prec", [G.GILA_FP32, G.GILA_FP32_COMPENSATED, G.GILA_FP64],
                         ids=["fp32", "fp32c", "fp64"])
@pytest.mark.parametrize("name,maker,k", STEP_CASES, ids=[c[0] for c in STEP_CASES])
def test_step_parity(name, maker, k, prec):
    g = maker()
    pos = I.uniform_positions(g.n, 11)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    for t in (0.1 * math.sqrt(g.n), 1e30):
        base, new, disp = gpu_step(g, k, pos, t, prec)
        _, odisp = O.step(g.n, g.row_ptr, g.col_idx, okrow, okcol, base, t)
        scale = np.abs(odisp).max()
        err = np.abs(disp - odisp).max()
        assert err <= TOL[prec] * scale, (t, err, scale)
        assert np.array_equal(new, (base.astype(_np_dt(prec)) + disp.astype(_np_dt(prec))).astype(np.float64))


TUNINGS = [
    ("untiled", dict(tiled=0)),
    ("tiled", dict(tiled=1)),
    ("tiled_small_tiles", dict(tiled=1, tile_vertices=1000)),
    ("tiled_small_tiles_ascending", dict(tiled=1, tile_vertices=1000, bank_spread=-1)),
    ("tiled_divergent_steps", dict(tiled=1, tile_vertices=1000, step_schedule=-1)),
    ("untiled_small_classes", dict(tiled=0, small_max=4, warp_max=64, block_max=512, chunk=300)),
]


@pytest.mark.parametrize("prec", [G.GILA_FP32, G.GILA_FP32_COMPENSATED, G.GILA_FP64],
                         ids=["fp32", "fp32c", "fp64"])
@pytest.mark.parametrize("tname,tune", TUNINGS, ids=[t[0] for t in TUNINGS])
@pytest.mark.parametrize("name,maker,k", [
    ("ba20k_k2", lambda: I.barabasi_albert(20000, 3, 7), 2),
    ("cl9k_k3", lambda: I.chung_lu(9001, 2.3, 8.0, 36000, 5), 3),
    ("mesh50_k3", lambda: I.tri_mesh(50, 51), 3),
], ids=["ba20k_k2", "cl9k_k3", "mesh50_k3"])
def test_step_parity_tunings(name, maker, k, tname, tune, prec):
    """Every scheduling (tiled with one or many tiles, untiled with every row
    class populated) matches the oracle within the precision's tolerance."""
    torch = _torch()
    g = maker()
    pos = I.uniform_positions(g.n, 5)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    t = 0.1 * math.sqrt(g.n)
    with G.Graph.from_inputs(g) as h:
        G.gila_graph_tune(h.handle, **tune)
        p_in = torch.tensor(pos, dtype=_dt(prec), device="cuda")
        p_out = torch.empty_like(p_in)
        disp = torch.empty_like(p_in)
        G.gila_layout_step(h.handle, G.params(k=k, precision=prec), t, p_in, p_out, disp)
        torch.cuda.synchronize()
        base = p_in.double().cpu().numpy()
        got = disp.double().cpu().numpy()
    _, odisp = O.step(g.n, g.row_ptr, g.col_idx, okrow, okcol, base, t)
    assert np.abs(got - odisp).max() <= TOL[prec] * np.abs(odisp).max()


def _mesh_with_isolated(r, c, extra):
    g = I.tri_mesh(r, c)
    u = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    keep = u < g.col_idx
    return I.csr_from_edges(g.n + extra, u[keep], g.col_idx[keep])


@pytest.mark.parametrize("prec", [G.GILA_FP32, G.GILA_FP32_COMPENSATED, G.GILA_FP64],
                         ids=["fp32", "fp32c", "fp64"])
@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("tune", [dict(tiled=1), dict(tiled=1, ctas_per_sm=1),
                                  dict(tiled=1, ctas_per_sm=12)], ids=["cps4", "cps1", "cps12"])
def test_step_parity_window_mode(k, prec, tune):
    """Banded ids (a triangulated mesh, then 37 isolated vertices with empty
    rows): every row range gets its own shared-memory window of positions
    (its first id rounded down to a 16-byte boundary), streams its rows'
    16-bit window-relative ids and finishes its rows in the CTA; the
    isolated vertices' ranges have nothing to stream and must not move."""
    torch = _torch()
    g = _mesh_with_isolated(37, 41, 37)
    pos = I.uniform_positions(g.n, 6)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    for t in (0.1 * math.sqrt(g.n), 1e30):
        with G.Graph.from_inputs(g) as h:
            G.gila_graph_tune(h.handle, **tune)
            p_in = torch.tensor(pos, dtype=_dt(prec), device="cuda")
            p_out = torch.empty_like(p_in)
            disp = torch.empty_like(p_in)
            G.gila_layout_step(h.handle, G.params(k=k, precision=prec), t, p_in, p_out, disp)
            torch.cuda.synchronize()
            base = p_in.double().cpu().numpy()
            got = disp.double().cpu().numpy()
        _, odisp = O.step(g.n, g.row_ptr, g.col_idx, okrow, okcol, base, t)
        assert np.abs(got - odisp).max() <= TOL[prec] * np.abs(odisp).max()
        assert (got[g.n - 37:] == 0).all()  # isolated vertices do not move


@pytest.mark.parametrize("prec,tol", [(G.GILA_FP32, 2e-5), (G.GILA_FP64, 1e-13)],
                         ids=["fp32", "fp64"])
@pytest.mark.parametrize("tv", [0, 1200, 960], ids=["tv_default", "tv1200", "tv960"])
def test_bank_spread_only_reorders(prec, tol, tv):
    """The blocked path with each segment's ids ordered for distinct banks
    and with them in ascending order sums the same terms: displacements
    agree to rounding (a lost or repeated id would move them by a whole
    term). n = 30,000 gives tiles of 15,000 (FP32) or about 10,000 (FP64)
    positions by default, 1,200 (tile starts at multiples of the bank
    period) and 938 (starts off it)."""
    torch = _torch()
    g = I.barabasi_albert(30000, 3, 17)
    pos = I.uniform_positions(g.n, 18)
    t = 1e30  # uncapped: the displacement is the force
    out = []
    for spread in (0, -1):
        with G.Graph.from_inputs(g) as h:
            G.gila_graph_tune(h.handle, tiled=1, tile_vertices=tv, bank_spread=spread)
            assert G.gila_graph_get_tuning(h.handle)["bank_spread"] == (1 if spread == 0 else -1)
            p_in = torch.tensor(pos, dtype=_dt(prec), device="cuda")
            p_out, disp = torch.empty_like(p_in), torch.empty_like(p_in)
            G.gila_layout_step(h.handle, G.params(k=3, precision=prec), t, p_in, p_out, disp)
            torch.cuda.synchronize()
            out.append(disp.double().cpu().numpy())
    scale = np.abs(out[1]).max()
    assert np.abs(out[0] - out[1]).max() <= tol * scale


@pytest.mark.parametrize("prec", [G.GILA_FP32, G.GILA_FP32_COMPENSATED, G.GILA_FP64],
                         ids=["fp32", "fp32c", "fp64"])
@pytest.mark.parametrize("spread", [0, -1], ids=["spread", "ascending"])
def test_step_parity_blocks_smaller_than_a_cta(prec, spread):
    """Tiles of 48 positions on a 2,000-vertex graph: blocks of a few
    hundred entries for 1024 threads, so most shares are empty or a single
    step, and rows are cut by many share and warp bounds."""
    g = I.barabasi_albert(2000, 3, 29)
    pos = I.uniform_positions(g.n, 31)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
    t = 1e30
    base, _, disp = gpu_step(g, 2, pos, t, prec,
                             tune=dict(tiled=1, tile_vertices=48, bank_spread=spread))
    _, odisp = O.step(g.n, g.row_ptr, g.col_idx, okrow, okcol, base, t)
    assert np.abs(disp - odisp).max() <= TOL[prec] * np.abs(odisp).max()


@pytest.mark.parametrize("tiled", [0, 1], ids=["plain", "blocked"])
def test_fp64_two_vertex_force_across_scales(tiled):
    """FP64 repulsion uses a Newton-Raphson reciprocal: the force of a single
    edge (k = 1, uncapped) matches the closed form d^2/delta - delta^2/d to
    1e-14 relative at distances from 1e-6 to 1e6."""
    torch = _torch()
    g = I.path(2)
    d = 1.7
    with G.Graph.from_inputs(g) as h:
        G.gila_graph_tune(h.handle, tiled=tiled)
        for delta in (1e-6, 3.3e-3, 0.37, 1.0, 2.9, 29.0, 4.1e3, 1e6):  # away from delta = d
            pos = np.array([[0.25, -1.5], [0.25 + delta * 0.6, -1.5 + delta * 0.8]])
            x = torch.tensor(pos, dtype=torch.float64, device="cuda")
            y, disp = torch.empty_like(x), torch.empty_like(x)
            G.gila_layout_step(h.handle, G.params(k=1, d=d, precision=G.GILA_FP64), 1e300, x, y,
                               disp)
            got = disp.cpu().numpy()
            dl = math.hypot(pos[1, 0] - pos[0, 0], pos[1, 1] - pos[0, 1])
            mag = d * d / dl - dl * dl / d  # along (x_0 - x_1) / delta on vertex 0
            ux, uy = (pos[0] - pos[1]) / dl
            assert got[0] == pytest.approx([mag * ux, mag * uy], rel=1e-14, abs=0), delta
            assert got[1] == pytest.approx([-mag * ux, -mag * uy], rel=1e-14, abs=0), delta


def _np_dt(prec):
    return np.float64 if prec in (G.GILA_FP64, G.GILA_FP64_ORDERED) else np.float32


@pytest.mark.parametrize("p,q", [(3, 2), (0, 1), (1, 3)])
@pytest.mark.parametrize("prec", [G.GILA_FP32, G.GILA_FP64], ids=["fp32", "fp64"])
def test_step_parity_generic_exponents(p, q, prec):
    g = I.barabasi_albert(4000, 3, 9)
    k, d = 2, 1.7
    pos = I.uniform_positions(g.n, 3)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    t = 1e30
    base, _, disp = gpu_step(g, k, pos, t, prec, d=d, p=p, q=q)
    _, odisp = O.step(g.n, g.row_ptr, g.col_idx, okrow, okcol, base, t, d=d, p=p, q=q)
    assert np.abs(disp - odisp).max() <= TOL[prec] * np.abs(odisp).max()


@pytest.mark.parametrize("p,q", [(3, 2), (0, 1), (1, 0), (2, 3)])
@pytest.mark.parametrize("prec", [G.GILA_FP32, G.GILA_FP32_COMPENSATED, G.GILA_FP64],
                         ids=["fp32", "fp32c", "fp64"])
def test_step_parity_generic_exponents_blocked(p, q, prec):
    """The generic force model on the blocked path (tiles of 998 positions,
    so segments of every length and their padding to 4 entries occur): q = 0
    and q = 1 are where a padding entry's far position would add a visible
    term if the model did not cut it."""
    g = I.barabasi_albert(6000, 3, 19)
    k, d = 3, 1.3
    pos = I.uniform_positions(g.n, 23)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    t = 1e30
    base, _, disp = gpu_step(g, k, pos, t, prec, d=d, p=p, q=q,
                             tune=dict(tiled=1, tile_vertices=998))
    _, odisp = O.step(g.n, g.row_ptr, g.col_idx, okrow, okcol, base, t, d=d, p=p, q=q)
    assert np.abs(disp - odisp).max() <= TOL[prec] * np.abs(odisp).max()


@pytest.mark.parametrize("name,maker,k", [
    ("grid32_k2", lambda: I.grid(32, 32), 2),
    ("ba20k_k3", lambda: I.barabasi_albert(20000, 3, 4), 3),
])
def test_fp64_first_ten_iterations(name, maker, k):
    """FP64 mode over the first 10 iterations of a linear-cooling run: at each
    iteration both sides step from the oracle's placement (identical
    positions) and the moves agree within 1e-12 of the largest move. The
    free-running trajectories are also followed: rounding-order differences
    of one ulp grow with the dynamics (about 3x per iteration on the grid),
    so they are held to a looser bound that states that growth."""
    torch = _torch()
    g = maker()
    pos = I.uniform_positions(g.n, 1)
    iters = 100
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    prm = G.params(k=k, iters=iters, precision=G.GILA_FP64)
    t0 = 0.1 * math.sqrt(g.n)
    with G.Graph.from_inputs(g) as h:
        a = torch.tensor(pos, dtype=torch.float64, device="cuda")
        b = torch.empty_like(a)
        free_a = a.clone()
        free_b = torch.empty_like(a)
        disp = torch.empty_like(a)
        ref = pos.copy()
        for i in range(10):
            t = G.gila_temperature(prm, t0, i)
            assert t == O.temperature(O.SCHED_LINEAR, t0, i, iters)
            a.copy_(torch.from_numpy(ref))
            G.gila_layout_step(h.handle, prm, t, a, b, disp)
            G.gila_layout_step(h.handle, prm, t, free_a, free_b)
            ref, odisp = O.step(g.n, g.row_ptr, g.col_idx, okrow, okcol, ref, t)
            scale = np.abs(odisp).max()
            assert np.abs(disp.cpu().numpy() - odisp).max() <= 1e-12 * scale, i
            free_a, free_b = free_b, free_a
            drift = np.abs(free_a.cpu().numpy() - ref).max()
            assert drift <= 1e-15 * np.abs(ref).max() * 8.0 ** (i + 1), (i, drift)


def test_run_device_equals_step_loop():
    torch = _torch()
    g = I.barabasi_albert(3000, 3, 2)
    pos = I.uniform_positions(g.n, 4)
    for prec in (G.GILA_FP32, G.GILA_FP64):
        prm = G.params(k=2, iters=7, precision=prec)
        with G.Graph.from_inputs(g) as h:
            x = torch.tensor(pos, dtype=_dt(prec), device="cuda")
            G.gila_layout_run_device(h.handle, prm, x)
            a = torch.tensor(pos, dtype=_dt(prec), device="cuda")
            b = torch.empty_like(a)
            t0 = 0.1 * math.sqrt(g.n)
            for i in range(7):
                G.gila_layout_step(h.handle, prm, G.gila_temperature(prm, t0, i), a, b)
                a, b = b, a
            torch.cuda.synchronize()
            assert torch.equal(x, a)
            host = G.gila_layout_run(h.handle, prm, pos)
            want = a.double().cpu().numpy()
            assert np.array_equal(host, want)


def test_determinism():
    g = I.chung_lu(30000, 2.3, 8.0, 120000, 8)
    pos = I.uniform_positions(g.n, 2)
    for prec in (G.GILA_FP32, G.GILA_FP32_COMPENSATED, G.GILA_FP64):
        prm = G.params(k=2, iters=20, precision=prec)
        outs = []
        for _ in range(2):
            with G.Graph.from_inputs(g) as h:
                outs.append(G.gila_layout_run(h.handle, prm, pos))
        assert np.array_equal(outs[0], outs[1])


def test_whole_run_grid_fp64_ordered_bit_exact():
    """32x32 grid, k=2, d=1, 100 iterations, linear cooling from 0.1 sqrt(n),
    FP64 in the ordered validation mode: the whole trajectory reproduces the
    oracle's bit for bit, so the quality figures agree exactly."""
    torch = _torch()
    g = I.grid(32, 32)
    pos = I.uniform_positions(g.n, 1)
    prm = G.params(k=2, iters=100, precision=G.GILA_FP64_ORDERED)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
    ref = O.run(g.n, g.row_ptr, g.col_idx, okrow, okcol, pos, 100)
    mo = O.metrics(g.n, g.row_ptr, g.col_idx, okrow, okcol, ref)
    with G.Graph.from_inputs(g) as h:
        out = G.gila_layout_run(h.handle, prm, pos)
        m = G.gila_layout_metrics(h.handle, prm, torch.tensor(out, device="cuda"))
    assert np.array_equal(out, ref)
    for key in mo:
        assert m[key] == pytest.approx(mo[key], rel=1e-12), key


@pytest.mark.parametrize("prec", [G.GILA_FP64, G.GILA_FP32], ids=["fp64", "fp32"])
def test_whole_run_grid_ensemble(prec):
    """The same grid run in the fast modes. A one-ulp change of a single
    coordinate already moves the oracle's own 100-iteration layout by several
    units and its edge-length CV by up to 7%, so single runs are compared
    through the mean over 32 seeded placements (seed-to-seed spread of the
    CV about 3%, of the ratio about 1%): both means within 2%."""
    g = I.grid(32, 32)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
    prm = G.params(k=2, iters=100, precision=prec)
    got, want = [], []
    with G.Graph.from_inputs(g) as h:
        for s in range(1, 33):
            pos = I.uniform_positions(g.n, s)
            out = G.gila_layout_run(h.handle, prm, pos)
            ref = O.run(g.n, g.row_ptr, g.col_idx, okrow, okcol,
                        pos.astype(np.float32).astype(np.float64) if prec == G.GILA_FP32 else pos,
                        100)
            got.append(gpu_quality(g, 2, out, prec))
            want.append(O.metrics(g.n, g.row_ptr, g.col_idx, okrow, okcol, ref))
    for key in ("edge_cv", "rep_att_ratio"):
        a = np.mean([m[key] for m in got])
        b = np.mean([m[key] for m in want])
        assert abs(a - b) <= 0.02 * abs(b), (key, a, b)


@pytest.mark.parametrize("name,maker,k", STEP_CASES, ids=[c[0] for c in STEP_CASES])
def test_ordered_step_bit_exact(name, maker, k):
    g = maker()
    pos = I.uniform_positions(g.n, 11)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    for t in (0.1 * math.sqrt(g.n), 1e30):
        base, new, disp = gpu_step(g, k, pos, t, G.GILA_FP64_ORDERED)
        onew, odisp = O.step(g.n, g.row_ptr, g.col_idx, okrow, okcol, base, t)
        assert np.array_equal(disp, odisp)
        assert np.array_equal(new, onew)
    # generic exponents and ideal length
    base, new, disp = gpu_step(g, k, pos, 1e30, G.GILA_FP64_ORDERED, d=1.7, p=3, q=2)
    _, odisp = O.step(g.n, g.row_ptr, g.col_idx, okrow, okcol, base, 1e30, d=1.7, p=3, q=2)
    assert np.array_equal(disp, odisp)


@pytest.mark.parametrize("prec", [G.GILA_FP32, G.GILA_FP32_COMPENSATED], ids=["fp32", "fp32c"])
def test_whole_run_ba_fp32_quality(prec):
    g = I.barabasi_albert(20000, 3, 2)
    pos = I.uniform_positions(g.n, 2)
    k, iters = 2, 100
    prm = G.params(k=k, iters=iters, precision=prec)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    ref = O.run(g.n, g.row_ptr, g.col_idx, okrow, okcol, pos.astype(np.float32).astype(np.float64),
                iters)
    mo = O.metrics(g.n, g.row_ptr, g.col_idx, okrow, okcol, ref)
    with G.Graph.from_inputs(g) as h:
        out = G.gila_layout_run(h.handle, prm, pos)
    mg = gpu_quality(g, k, out, prec)
    for key in ("edge_cv", "rep_att_ratio"):
        assert abs(mg[key] - mo[key]) <= 0.02 * abs(mo[key]), (key, mg[key], mo[key])


def test_metrics_kernel_matches_oracle():
    torch = _torch()
    g = I.barabasi_albert(8000, 3, 6)
    pos = I.uniform_positions(g.n, 9)
    for p, q in ((2, 1), (3, 2)):
        prm = G.params(k=2, d=1.3, p=p, q=q, precision=G.GILA_FP64)
        okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
        mo = O.metrics(g.n, g.row_ptr, g.col_idx, okrow, okcol, pos, d=1.3, p=p, q=q)
        with G.Graph.from_inputs(g) as h:
            m = G.gila_layout_metrics(h.handle, prm, torch.tensor(pos, device="cuda"))
        for key in mo:
            assert m[key] == pytest.approx(mo[key], rel=1e-11), key


def test_metrics_fp32_placement_matches_oracle():
    """FP32 placements: the edge figures are taken in FP64 and each pair's
    k-hop term in double-float arithmetic (relative error about 1e-13 per
    term), all summed in FP64, so every figure agrees with the oracle on the
    same (FP32-rounded) placement to 1e-11."""
    torch = _torch()
    g = I.barabasi_albert(8000, 3, 6)
    pos = I.uniform_positions(g.n, 9).astype(np.float32).astype(np.float64)
    for p, q in ((2, 1), (3, 2)):
        prm = G.params(k=2, d=1.3, p=p, q=q, precision=G.GILA_FP32)
        okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
        mo = O.metrics(g.n, g.row_ptr, g.col_idx, okrow, okcol, pos, d=1.3, p=p, q=q)
        with G.Graph.from_inputs(g) as h:
            m = G.gila_layout_metrics(h.handle, prm,
                                      torch.tensor(pos, dtype=torch.float32, device="cuda"))
        for key in mo:
            assert m[key] == pytest.approx(mo[key], rel=1e-11), key


def test_layout_run_metrics_output():
    """gila_layout_run's optional metrics equal gila_layout_metrics of the
    placement it returns."""
    torch = _torch()
    g = I.barabasi_albert(3000, 3, 8)
    pos = I.uniform_positions(g.n, 10)
    for prec, dt in ((G.GILA_FP64, torch.float64), (G.GILA_FP32, torch.float32)):
        prm = G.params(k=2, iters=20, precision=prec)
        with G.Graph.from_inputs(g) as h:
            out, m = G.gila_layout_run(h.handle, prm, pos, metrics=True)
            m2 = G.gila_layout_metrics(h.handle, prm, torch.tensor(out, dtype=dt, device="cuda"))
        for key in m:
            assert m[key] == pytest.approx(m2[key], rel=1e-12), key
    with G.Graph.from_inputs(I.path(1)) as h:
        out, m = G.gila_layout_run(h.handle, G.params(iters=3), np.array([[0.5, 0.25]]),
                                   metrics=True)
        assert m["edge_cv"] == 0.0 and m["rep_total"] == 0.0


def test_geometric_schedule_run():
    g = I.grid(20, 12)
    pos = I.uniform_positions(g.n, 5) * np.array([1.0, 0.5])
    prm = G.params(k=2, iters=15, schedule=G.GILA_COOL_GEOMETRIC, precision=G.GILA_FP64, d=1.2)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
    ref = O.run(g.n, g.row_ptr, g.col_idx, okrow, okcol, pos, 15, d=1.2, schedule=O.SCHED_GEOM)
    with G.Graph.from_inputs(g) as h:
        out = G.gila_layout_run(h.handle, prm, pos)
    assert np.abs(out - ref).max() <= 1e-9 * np.abs(ref).max()


def test_edge_cases():
    torch = _torch()
    # no vertices
    with G.Graph(0, np.zeros(1, np.int64), np.zeros(0, np.int32)) as h:
        assert G.gila_build_khop(h.handle, 2) == 0
        out = G.gila_layout_run(h.handle, G.params(iters=3), np.zeros((0, 2)))
        assert out.shape == (0, 2)
    # one vertex, no edges: nothing moves
    g = I.csr_from_edges(1, [], [])
    with G.Graph.from_inputs(g) as h:
        out = G.gila_layout_run(h.handle, G.params(iters=3), np.array([[0.5, 0.25]]))
        assert np.array_equal(out, [[0.5, 0.25]])
    # all vertices on one point: every pair is at distance 0 and contributes nothing
    g = I.complete(5)
    with G.Graph.from_inputs(g) as h:
        pos = np.ones((5, 2))
        for prec in (G.GILA_FP32, G.GILA_FP64):
            out = G.gila_layout_run(h.handle, G.params(k=1, iters=4, precision=prec), pos)
            assert np.array_equal(out, pos)
    # zero temperature: nothing moves
    g = I.barabasi_albert(500, 2, 1)
    pos = I.uniform_positions(g.n, 1)
    base, new, disp = gpu_step(g, 2, pos, 0.0, G.GILA_FP64)
    assert np.array_equal(new, base) and not disp.any()
    # bad arguments come back as GILA_EINVAL, not a crash
    with G.Graph.from_inputs(g) as h:
        x = torch.tensor(pos, device="cuda")
        for bad in (dict(k=0), dict(d=0.0), dict(p=9), dict(precision=7), dict(iters=-1)):
            with pytest.raises(G.GilaError) as e:
                G.gila_layout_run_device(h.handle, G.params(**bad), x)
            assert e.value.status == G.GILA_EINVAL
        with pytest.raises(G.GilaError):
            G.gila_layout_step(h.handle, G.params(), 1.0, x, x)


def test_graph_create_flags():
    # a CSR with a self-loop, a repeat and a missing reverse entry
    row = np.array([0, 3, 4, 5], dtype=np.int64)
    col = np.array([0, 1, 1, 2, 1], dtype=np.int32)
    with pytest.raises(G.GilaError) as e:
        G.gila_graph_create(3, row, col, G.GILA_GRAPH_VALIDATE)
    assert e.value.status == G.GILA_EINVAL
    h = G.gila_graph_create(3, row, col, G.GILA_GRAPH_SIMPLIFY)
    try:
        info = G.gila_graph_info(h)
        assert info["nnz_adj"] == 4  # edges 0-1 and 1-2, both directions
        G.gila_build_khop(h, 1)
        krow, kcol = G.gila_khop_export(h)
        assert krow.tolist() == [0, 1, 3, 4] and kcol.tolist() == [1, 0, 2, 1]
    finally:
        G.gila_graph_destroy(h)


@pytest.mark.parametrize("name,maker,k,tune", [
    ("ba_tiles", lambda: I.barabasi_albert(12000, 3, 21), 2, dict(tiled=1, tile_vertices=2000)),
    ("ba_tiles_k3", lambda: I.barabasi_albert(6000, 3, 22), 3, dict(tiled=1, tile_vertices=1000)),
    ("mesh_windows", lambda: I.tri_mesh(70, 60), 3, dict(tiled=1)),
], ids=["ba_tiles", "ba_tiles_k3", "mesh_windows"])
@pytest.mark.parametrize("pq", [(2, 1), (3, 2)], ids=["fr", "p3q2"])
def test_metrics_over_blocked_plan_match_oracle(name, maker, k, tune, pq):
    """Once a graph has a blocked plan (FP32), its repulsive total is summed
    over the plan's shared-memory position tiles or windows (each unordered
    pair from its smaller end): every figure within 1e-11 of the oracle on
    the same seeded FP32-rounded placement, as on the unplanned path."""
    torch = _torch()
    g = maker()
    p, q = pq
    pos = I.uniform_positions(g.n, 31).astype(np.float32).astype(np.float64)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    mo = O.metrics(g.n, g.row_ptr, g.col_idx, okrow, okcol, pos, d=1.3, p=p, q=q)
    prm = G.params(k=k, d=1.3, p=p, q=q, precision=G.GILA_FP32)
    with G.Graph.from_inputs(g) as h:
        G.gila_graph_tune(h.handle, **tune)
        x = torch.tensor(pos, dtype=torch.float32, device="cuda")
        y, disp = torch.empty_like(x), torch.empty_like(x)
        G.gila_profile_enable(h.handle, 2)
        G.gila_layout_step(h.handle, prm, 0.5, x, y, disp)  # builds the plan
        G.gila_profile_read(h.handle)
        assert G.gila_profile_read_kernel(h.handle)["name"].startswith("blocked_kernel")
        m = G.gila_layout_metrics(h.handle, prm, x)
    for key in mo:
        assert m[key] == pytest.approx(mo[key], rel=1e-11), key
