"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each check uses an independent
route (shortest paths from scipy, offset-counting closed forms, hand-worked
forces, the potential whose gradient the forces are, exact symmetries).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1606_02162_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold_rows(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- k-hop sets

def _brute_khop(g, k):
    """N_v(k) from all-pairs shortest paths (scipy), independent of BFS code."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path
    A = csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    D = shortest_path(A, unweighted=True, directed=False)
    rows = []
    for v in range(g.n):
        rows.append(sorted(int(u) for u in np.nonzero((D[v] >= 1) & (D[v] <= k))[0]))
    return rows


def _as_rows(krow, kcol):
    return [kcol[krow[v]:krow[v + 1]].tolist() for v in range(len(krow) - 1)]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("maker", [
    lambda: I.erdos_renyi(60, 3.0, 11),
    lambda: I.barabasi_albert(70, 2, 5),
    lambda: I.random_tree(50, 9),
    lambda: I.tri_mesh(6, 7),
    lambda: I.chung_lu(80, 2.3, 3.0, 120, 4),
])
def test_khop_matches_shortest_paths(maker, k):
    g = maker()
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    assert _as_rows(krow, kcol) == _brute_khop(g, k)


def _grid_closed_form(R, C, k):
    # grid distance is the L1 distance of (row, col) offsets
    tot = 0
    for a in range(-(R - 1), R):
        for b in range(-(C - 1), C):
            if 1 <= abs(a) + abs(b) <= k:
                tot += (R - abs(a)) * (C - abs(b))
    return tot


def _hexdist(a, b):
    # distance in the triangulated grid with (i,j)-(i+1,j+1) diagonals
    return max(abs(a), abs(b)) if a * b >= 0 else abs(a) + abs(b)


def _mesh_closed_form(R, C, k):
    tot = 0
    for a in range(-(R - 1), R):
        for b in range(-(C - 1), C):
            if 1 <= _hexdist(a, b) <= k:
                tot += (R - abs(a)) * (C - abs(b))
    return tot


@pytest.mark.parametrize("R,C", [(5, 7), (9, 4), (12, 12)])
@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_grid_and_mesh_counts_closed_form(R, C, k):
    g = I.grid(R, C)
    krow, _ = O.khop(g.n, g.row_ptr, g.col_idx, k)
    assert krow[-1] == _grid_closed_form(R, C, k)
    m = I.tri_mesh(R, C)
    krow, _ = O.khop(m.n, m.row_ptr, m.col_idx, k)
    assert krow[-1] == _mesh_closed_form(R, C, k)


def test_golden_counts():
    gold = {r[0]: (int(r[1]), int(r[2])) for r in _gold_rows("khop_counts.txt")}
    g = I.grid(32, 32)
    k, val = gold["grid32x32_total"]
    krow, _ = O.khop(g.n, g.row_ptr, g.col_idx, k)
    assert krow[-1] == val == _grid_closed_form(32, 32, 2)
    k, val = gold["trimesh_interior"]
    m = I.tri_mesh(11, 11)
    counts, _ = O.khop_rows(m.n, m.row_ptr, m.col_idx, k, [5 * 11 + 5])
    assert counts[0] == val


def test_khop_special_graphs():
    n = 9
    p = I.path(n)
    for k in (1, 2, 3):
        krow, kcol = O.khop(n, p.row_ptr, p.col_idx, k)
        for v in range(n):
            want = [u for u in range(max(0, v - k), min(n, v + k + 1)) if u != v]
            assert kcol[krow[v]:krow[v + 1]].tolist() == want
    s = I.star(8)
    krow, kcol = O.khop(8, s.row_ptr, s.col_idx, 1)
    assert kcol[krow[0]:krow[1]].tolist() == list(range(1, 8))
    assert all(kcol[krow[v]:krow[v + 1]].tolist() == [0] for v in range(1, 8))
    krow, kcol = O.khop(8, s.row_ptr, s.col_idx, 2)
    for v in range(8):
        assert kcol[krow[v]:krow[v + 1]].tolist() == [u for u in range(8) if u != v]
    c = I.complete(6)
    krow, kcol = O.khop(6, c.row_ptr, c.col_idx, 1)
    assert krow[-1] == 30
    # isolated vertices and the empty graph
    g = I.csr_from_edges(5, [0], [1])
    krow, kcol = O.khop(5, g.row_ptr, g.col_idx, 3)
    assert krow.tolist() == [0, 1, 2, 2, 2, 2]


def test_khop_symmetric():
    g = I.barabasi_albert(200, 3, 7)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
    pairs = set()
    for v in range(g.n):
        for u in kcol[krow[v]:krow[v + 1]]:
            pairs.add((v, int(u)))
    assert all((u, v) in pairs for (v, u) in pairs)


# ---------------------------------------------------------------- forces

def test_two_vertex_closed_form():
    g = I.path(2)
    krow, kcol = O.khop(2, g.row_ptr, g.col_idx, 1)
    for d in (1.0, 2.5, 48.2842712474619):
        for delta in (0.5, 1.0, 3.0):
            pos = np.array([[0.0, 0.0], [delta * d, 0.0]])
            F = O.forces(2, g.row_ptr, g.col_idx, krow, kcol, pos, d=d)
            dl = delta * d
            want = dl * dl / d - d * d / dl  # attraction minus repulsion, toward +x
            assert F[0, 0] == pytest.approx(want, rel=1e-14, abs=1e-12 * d)
            assert F[1, 0] == pytest.approx(-want, rel=1e-14, abs=1e-12 * d)
            assert F[0, 1] == 0.0 and F[1, 1] == 0.0
        # equilibrium at the ideal distance: d^2/delta = delta^2/d  <=>  delta = d
        pos = np.array([[0.0, 0.0], [d, 0.0]])
        F = O.forces(2, g.row_ptr, g.col_idx, krow, kcol, pos, d=d)
        assert abs(F[0, 0]) <= 1e-14 * d


def test_path3_hand_forces():
    gold = _gold_rows("path3_forces.txt")
    g = I.path(3)
    pos = np.array([[0.0, 0.0], [1.0, 0.0], [3.0, 0.0]])
    for k in (1, 2):
        krow, kcol = O.khop(3, g.row_ptr, g.col_idx, k)
        F = O.forces(3, g.row_ptr, g.col_idx, krow, kcol, pos)
        for r in gold:
            if int(r[0]) == k:
                v = int(r[1])
                assert F[v, 0] == pytest.approx(float(r[2]), abs=1e-15)
                assert F[v, 1] == pytest.approx(float(r[3]), abs=1e-15)


def _potential(g, krow, kcol, pos, d, p, q):
    """Energy whose negative gradient is the FR force field of Section 3.1:
    attraction delta^(p+1)/((p+1) d) per edge; repulsion -d^2 ln(delta)
    (q = 1) or d^2 delta^(1-q)/(q-1) per unordered k-hop pair."""
    U = 0.0
    eu, ev = g.edge_list()
    dl = np.hypot(*(pos[eu] - pos[ev]).T)
    U += np.sum(dl ** (p + 1)) / ((p + 1) * d)
    src = np.repeat(np.arange(g.n), np.diff(krow))
    keep = src < kcol
    a, b = src[keep], kcol[keep].astype(np.int64)
    dl = np.hypot(*(pos[a] - pos[b]).T)
    if q == 1:
        U += -d * d * np.sum(np.log(dl))
    else:
        U += d * d * np.sum(dl ** (1 - q)) / (q - 1)
    return U


@pytest.mark.parametrize("p,q", [(2, 1), (0, 1), (3, 2), (1, 3)])
@pytest.mark.parametrize("k", [1, 2])
def test_force_is_minus_energy_gradient(p, q, k):
    g = I.erdos_renyi(40, 3.0, 3)
    pos = I.uniform_positions(g.n, 17)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    d = 1.3
    F = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, d=d, p=p, q=q)
    h = 1e-6
    G = np.zeros_like(F)
    for u in range(g.n):
        for c in range(2):
            pp = pos.copy(); pp[u, c] += h
            pm = pos.copy(); pm[u, c] -= h
            G[u, c] = -(_potential(g, krow, kcol, pp, d, p, q)
                        - _potential(g, krow, kcol, pm, d, p, q)) / (2 * h)
    scale = np.abs(F).max()
    assert np.abs(F - G).max() <= 2e-6 * scale


def test_force_sum_vanishes():
    g = I.barabasi_albert(300, 3, 1)
    pos = I.uniform_positions(g.n, 5)
    for k in (1, 2, 3):
        krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
        F = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos)
        assert np.abs(F.sum(axis=0)).max() <= 1e-11 * np.abs(F).sum()


def test_k_at_diameter_is_all_pairs_fr():
    # Section 4.5 vs Section 3.1: once k reaches the diameter every vertex
    # repels every other one, which is the all-pairs FR force.
    g = I.random_tree(25, 2)
    pos = I.uniform_positions(g.n, 8)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 25)
    assert krow[-1] == g.n * (g.n - 1)
    allrow = np.arange(0, g.n * (g.n - 1) + 1, g.n - 1, dtype=np.int64)
    allcol = np.array([u for v in range(g.n) for u in range(g.n) if u != v], dtype=np.int32)
    Fk = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, d=0.7)
    Fa = O.forces(g.n, g.row_ptr, g.col_idx, allrow, allcol, pos, d=0.7)
    assert np.array_equal(Fk, Fa)
    # and both agree with the gradient of the all-pairs potential
    F_pot = np.zeros_like(Fa)
    h = 1e-6
    for u in range(g.n):
        for c in range(2):
            pp = pos.copy(); pp[u, c] += h
            pm = pos.copy(); pm[u, c] -= h
            F_pot[u, c] = -(_potential(g, allrow, allcol, pp, 0.7, 2, 1)
                            - _potential(g, allrow, allcol, pm, 0.7, 2, 1)) / (2 * h)
    assert np.abs(Fa - F_pot).max() <= 2e-6 * np.abs(Fa).max()


def test_exact_symmetries():
    g = I.barabasi_albert(150, 2, 4)
    pos = I.uniform_positions(g.n, 6)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
    F = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, d=1.0)
    # quarter turn (x, y) -> (-y, x) is exact in floating point
    rot = np.stack([-pos[:, 1], pos[:, 0]], axis=1)
    Fr = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, rot, d=1.0)
    assert np.array_equal(Fr, np.stack([-F[:, 1], F[:, 0]], axis=1))
    # mirror y -> -y
    mir = pos * np.array([1.0, -1.0])
    Fm = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, mir, d=1.0)
    assert np.array_equal(Fm, F * np.array([1.0, -1.0]))
    # scaling lengths and d by 2 scales the forces by 2, exactly (p=2, q=1)
    F2 = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, 2 * pos, d=2.0)
    assert np.array_equal(F2, 2 * F)
    # translation: same forces up to rounding
    Ft = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos + 3.25, d=1.0)
    assert np.abs(Ft - F).max() <= 1e-9 * np.abs(F).max()


def test_relabelling_equivariance():
    g = I.erdos_renyi(120, 3.0, 21)
    pos = I.uniform_positions(g.n, 2)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 3)
    F = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos)
    perm = np.random.default_rng(0).permutation(g.n)  # new id of old vertex
    eu, ev = g.edge_list()
    h = I.csr_from_edges(g.n, perm[eu], perm[ev])
    pos_h = np.empty_like(pos); pos_h[perm] = pos
    kr2, kc2 = O.khop(h.n, h.row_ptr, h.col_idx, 3)
    F2 = O.forces(h.n, h.row_ptr, h.col_idx, kr2, kc2, pos_h)
    assert np.abs(F2[perm] - F).max() <= 1e-12 * np.abs(F).max()


# ---------------------------------------------------------------- the move

def test_step_is_synchronous_and_capped():
    g = I.barabasi_albert(200, 3, 9)
    pos = I.uniform_positions(g.n, 3)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
    F = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos)
    norms = np.hypot(F[:, 0], F[:, 1])
    t = float(np.median(norms))
    new, disp = O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, t)
    # every move is computed from the old placement (Jacobi)
    big = norms > t
    assert big.any() and (~big).any()
    assert np.allclose(np.hypot(disp[big, 0], disp[big, 1]), t, rtol=1e-14)
    assert np.allclose(disp[big], F[big] * (t / norms[big])[:, None], rtol=1e-14, atol=0)
    assert np.array_equal(disp[~big], F[~big])
    assert np.array_equal(new, pos + disp)
    # a cold system does not move
    new0, disp0 = O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, 0.0)
    assert np.array_equal(new0, pos) and not disp0.any()


def test_zero_force_and_coincident_pairs():
    g = I.path(2)
    krow, kcol = O.khop(2, g.row_ptr, g.col_idx, 1)
    pos = np.array([[1.0, 1.0], [1.0, 1.0]])
    F = O.forces(2, g.row_ptr, g.col_idx, krow, kcol, pos)
    assert not F.any()
    new, disp = O.step(2, g.row_ptr, g.col_idx, krow, kcol, pos, 5.0)
    assert np.array_equal(new, pos)


def test_temperature_schedules():
    for i in range(10):
        assert O.temperature(O.SCHED_LINEAR, 3.2, i, 10) == pytest.approx(3.2 * (10 - i) / 10, rel=1e-15)
        assert O.temperature(O.SCHED_GEOM, 2.0, i, 10) == pytest.approx(2.0 * 0.93 ** i, rel=1e-14)
    pos = np.array([[0.0, 0.0], [4.0, 1.0], [2.0, 2.0]])
    assert O.default_t0(O.SCHED_LINEAR, 100, 1.0, np.zeros((100, 2))) == pytest.approx(1.0)
    # frame 4 wide, 2 high -> aspect 0.5 -> sqrt(3 * 1 / 0.5)
    assert O.default_t0(O.SCHED_GEOM, 3, 1.0, pos) == pytest.approx(math.sqrt(6.0))


def test_single_edge_settles_at_ideal_length():
    g = I.path(2)
    krow, kcol = O.khop(2, g.row_ptr, g.col_idx, 1)
    pos0 = np.array([[0.0, 0.0], [3.0, 0.0]])
    iters, t0 = 200, 0.5
    out = O.run(2, g.row_ptr, g.col_idx, krow, kcol, pos0, iters, d=1.0, t0=t0)
    dl = np.hypot(*(out[1] - out[0]))
    # the capped move bounds the final error by the last two temperatures
    assert abs(dl - 1.0) <= 2 * 2 * t0 / iters
    assert out[0, 1] == 0.0 and out[1, 1] == 0.0


def test_metrics_closed_forms():
    c = I.cycle(4)
    for L, d in ((2.0, 1.0), (2.0, 1.5), (0.75, 3.0)):
        pos = np.array([[0, 0], [L, 0], [L, L], [0, L]], dtype=float)
        krow, kcol = O.khop(4, c.row_ptr, c.col_idx, 1)
        m = O.metrics(4, c.row_ptr, c.col_idx, krow, kcol, pos, d=d)
        assert m["edge_cv"] == 0.0 and m["edge_mean"] == L
        assert m["rep_total"] == pytest.approx(4 * d * d / L, rel=1e-15)
        assert m["att_total"] == pytest.approx(4 * L * L / d, rel=1e-15)
        assert m["rep_att_ratio"] == pytest.approx(d ** 3 / L ** 3, rel=1e-14)
        krow, kcol = O.khop(4, c.row_ptr, c.col_idx, 2)
        m = O.metrics(4, c.row_ptr, c.col_idx, krow, kcol, pos, d=d)
        rep = 4 * d * d / L + 2 * d * d / (L * math.sqrt(2))
        att = 4 * L * L / d
        assert m["rep_att_ratio"] == pytest.approx(rep / att, rel=1e-14)
        # generic exponents: |f^r| = d^2/delta^q, |f^a| = delta^p/d
        m = O.metrics(4, c.row_ptr, c.col_idx, krow, kcol, pos, d=d, p=3, q=2)
        rep = 4 * d * d / L ** 2 + 2 * d * d / (2 * L * L)
        assert m["rep_total"] == pytest.approx(rep, rel=1e-14)
        assert m["att_total"] == pytest.approx(4 * L ** 3 / d, rel=1e-14)
    p = I.path(3)
    pos = np.array([[0, 0], [1, 0], [3, 0]], dtype=float)
    krow, kcol = O.khop(3, p.row_ptr, p.col_idx, 1)
    m = O.metrics(3, p.row_ptr, p.col_idx, krow, kcol, pos)
    assert m["edge_mean"] == 1.5 and m["edge_std"] == 0.5
    assert m["edge_cv"] == pytest.approx(1.0 / 3.0, rel=1e-15)


def test_thread_count_does_not_change_results():
    g = I.barabasi_albert(500, 3, 2)
    pos = I.uniform_positions(g.n, 1)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
    n0 = O.threads()
    O.set_threads(1)
    a = O.run(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, 5)
    O.set_threads(max(2, n0))
    b = O.run(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, 5)
    O.set_threads(n0)
    assert np.array_equal(a, b)
