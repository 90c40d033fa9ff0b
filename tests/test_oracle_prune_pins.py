"""Pins of the oracle's degree-one pruning (Section 4.3), weighted repulsion
and reinsertion (Section 4.6) against independent routes: scipy/numpy
restatements of the definitions, hand-worked special graphs, closed forms,
and invariants a plausible mistake would break."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1606_02162_gb300 import inputs as I


# ---------------------------------------------------------------- pruning

def _prune_numpy(g):
    """Section 4.3 with numpy: degree-one vertices go, a single-edge
    component keeps its smaller id; w counts removed neighbours."""
    deg = np.diff(g.row_ptr)
    anchor = np.full(g.n, -1, dtype=np.int64)
    for v in np.nonzero(deg == 1)[0]:
        a = g.col_idx[g.row_ptr[v]]
        if deg[a] == 1 and a > v:
            continue
        anchor[v] = a
    w = np.bincount(anchor[anchor >= 0], minlength=g.n)
    keep = anchor < 0
    return anchor, w, keep


def _induced_numpy(g, keep):
    from scipy.sparse import csr_matrix
    A = csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    idx = np.nonzero(keep)[0]
    B = A[idx][:, idx].tocsr()
    B.sort_indices()
    return B.indptr.astype(np.int64), B.indices.astype(np.int32)


@pytest.mark.parametrize("maker", [
    lambda: I.random_tree(200, 3),
    lambda: I.barabasi_albert(300, 1, 4),
    lambda: I.barabasi_albert(300, 2, 5),
    lambda: I.erdos_renyi(400, 1.5, 6),
    lambda: I.chung_lu(500, 2.3, 3.0, 700, 7),
    lambda: I.star(9),
    lambda: I.path(2),
    lambda: I.path(7),
])
def test_prune_matches_definition(maker):
    g = maker()
    anchor, w, newid, kept = O.prune(g.n, g.row_ptr, g.col_idx)
    ea, ew, ekeep = _prune_numpy(g)
    assert np.array_equal(anchor, ea)
    assert np.array_equal(w, ew)
    assert kept == int(ekeep.sum())
    assert np.array_equal(newid >= 0, ekeep)
    assert np.array_equal(newid[ekeep], np.arange(kept))
    prow, pcol = O.pruned_csr(g.n, g.row_ptr, g.col_idx, newid, kept)
    er, ec = _induced_numpy(g, ekeep)
    assert np.array_equal(prow, er) and np.array_equal(pcol, ec)


def test_prune_special_graphs():
    # star: the centre keeps all leaves, the pruned graph is one vertex
    g = I.star(6)
    anchor, w, newid, kept = O.prune(g.n, g.row_ptr, g.col_idx)
    assert kept == 1 and w[0] == 5 and list(anchor[1:]) == [0] * 5 and newid[0] == 0
    # single edge: the smaller id stays with one removed neighbour
    g = I.path(2)
    anchor, w, newid, kept = O.prune(g.n, g.row_ptr, g.col_idx)
    assert list(anchor) == [-1, 0] and list(w) == [1, 0] and kept == 1
    # path of 5: one pass only, so 1 and 3 stay although they end with degree one
    g = I.path(5)
    anchor, w, newid, kept = O.prune(g.n, g.row_ptr, g.col_idx)
    assert list(anchor) == [1, -1, -1, -1, 3] and list(w) == [0, 1, 0, 1, 0]
    assert list(newid) == [-1, 0, 1, 2, -1] and kept == 3
    prow, pcol = O.pruned_csr(g.n, g.row_ptr, g.col_idx, newid, kept)
    assert list(prow) == [0, 1, 3, 4] and list(pcol) == [1, 0, 2, 1]
    # a cycle has no degree-one vertex
    g = I.cycle(8)
    anchor, w, newid, kept = O.prune(g.n, g.row_ptr, g.col_idx)
    assert kept == 8 and (anchor < 0).all() and (w == 0).all()


# ---------------------------------------------------------- weighted forces

def test_weights_of_one_change_nothing():
    g = I.barabasi_albert(150, 2, 8)
    pos = I.uniform_positions(g.n, 3)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
    F0 = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos)
    F1 = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, wt=np.ones(g.n))
    assert np.array_equal(F0, F1)


@pytest.mark.parametrize("w0,w1", [(1.0, 4.0), (3.0, 1.0), (2.5, 7.0)])
def test_two_vertex_weighted_closed_form(w0, w1):
    """One edge, k = 1: vertex 0 is pushed with w1 d^2/delta and pulled with
    delta^2/d; the weight of the pushing vertex counts, not the receiver's."""
    g = I.path(2)
    d, delta = 1.3, 0.7
    pos = np.array([[0.0, 0.0], [delta, 0.0]])
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 1)
    F = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, d=d, wt=np.array([w0, w1]))
    assert F[0, 0] == pytest.approx(-(w1 * d * d / delta - delta * delta / d), rel=1e-14)
    assert F[1, 0] == pytest.approx(w0 * d * d / delta - delta * delta / d, rel=1e-14)
    assert F[0, 1] == 0.0 and F[1, 1] == 0.0


def test_weight_acts_only_through_the_weighted_vertex():
    """Raising wt[v] changes F(u) only for u with v in N_u(k), and not F(v)."""
    g = I.erdos_renyi(120, 3.0, 9)
    pos = I.uniform_positions(g.n, 5)
    k = 2
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    wt = 1.0 + np.arange(g.n) % 3
    F0 = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, wt=wt)
    v = 17
    wt2 = wt.copy()
    wt2[v] += 2.0
    F1 = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, wt=wt2)
    touched = {u for u in range(g.n) if v in set(kcol[krow[u]:krow[u + 1]].tolist())}
    for u in range(g.n):
        if u in touched:
            assert not np.array_equal(F0[u], F1[u])
            dx = pos[u] - pos[v]
            r2 = float(dx @ dx)
            assert np.allclose(F1[u] - F0[u], 2.0 * dx / r2, rtol=1e-9, atol=1e-12)
        else:
            assert np.array_equal(F0[u], F1[u])


def test_weighted_sum_of_forces():
    """With weights the forces no longer cancel; summed over all vertices of a
    complete graph (k = 1) they equal sum over pairs (w_v - w_u) d^2 (x_u - x_v)/delta^2,
    which vanishes when all weights agree."""
    g = I.complete(7)
    pos = I.uniform_positions(g.n, 12)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 1)
    wt = np.array([1.0, 2.0, 1.0, 5.0, 1.0, 3.0, 1.0])
    F = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, wt=wt)
    expect = np.zeros(2)
    for u in range(g.n):
        for v in range(u + 1, g.n):
            dx = pos[u] - pos[v]
            expect += (wt[v] - wt[u]) * dx / float(dx @ dx)
    assert np.allclose(F.sum(axis=0), expect, rtol=1e-10, atol=1e-12)
    Fc = O.forces(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, wt=np.full(g.n, 3.0))
    assert np.abs(Fc.sum(axis=0)).max() < 1e-10


# -------------------------------------------------------------- reinsertion

def _rotation_numpy(xv, edge_dirs, m, candidates=64):
    """Best rotation of the reinsertion rule, restated with numpy."""
    s = 2 * math.pi / m
    theta = s * (np.arange(candidates) + 0.5) / candidates
    if len(edge_dirs) == 0:
        return theta[0]
    a = np.mod(np.array(edge_dirs), s)
    diff = np.abs(a[None, :] - theta[:, None])
    score = np.minimum(diff, s - diff).min(axis=1)
    return theta[int(np.argmax(score))]


def test_reinsert_star_around_lonely_centre():
    g = I.star(6)
    anchor, w, newid, kept = O.prune(g.n, g.row_ptr, g.col_idx)
    prow, pcol = O.pruned_csr(g.n, g.row_ptr, g.col_idx, newid, kept)
    d = 1.5
    out = O.reinsert(g.n, g.row_ptr, g.col_idx, newid, anchor, w, prow, pcol,
                     np.array([[2.0, -1.0]]), d=d)
    assert list(out[0]) == [2.0, -1.0]
    s = 2 * math.pi / 5
    for i in range(5):
        a = s * 0.5 / 64 + i * s  # no edges: every rotation ties, the first wins
        assert out[1 + i, 0] == pytest.approx(2.0 + 0.2 * d * math.cos(a), abs=1e-15)
        assert out[1 + i, 1] == pytest.approx(-1.0 + 0.2 * d * math.sin(a), abs=1e-15)


def test_reinsert_two_leaves_beside_one_edge():
    """Kept vertex 0 at the origin with kept neighbours at (5, 0) and (3, 4)
    (both edges of length 5, so rho = 1) and two leaves: they sit half a turn
    apart at the rotation the numpy restatement picks."""
    g = I.csr_from_edges(5, [0, 0, 0, 1, 4], [1, 2, 3, 4, 0])
    anchor, w, newid, kept = O.prune(g.n, g.row_ptr, g.col_idx)
    assert list(anchor) == [-1, -1, 0, 0, -1] and w[0] == 2
    prow, pcol = O.pruned_csr(g.n, g.row_ptr, g.col_idx, newid, kept)
    ppos = np.array([[0.0, 0.0], [5.0, 0.0], [3.0, 4.0]])  # kept ids 0, 1, 4
    out = O.reinsert(g.n, g.row_ptr, g.col_idx, newid, anchor, w, prow, pcol, ppos)
    # edges at 0: to (5, 0) (angle 0) and to (3, 4) (angle atan2(4, 3)); shortest is 5
    theta = _rotation_numpy(0, [0.0, math.atan2(4, 3)], 2)
    rho = 0.2 * 5.0
    for i, leaf in enumerate((2, 3)):
        a = theta + i * math.pi
        assert out[leaf] == pytest.approx([rho * math.cos(a), rho * math.sin(a)], abs=1e-14)


def test_reinsert_two_leaves_one_edge_tie_rule():
    g = I.csr_from_edges(5, [0, 0, 0, 1], [1, 2, 3, 4])
    anchor, w, newid, kept = O.prune(g.n, g.row_ptr, g.col_idx)
    # 4 hangs on 1; 2 and 3 hang on 0
    assert list(anchor) == [-1, -1, 0, 0, 1]
    prow, pcol = O.pruned_csr(g.n, g.row_ptr, g.col_idx, newid, kept)
    ppos = np.array([[0.0, 0.0], [5.0, 0.0]])
    out = O.reinsert(g.n, g.row_ptr, g.col_idx, newid, anchor, w, prow, pcol, ppos)
    a = math.pi * 31.5 / 64
    assert out[2] == pytest.approx([math.cos(a), math.sin(a)], abs=1e-14)
    assert out[3] == pytest.approx([math.cos(a + math.pi), math.sin(a + math.pi)], abs=1e-14)
    # vertex 1: one leaf (s = 2 pi), edge direction pi; candidates at 2 pi (c + 1/2)/64,
    # the farthest from pi modulo 2 pi are c = 0 and 63 (tie): c = 0
    b = math.pi / 64
    assert out[4] == pytest.approx([5.0 + math.cos(b), math.sin(b)], abs=1e-14)


def test_reinsert_invariants_random():
    g = I.barabasi_albert(400, 1, 13)  # a tree: many leaves
    anchor, w, newid, kept = O.prune(g.n, g.row_ptr, g.col_idx)
    prow, pcol = O.pruned_csr(g.n, g.row_ptr, g.col_idx, newid, kept)
    ppos = I.uniform_positions(kept, 14) * 3.0
    out = O.reinsert(g.n, g.row_ptr, g.col_idx, newid, anchor, w, prow, pcol, ppos, d=1.0)
    keep = newid >= 0
    assert np.array_equal(out[keep], ppos)
    for v in np.nonzero(keep & (w > 0))[0]:
        pv = newid[v]
        nb = pcol[prow[pv]:prow[pv + 1]]
        vecs = ppos[nb] - ppos[pv]
        lens = np.hypot(vecs[:, 0], vecs[:, 1])
        rho = 0.2 * (lens.min() if len(nb) else 1.0)
        leaves = [u for u in g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]] if anchor[u] == v]
        assert len(leaves) == w[v]
        theta = _rotation_numpy(0, [math.atan2(y, x) for x, y in vecs], w[v])
        s = 2 * math.pi / w[v]
        for i, u in enumerate(leaves):
            r = out[u] - ppos[pv]
            assert math.hypot(*r) == pytest.approx(rho, rel=1e-12)
            a = theta + i * s
            assert r == pytest.approx([rho * math.cos(a), rho * math.sin(a)], abs=1e-12)


# ---------------------------------------------------------------- pipeline

def test_pipeline_star_is_centre_plus_circle():
    g = I.star(8)
    pos0 = I.uniform_positions(g.n, 2)
    out = O.pipeline(g.n, g.row_ptr, g.col_idx, pos0, k=2, iters=50)
    assert list(out[0]) == list(pos0[0])  # one vertex: no force, no move
    r = out[1:] - out[0]
    assert np.allclose(np.hypot(r[:, 0], r[:, 1]), 0.2)


@pytest.mark.parametrize("m", [1, 3, 7])
def test_pipeline_dumbbell_settles_at_weighted_length(m):
    """Two hubs joined by an edge, m leaves on each: the pruned graph is one
    edge whose ends repel with weight 1 + m, so it settles where
    (1 + m) d^2 / delta = delta^2 / d, delta = d (1 + m)^(1/3)."""
    u = [0] + [0] * m + [1] * m
    v = [1] + list(range(2, 2 + m)) + list(range(2 + m, 2 + 2 * m))
    g = I.csr_from_edges(2 + 2 * m, u, v)
    pos0 = I.uniform_positions(g.n, 4)
    d = 1.0
    # under the cap the pair ends within about 2 t_last = 2 t0 / iters of it
    iters, t0 = 2000, 2.0
    out = O.pipeline(g.n, g.row_ptr, g.col_idx, pos0, k=1, iters=iters, d=d, t0=t0)
    delta = math.hypot(*(out[0] - out[1]))
    assert abs(delta - d * (1 + m) ** (1.0 / 3.0)) <= 2.5 * t0 / iters
    for leaf in range(2, 2 + 2 * m):
        hub = 0 if leaf < 2 + m else 1
        assert math.hypot(*(out[leaf] - out[hub])) == pytest.approx(0.2 * delta, rel=1e-12)
