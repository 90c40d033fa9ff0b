"""Pins of the oracle's per-component layout (Section 4.6: the pipeline runs
on every connected component, whose drawings are then arranged without
overlap; Section 5.1: the maximum displacement of a component follows its
own n and initial frame) against independent routes."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1606_02162_gb300 import inputs as I


def _canon(label):
    """Relabel components in the order of their smallest vertex id."""
    first = {}
    out = np.empty_like(label)
    for v, c in enumerate(label):
        if c not in first:
            first[c] = len(first)
        out[v] = first[c]
    return out


@pytest.mark.parametrize("maker", [
    lambda: I.erdos_renyi(300, 0.7, 1),
    lambda: I.erdos_renyi(500, 1.2, 2),
    lambda: I.chung_lu(600, 2.3, 2.0, 500, 3),
    lambda: I.random_tree(50, 4),
    lambda: I.csr_from_edges(7, [], []),
])
def test_components_match_scipy(maker):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    g = maker()
    label, count = O.components(g.n, g.row_ptr, g.col_idx)
    A = csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    c2, l2 = connected_components(A, directed=False)
    assert count == c2
    assert np.array_equal(label, _canon(l2))


def test_pack_four_unit_squares():
    """Four unit boxes, gap 1: W = sqrt(4 * 2 * 2) = 4, two per row."""
    bbox = np.array([[0, 0, 1, 1], [5, 5, 6, 6], [-3, 2, -2, 3], [10, 10, 11, 11]], float)
    off = O.pack(bbox, np.array([4, 4, 4, 4]), 1.0)
    placed = bbox[:, :2] + off
    assert placed.tolist() == [[0, 0], [2, 0], [0, 2], [2, 2]]


def test_pack_invariants_random():
    rng = np.random.default_rng(5)
    c = 60
    lo = rng.uniform(-50, 50, (c, 2))
    wh = rng.exponential(3.0, (c, 2))
    wh[:5] = 0.0  # points (single vertices)
    bbox = np.hstack([lo, lo + wh])
    size = rng.integers(1, 100, c)
    gap = 0.75
    off = O.pack(bbox, size, gap)
    box = np.hstack([bbox[:, :2] + off, bbox[:, 2:] + off])
    # no two boxes come closer than the gap
    for i in range(c):
        for j in range(i + 1, c):
            sep_x = max(box[j, 0] - box[i, 2], box[i, 0] - box[j, 2])
            sep_y = max(box[j, 1] - box[i, 3], box[i, 1] - box[j, 3])
            assert max(sep_x, sep_y) >= gap - 1e-9
    # reading order follows decreasing size (ties by index)
    order = sorted(range(c), key=lambda i: (-size[i], i))
    ys = [box[i, 1] for i in order]
    assert all(ys[i] <= ys[i + 1] + 1e-12 for i in range(c - 1))
    assert box[order[0], 0] == 0.0 and box[order[0], 1] == 0.0
    # rows stay within W unless a row holds a single box
    W = max((bbox[:, 2] - bbox[:, 0]).max(),
            math.sqrt(((bbox[:, 2] - bbox[:, 0] + gap) * (bbox[:, 3] - bbox[:, 1] + gap)).sum()))
    for y in set(np.round(box[:, 1], 9)):
        members = np.nonzero(np.round(box[:, 1], 9) == y)[0]
        if len(members) > 1:
            assert box[members, 2].max() <= W + 1e-9


def _two_copies(g, shift):
    """g twice, disjoint: the copy's ids follow the original's."""
    u = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    v = g.col_idx
    keep = u < v
    u, v = u[keep], v[keep]
    return I.csr_from_edges(2 * g.n, np.concatenate([u, u + g.n]), np.concatenate([v, v + g.n]))


def test_identical_components_get_identical_drawings():
    g = I.barabasi_albert(120, 2, 7)
    pos = I.uniform_positions(g.n, 8)
    gg = _two_copies(g, 0)
    # the same initial coordinates: components never interact, and a shifted
    # copy would only differ by rounding that the iterations amplify
    pos2 = np.vstack([pos, pos])
    out = O.components_layout(gg.n, gg.row_ptr, gg.col_idx, pos2, k=2, iters=40)
    a, b = out[:g.n], out[g.n:]
    assert np.allclose(a - a[0], b - b[0], rtol=0, atol=1e-9)
    # and each equals the component laid out alone, up to translation
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
    alone = O.run(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, 40)
    assert np.allclose(a - a[0], alone - alone[0], rtol=0, atol=1e-9)


def test_each_component_has_its_own_initial_temperature():
    """Geometric cooling: t0 of a component is sqrt(n_c d / a_c) with a_c
    the height/width of its own initial frame (Section 5.1)."""
    g1 = I.grid(6, 9)
    g2 = I.path(7)
    n1 = g1.n
    u1 = np.repeat(np.arange(g1.n), np.diff(g1.row_ptr))
    u2 = np.repeat(np.arange(g2.n), np.diff(g2.row_ptr))
    g = I.csr_from_edges(g1.n + g2.n, np.concatenate([u1, u2 + n1]),
                         np.concatenate([g1.col_idx, g2.col_idx + n1]))
    rng = np.random.default_rng(11)
    p1 = rng.uniform(0, 1, (g1.n, 2)) * [8.0, 3.0]
    p2 = rng.uniform(0, 1, (g2.n, 2)) * [2.0, 6.0]
    pos = np.vstack([p1, p2])
    d, iters = 1.5, 25
    out = O.components_layout(g.n, g.row_ptr, g.col_idx, pos, k=2, iters=iters, d=d,
                              schedule=O.SCHED_GEOM)
    for gc, pc, sl in ((g1, p1, slice(0, n1)), (g2, p2, slice(n1, None))):
        w, h = np.ptp(pc[:, 0]), np.ptp(pc[:, 1])
        t0 = math.sqrt(gc.n * d / (h / w))
        krow, kcol = O.khop(gc.n, gc.row_ptr, gc.col_idx, 2)
        alone = O.run(gc.n, gc.row_ptr, gc.col_idx, krow, kcol, pc, iters, d=d,
                      schedule=O.SCHED_GEOM, t0=t0)
        got = out[sl]
        assert np.allclose(got - got[0], alone - alone[0], rtol=0, atol=1e-9)


def test_single_component_is_only_translated():
    g = I.grid(5, 5)
    pos = I.uniform_positions(g.n, 3)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
    alone = O.run(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, 20)
    out = O.components_layout(g.n, g.row_ptr, g.col_idx, pos, k=2, iters=20)
    assert np.allclose(out, alone - alone.min(axis=0), rtol=0, atol=1e-12)
