"""GPU parity of the per-component layout (Section 4.6) and its component
labels against the oracle."""
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


def _graphs():
    return [
        ("er_sparse", I.erdos_renyi(20000, 0.9, 1)),
        ("er_giant", I.erdos_renyi(30000, 1.6, 2)),
        ("chunglu", I.chung_lu(40000, 2.3, 3.0, 60000, 3)),
        ("mesh", I.tri_mesh(120, 90)),
        ("isolated", I.csr_from_edges(500, [], [])),
        ("path", I.path(4097)),
        ("single", I.path(1)),
    ]


@pytest.mark.parametrize("name,g", _graphs(), ids=[n for n, _ in _graphs()])
def test_component_labels_match_oracle(name, g):
    _torch()
    label, count = O.components(g.n, g.row_ptr, g.col_idx)
    with G.Graph.from_inputs(g) as h:
        l2, c2 = G.gila_graph_components(h.handle, g.n)
    assert c2 == count and np.array_equal(l2, label)


def _mixed_graph():
    """A big component (beyond the batch size), many small ones of several
    families, and isolated vertices, with ids interleaved."""
    parts = [I.barabasi_albert(6000, 2, 11), I.grid(12, 15), I.random_tree(300, 12),
             I.erdos_renyi(400, 3.0, 13), I.path(2), I.cycle(9)]
    parts += [I.random_tree(int(n), 20 + i) for i, n in enumerate([30, 45, 70, 120, 5, 3])]
    n = sum(p.n for p in parts) + 25
    perm = np.random.default_rng(5).permutation(n)
    us, vs, base = [], [], 0
    for p in parts:
        u = np.repeat(np.arange(p.n), np.diff(p.row_ptr))
        keep = u < p.col_idx
        us.append(perm[base + u[keep]])
        vs.append(perm[base + p.col_idx[keep]])
        base += p.n
    return I.csr_from_edges(n, np.concatenate(us), np.concatenate(vs))


@pytest.mark.parametrize("prec,iters", [(G.GILA_FP64, 5), (G.GILA_FP32, 1)],
                         ids=["fp64", "fp32"])
def test_components_layout_matches_oracle_few_iterations(prec, iters):
    """Linear cooling, a few iterations: every component against the oracle's
    own run of it, and the packed placement (FP64 within 1e-9 of the extent;
    FP32 one iteration within 1e-4 of the largest move plus the rounding of
    the coordinates)."""
    _torch()
    g = _mixed_graph()
    pos = I.uniform_positions(g.n, 7)
    ref = O.components_layout(g.n, g.row_ptr, g.col_idx, pos, k=2, iters=iters)
    with G.Graph.from_inputs(g) as h:
        out, count = G.gila_layout_components_run(h.handle, G.params(k=2, iters=iters,
                                                                     precision=prec), pos)
    label, c2 = O.components(g.n, g.row_ptr, g.col_idx)
    assert count == c2
    scale = np.abs(ref).max()
    if prec == G.GILA_FP64:
        assert np.abs(out - ref).max() <= 1e-9 * scale
    else:
        # the largest move of any vertex (the packing shift cancels within a component)
        move = max(np.abs((ref[label == c] - ref[label == c][0]) -
                          (pos[label == c] - pos[label == c][0])).max() for c in range(count))
        assert np.abs(out - ref).max() <= 2e-4 * move + 1e-6 * scale


@pytest.mark.parametrize("schedule", [O.SCHED_LINEAR, O.SCHED_GEOM], ids=["linear", "geom"])
def test_components_layout_whole_run_quality(schedule):
    """200 iterations in FP32: edge-length CV and repulsive/attractive ratio of
    the packed drawing (the library's FP64 reductions) within 2% of the
    oracle's (both are unchanged by the packing, which only translates
    components)."""
    torch = _torch()
    g = _mixed_graph()
    pos = I.uniform_positions(g.n, 8)
    iters = 200
    ref = O.components_layout(g.n, g.row_ptr, g.col_idx, pos, k=2, iters=iters,
                              schedule=schedule)
    with G.Graph.from_inputs(g) as h:
        out, _ = G.gila_layout_components_run(
            h.handle, G.params(k=2, iters=iters, schedule=schedule), pos)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, 2)
    mo = O.metrics(g.n, g.row_ptr, g.col_idx, krow, kcol, ref)
    with G.Graph.from_inputs(g) as h:
        mg = G.gila_layout_metrics(h.handle, G.params(k=2, iters=iters, schedule=schedule),
                                   torch.tensor(out, dtype=torch.float32, device="cuda"))
    for key in ("edge_cv", "rep_att_ratio"):
        assert abs(mg[key] - mo[key]) <= 0.02 * abs(mo[key]), (key, mg[key], mo[key])


def test_packed_boxes_do_not_overlap():
    _torch()
    g = _mixed_graph()
    pos = I.uniform_positions(g.n, 9)
    gap = 2.5
    with G.Graph.from_inputs(g) as h:
        out, count = G.gila_layout_components_run(h.handle, G.params(k=2, iters=30), pos,
                                                  gap=gap)
    label, _ = O.components(g.n, g.row_ptr, g.col_idx)
    box = np.array([[out[label == c, 0].min(), out[label == c, 1].min(),
                     out[label == c, 0].max(), out[label == c, 1].max()] for c in range(count)])
    for i in range(count):
        for j in range(i + 1, count):
            sep = max(box[j, 0] - box[i, 2], box[i, 0] - box[j, 2],
                      box[j, 1] - box[i, 3], box[i, 1] - box[j, 3])
            assert sep >= gap * (1 - 1e-9)
    assert box[:, 0].min() == 0.0 and box[:, 1].min() == 0.0


def test_identical_components_identical_drawings():
    _torch()
    g1 = I.barabasi_albert(800, 2, 21)
    u = np.repeat(np.arange(g1.n), np.diff(g1.row_ptr))
    keep = u < g1.col_idx
    g = I.csr_from_edges(2 * g1.n, np.concatenate([u[keep], u[keep] + g1.n]),
                         np.concatenate([g1.col_idx[keep], g1.col_idx[keep] + g1.n]))
    p = I.uniform_positions(g1.n, 22)
    with G.Graph.from_inputs(g) as h:
        out, count = G.gila_layout_components_run(h.handle, G.params(k=2, iters=50),
                                                  np.vstack([p, p]))
    assert count == 2
    a, b = out[:g1.n], out[g1.n:]
    assert np.allclose(a - a[0], b - b[0], rtol=0, atol=1e-9 * np.abs(out).max())
