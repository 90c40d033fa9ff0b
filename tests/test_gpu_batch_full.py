"""The batch workload at its own size and in the launch shapes the benchmark
uses: 4,096 graphs of 50-5,000 vertices (log-uniform; random labelled trees,
near-square grids and G(n, 4/(n-1)), seed 4), k = 2, 200 iterations, in one
persistent launch whose shape the library's autotuner picks on this batch
(as bench.py does), and again with 256-thread CTAs at 8 per SM, where every
graph beyond the shared-memory cut (about 1,700 vertices in FP32, 880 in
FP64) iterates on global placement buffers instead.

A systematic sample (every 16th graph in batch order, and the largest graph)
is checked against the oracle graph by graph:

  k-hop lists            bit-exact (the batch's own export, union numbering)
  one iteration          FP32 within 1e-4, FP64 within 1e-12 of the graph's
                         largest move (the linear schedule's first
                         temperature, 0.1 sqrt(n) of that graph)
  200 iterations         edge-length CV and repulsive/attractive ratio of the
                         GPU layouts (GPU FP64 reductions): per family
                         (trees, grids, G(n, p)) the mean over the sampled
                         graphs within 2% of the mean of the oracle's own
                         200-iteration layouts, every graph within 25%

Why means for the whole runs: 200 iterations of these small graphs are
chaotic. The oracle's own layout moves when its initial placement is merely
rounded to FP32 (a relative change of 1e-7): over the sample its edge-length
CV then changes by up to 16% on a grid (median 3%), 7% on G(n, p) and 4% on a
tree, its ratio by up to 4%, while the family means change by at most 1%.
A single graph's whole-run figure therefore carries no 2% signal; the step
itself is compared element by element above.
"""
import math

import numpy as np
import pytest

import __graft_entry__
import oracle as O
from paper_1606_02162_gb300 import gila as G
from paper_1606_02162_gb300 import inputs as I

pytestmark = pytest.mark.gpu

K, ITERS = 2, 200


@pytest.fixture(scope="module")
def batch():
    import torch
    __graft_entry__.build()
    torch.cuda.set_device(0)
    graphs = I.batch_mix(4096, 50, 5000, 4)
    pos = [I.uniform_positions(g.n, 400000 + i) for i, g in enumerate(graphs)]
    sizes = np.array([g.n for g in graphs])
    sample = sorted(set(range(0, len(graphs), 16)) | {int(np.argmax(sizes))})
    ref = {}
    for i in sample:
        g = graphs[i]
        krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, K)
        lay = O.run(g.n, g.row_ptr, g.col_idx, krow, kcol, pos[i], ITERS)
        ref[i] = (krow, kcol, O.metrics(g.n, g.row_ptr, g.col_idx, krow, kcol, lay))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return graphs, pos, sample, ref, off


def _shape(b, prec, x0, mode):
    if mode == "autotuned":
        return G.gila_batch_autotune(b.handle, G.params(k=K, iters=ITERS, precision=prec), x0, 10)
    G.gila_batch_tune(b.handle, threads=256, ctas_per_sm=8)
    return G.gila_batch_get_tuning(b.handle, prec)


def test_full_batch_khop_lists_exact(batch):
    graphs, _, sample, ref, off = batch
    with G.Batch(graphs) as b:
        nnz = G.gila_batch_build_khop(b.handle, K)
        krow, kcol = G.gila_batch_khop_export(b.handle)
    assert nnz == krow[-1] == len(kcol)
    for i in sample:
        okrow, okcol, _ = ref[i]
        a, e = int(off[i]), int(off[i + 1])
        rows = krow[a:e + 1] - krow[a]
        ids = kcol[krow[a]:krow[e]].astype(np.int64) - a
        assert np.array_equal(rows, okrow), graphs[i].name
        assert np.array_equal(ids, okcol.astype(np.int64)), graphs[i].name


@pytest.mark.parametrize("mode", ["autotuned", "8_per_sm"])
@pytest.mark.parametrize("prec,tol", [(G.GILA_FP32, 1e-4), (G.GILA_FP64, 1e-12)],
                         ids=["fp32", "fp64"])
def test_full_batch_against_oracle(batch, prec, tol, mode):
    import torch
    graphs, pos, sample, ref, off = batch
    dt = torch.float64 if prec == G.GILA_FP64 else torch.float32
    with G.Batch(graphs) as b:
        x0 = torch.tensor(np.concatenate(pos), dtype=dt, device="cuda")
        tuning = _shape(b, prec, x0, mode)
        if mode == "8_per_sm":
            assert tuning["ctas_per_sm"] == 8 and tuning["threads"] == 256
        # one iteration of every graph
        x = x0.clone()
        G.gila_layout_batch_device(b.handle, G.params(k=K, iters=1, precision=prec), x)
        one = x.double().cpu().numpy()
        # the whole 200-iteration layouts
        x = x0.clone()
        G.gila_layout_batch_device(b.handle, G.params(k=K, iters=ITERS, precision=prec), x)
        lay = x.double().cpu().numpy()
        base_all = x0.double().cpu().numpy()
    worst_step, dev = 0.0, []
    fam_gpu, fam_ora = {}, {}
    for i in sample:
        g = graphs[i]
        a, e = int(off[i]), int(off[i + 1])
        krow, kcol, mo = ref[i]
        base = base_all[a:e]
        t = 0.1 * math.sqrt(g.n)
        _, odisp = O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, base, t)
        scale = np.abs(odisp).max()
        # FP32: the move is read back as (base + move) - base in FP32
        slack = 4 * np.finfo(np.float32).eps * np.abs(base).max() if prec == G.GILA_FP32 else 0.0
        err = np.abs((one[a:e] - base) - odisp).max()
        worst_step = max(worst_step, err / scale)
        assert err <= tol * scale + slack, (g.name, err, scale)
        # quality of the GPU's own layout, by the library's FP64 reductions
        with G.Graph.from_inputs(g) as h:
            p = torch.tensor(lay[a:e], dtype=dt, device="cuda")
            m = G.gila_layout_metrics(h.handle, G.params(k=K, iters=ITERS, precision=prec), p)
        fam = g.name.split("_")[0].rstrip("0123456789x")
        for key in ("edge_cv", "rep_att_ratio"):
            dev.append((abs(m[key] - mo[key]) / abs(mo[key]), g.name, key))
            fam_gpu.setdefault((fam, key), []).append(m[key])
            fam_ora.setdefault((fam, key), []).append(mo[key])
    dev.sort(reverse=True)
    means = {fk: (float(np.mean(fam_gpu[fk])), float(np.mean(fam_ora[fk])), len(fam_gpu[fk]))
             for fk in fam_gpu}
    print(f"mode {mode} tuning {tuning}: worst one-step error {worst_step:.3g} of the largest "
          f"move; family means (gpu, oracle, graphs) {means}; largest single deviations {dev[:3]}")
    assert len({fk[0] for fk in means}) == 3
    for fk, (mg, mo, cnt) in means.items():
        assert abs(mg - mo) <= 0.02 * abs(mo), (fk, mg, mo, cnt)
    assert dev[0][0] <= 0.25, dev[:4]
