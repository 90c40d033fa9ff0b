"""Serving engine: admission by device memory, concurrent jobs, and each
result identical alone and in the mix (the job runs the same kernels)."""
import math
import threading

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


def _jobs():
    out = []
    for i, (n, k) in enumerate([(3000, 2), (400, 3), (20000, 2), (1500, 3), (8000, 2), (60, 2)]):
        g = I.barabasi_albert(n, 3, 40 + i)
        out.append((g, I.uniform_positions(g.n, 70 + i), k))
    return out


def _alone(g, pos, prm):
    with G.Graph.from_inputs(g) as h:
        return G.gila_layout_run(h.handle, prm, pos)


@pytest.mark.parametrize("prec", [G.GILA_FP32, G.GILA_FP64], ids=["fp32", "fp64"])
def test_results_same_alone_and_in_the_mix(prec):
    jobs = _jobs()
    with G.Server(8 << 30, 8) as s:
        tickets = [s.submit(g, pos, G.params(k=k, iters=40, precision=prec))
                   for g, pos, k in jobs]
        results = [s.wait(t) for t in tickets]
        st = s.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["bytes_in_use"] == 0
    for (g, pos, k), (out, info) in zip(jobs, results):
        assert info["status"] == G.GILA_OK and info["latency_ms"] > 0
        ref = _alone(g, pos, G.params(k=k, iters=40, precision=prec))
        assert np.array_equal(out, ref), g.name


def test_one_step_matches_oracle():
    g, pos, k = _jobs()[0]
    with G.Server(1 << 30, 2) as s:
        t = s.submit(g, pos, G.params(k=k, iters=1, precision=G.GILA_FP64))
        out, info = s.wait(t)
    krow, kcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    assert info["nnz_khop"] == krow[-1]
    _, odisp = O.step(g.n, g.row_ptr, g.col_idx, krow, kcol, pos, 0.1 * math.sqrt(g.n))
    assert np.abs((out - pos) - odisp).max() <= 1e-12 * np.abs(odisp).max()


def test_admission_respects_the_budget():
    jobs = [j for j in _jobs() if j[0].n != 20000]
    giant = I.barabasi_albert(60000, 3, 9)  # k = 3 lists of several hundred MB
    jobs.insert(2, (giant, I.uniform_positions(giant.n, 3), 3))
    budget = 16 << 20  # a few small jobs at a time
    with G.Server(budget, 8) as s:
        tickets = [s.submit(g, pos, G.params(k=k, iters=20)) for g, pos, k in jobs]
        outs = []
        for t in tickets:
            try:
                outs.append(s.wait(t))
            except G.GilaError as e:
                outs.append(e)
        st = s.stats()
    assert st["bytes_peak"] <= budget
    # the giant job can never fit and fails cleanly; the others all run
    for (g, pos, k), r in zip(jobs, outs):
        if g is giant:
            assert isinstance(r, G.GilaError) and r.status == G.GILA_EBUDGET
        else:
            assert np.array_equal(r[0], _alone(g, pos, G.params(k=k, iters=20)))


def test_one_slot_serialises_but_completes():
    jobs = _jobs()[:4]
    with G.Server(4 << 30, 1) as s:
        tickets = [s.submit(g, pos, G.params(k=k, iters=15)) for g, pos, k in jobs]
        for (g, pos, k), t in zip(jobs, tickets):
            out, _ = s.wait(t)
            assert np.array_equal(out, _alone(g, pos, G.params(k=k, iters=15)))


def test_wait_timeout_poll_and_unknown_ticket():
    g = I.barabasi_albert(50000, 3, 5)
    pos = I.uniform_positions(g.n, 1)
    with G.Server(8 << 30, 2) as s:
        t = s.submit(g, pos, G.params(k=3, iters=300))
        with pytest.raises(G.GilaError) as e:
            s.wait(t, timeout_ms=0)
        assert e.value.status == G.GILA_ETIMEDOUT
        out, info = s.wait(t)  # the ticket stays valid after a timeout
        assert info["status"] == G.GILA_OK and np.isfinite(out).all()
        with pytest.raises(G.GilaError) as e:
            s.wait(t)
        assert e.value.status == G.GILA_EINVAL
        with pytest.raises(G.GilaError):
            s.poll(12345)


def test_concurrent_submitters():
    jobs = _jobs()
    prm = G.params(k=2, iters=25)
    results = {}
    with G.Server(8 << 30, 4) as s:
        def worker(i):
            g, pos, _ = jobs[i]
            t = s.submit(g, pos, prm)
            results[i] = s.wait(t)[0]
        th = [threading.Thread(target=worker, args=(i,)) for i in range(len(jobs))]
        for x in th:
            x.start()
        for x in th:
            x.join()
    for i, (g, pos, _) in enumerate(jobs):
        assert np.array_equal(results[i], _alone(g, pos, prm))


def test_destroy_with_jobs_in_flight():
    jobs = _jobs()
    s = G.Server(8 << 30, 4)
    for g, pos, k in jobs:
        s.submit(g, pos, G.params(k=k, iters=200))
    s.close()  # stops the threads, fails unfinished jobs, frees memory
