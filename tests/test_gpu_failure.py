"""Failure detection on the GPU without a fault: the blocked path's tile
waits are bounded; a test hook announces the tiles without copying them, so
every wait runs out, the kernels return early, the next synchronising call
reports GILA_ECUDA, and the context goes on working."""
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


@pytest.mark.parametrize("name,maker,k", [
    ("tiles", lambda: I.barabasi_albert(20000, 3, 31), 2),
    ("windows", lambda: I.tri_mesh(60, 70), 2),
], ids=["tiles", "windows"])
def test_tile_wait_timeout_is_reported_and_context_survives(name, maker, k):
    torch = _torch()
    g = maker()
    pos = I.uniform_positions(g.n, 32)
    okrow, okcol = O.khop(g.n, g.row_ptr, g.col_idx, k)
    prm = G.params(k=k)
    t = 0.1 * math.sqrt(g.n)
    with G.Graph.from_inputs(g) as h:
        G.gila_graph_tune(h.handle, tiled=1)
        x = torch.tensor(pos, dtype=torch.float32, device="cuda")
        y, disp = torch.empty_like(x), torch.empty_like(x)
        G.gila_graph_set_wait_test(h.handle, True)
        G.gila_layout_step(h.handle, prm, t, x, y, disp)  # asynchronous: no error yet
        with pytest.raises(G.GilaError) as err:
            G.gila_layout_metrics(h.handle, prm, x)
        assert err.value.status == G.GILA_ECUDA and "did not complete" in str(err.value)
        # the flag was cleared and the context is usable
        G.gila_graph_set_wait_test(h.handle, False)
        G.gila_layout_metrics(h.handle, prm, x)
        G.gila_layout_step(h.handle, prm, t, x, y, disp)
        got = disp.double().cpu().numpy()
    _, odisp = O.step(g.n, g.row_ptr, g.col_idx, okrow, okcol, pos.astype(np.float32), t)
    assert np.abs(got - odisp).max() <= 1e-4 * np.abs(odisp).max()
