"""gila_khop_count_noalloc: k-hop list sizes for callers that must not
allocate device memory (for example a serving process whose own memory
manager owns the device and needs these sizes to decide admission before it
reserves anything).

The entry point is checked through the C ABI against the allocating path
(gila_build_khop + gila_khop_export, whose row offsets give the same sizes),
on two calls in a row, since every call reuses the library's one scratch
array. Counts are integers, so the tolerance is exact equality, as for the
k-hop lists themselves. This file is named to be collected last.
"""
import numpy as np
import pytest

import __graft_entry__
from paper_1606_02162_gb300 import gila as G
from paper_1606_02162_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LIMIT = 1 << 18


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    import torch
    torch.cuda.set_device(0)


CASES = [
    ("grid32_k2", lambda: I.grid(32, 32), 2),
    ("ba20k_k2", lambda: I.barabasi_albert(20000, 3, 7), 2),
    ("ba20k_k3", lambda: I.barabasi_albert(20000, 3, 7), 3),  # most balls overflow tier 1
    ("star3k_k2", lambda: I.star(3000), 2),
    ("isolated", lambda: I.csr_from_edges(40, [0, 5], [1, 6]), 3),
]


def _allocating_counts(g, k):
    with G.Graph.from_inputs(g) as h:
        total = G.gila_build_khop(h.handle, k)
        krow, _ = G.gila_khop_export(h.handle)
    return np.diff(krow), total


@pytest.mark.parametrize("name,maker,k", CASES, ids=[c[0] for c in CASES])
def test_noalloc_counts_match_allocating_path(name, maker, k):
    import torch
    g = maker()
    want, want_total = _allocating_counts(g, k)
    row = torch.tensor(g.row_ptr, dtype=torch.int64, device="cuda")
    col = torch.tensor(g.col_idx, dtype=torch.int32, device="cuda")
    for i in range(2):  # the second call must not see the first call's scratch
        counts = torch.full((g.n,), -7, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
        total = G.gila_khop_count_noalloc(g.n, row, col, k, counts)
        torch.cuda.synchronize()
        after = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
        if i == 1:
            # the defining property: the call takes no device memory (the
            # first call may still load the library's module on the device)
            assert after == before, (before, after)
        assert total == want_total
        assert np.array_equal(counts.cpu().numpy(), want)


def test_noalloc_alternating_graphs():
    import torch
    a, b = I.barabasi_albert(5000, 3, 1), I.grid(40, 30)
    wa, _ = _allocating_counts(a, 3)
    wb, _ = _allocating_counts(b, 2)
    for g, k, want in ((a, 3, wa), (b, 2, wb), (a, 3, wa)):
        row = torch.tensor(g.row_ptr, dtype=torch.int64, device="cuda")
        col = torch.tensor(g.col_idx, dtype=torch.int32, device="cuda")
        counts = torch.empty(g.n, dtype=torch.int64, device="cuda")
        total = G.gila_khop_count_noalloc(g.n, row, col, k, counts)
        assert total == want.sum()
        assert np.array_equal(counts.cpu().numpy(), want)


def test_noalloc_rejects_sizes_beyond_the_limit():
    import torch
    n = LIMIT + 1
    row = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    counts = torch.zeros(n, dtype=torch.int64, device="cuda")
    with pytest.raises(G.GilaError) as e:
        G.gila_khop_count_noalloc(n, row, col, 2, counts)
    assert e.value.status == G.GILA_EINVAL
    assert "262144" in str(e.value)
    # at the limit it works (a graph without edges: every list is empty)
    n = LIMIT
    row = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    counts = torch.full((n,), 5, dtype=torch.int64, device="cuda")
    assert G.gila_khop_count_noalloc(n, row, col, 2, counts) == 0
    assert int(counts.abs().sum()) == 0
