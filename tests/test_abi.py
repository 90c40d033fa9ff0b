"""C-ABI library checks that need no GPU: it loads, exports every entry
point declared in include/gila.h, and its host-side logic (CSR validation,
defaults, cooling schedules) behaves as documented."""
import math
import os
import re

import numpy as np
import pytest

import __graft_entry__
from paper_1606_02162_gb300 import gila as G
from paper_1606_02162_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(gila_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported():
    lib = G.load()
    declared = _declared()
    assert len(declared) >= 15
    bound = {s[0] for s in G.SIGNATURES}
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} not exported"
        assert name in bound, f"{name} has no Python binding"


def test_params_default():
    p = G.gila_params_default()
    assert (p.k, p.iters, p.d, p.t0, p.schedule, p.p, p.q, p.precision) == (
        2, 300, 1.0, 0.0, G.GILA_COOL_LINEAR, 2, 1, G.GILA_FP32)


def test_temperature_schedules_host():
    p = G.params(iters=10, schedule=G.GILA_COOL_LINEAR)
    for i in range(10):
        assert G.gila_temperature(p, 3.2, i) == pytest.approx(3.2 * (10 - i) / 10, rel=1e-15)
    p = G.params(iters=10, schedule=G.GILA_COOL_GEOMETRIC)
    for i in range(10):
        assert G.gila_temperature(p, 2.0, i) == pytest.approx(2.0 * 0.93 ** i, rel=1e-14)


def test_csr_validate_accepts_generated_graphs():
    for g in (I.grid(7, 5), I.barabasi_albert(300, 3, 1), I.random_tree(40, 2),
              I.csr_from_edges(4, [], [])):
        assert G.gila_csr_validate(g.n, g.row_ptr, g.col_idx) == G.GILA_OK


@pytest.mark.parametrize("case,needle", [
    ("selfloop", "self-loop"),
    ("repeat", "repeated"),
    ("asym", "reverse"),
    ("range", "out of range"),
    ("rowptr", "row_ptr"),
])
def test_csr_validate_rejects(case, needle):
    row = np.array([0, 2, 4, 6], dtype=np.int64)
    col = np.array([1, 2, 0, 2, 0, 1], dtype=np.int32)  # triangle
    assert G.gila_csr_validate(3, row, col) == G.GILA_OK
    if case == "selfloop":
        col = np.array([1, 0, 0, 2, 0, 1], dtype=np.int32)
    elif case == "repeat":
        col = np.array([1, 1, 0, 2, 0, 1], dtype=np.int32)
    elif case == "asym":
        row = np.array([0, 2, 3, 5], dtype=np.int64)
        col = np.array([1, 2, 0, 0, 1], dtype=np.int32)
    elif case == "range":
        col = np.array([1, 3, 0, 2, 0, 1], dtype=np.int32)
    elif case == "rowptr":
        row = np.array([0, 4, 2, 6], dtype=np.int64)
    assert G.gila_csr_validate(3, row, col) == G.GILA_EINVAL
    assert needle in G.gila_last_error()


def test_binding_fails_loudly_without_library(tmp_path):
    import importlib
    mod = importlib.import_module("paper_1606_02162_gb300.gila")
    with pytest.raises(RuntimeError, match="not found"):
        saved = mod._lib
        try:
            mod._lib = None
            mod.load(str(tmp_path / "missing.so"))
        finally:
            mod._lib = saved


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1606_02162_gb300")
    bad = re.compile(r"(import\s+oracle|from\s+oracle|liboracle|gila_oracle)")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert not bad.search(src), f"{f} reaches into the oracle"


@pytest.mark.parametrize("row,col,needle", [
    ([0, 1, 2], [1, 2], "out of range"),
    ([0, 2, 1], [1, 0], "decreases"),
    ([1, 2, 3], [1, 0], "row_ptr[0]"),
    ([0, 1, 2], [1, -1], "out of range"),
])
def test_graph_create_rejects_unsafe_csr_without_gpu(row, col, needle):
    """Offsets and ids are checked before any device work, flags or not, so a
    malformed CSR can never reach a kernel."""
    from paper_1606_02162_gb300 import gila as G
    with pytest.raises(G.GilaError) as err:
        G.gila_graph_create(2, np.array(row, dtype=np.int64), np.array(col, dtype=np.int32))
    assert err.value.status == G.GILA_EINVAL and needle in str(err.value)


def test_batch_create_rejects_unsafe_csr_without_gpu():
    from paper_1606_02162_gb300 import gila as G
    good = I.path(4)
    bad = I.path(3)
    bad_col = bad.col_idx.copy()
    bad_col[0] = 7
    import ctypes
    lib = G.load()
    ns = (ctypes.c_int64 * 2)(good.n, bad.n)
    rows = (ctypes.c_void_p * 2)(good.row_ptr.ctypes.data, bad.row_ptr.ctypes.data)
    cols = (ctypes.c_void_p * 2)(good.col_idx.ctypes.data, bad_col.ctypes.data)
    out = ctypes.c_void_p()
    st = lib.gila_batch_create(2, ns, rows, cols, 0, ctypes.byref(out))
    assert st == G.GILA_EINVAL and b"graph 1" in lib.gila_last_error()


def _declared_arity():
    """Parameter count of every function declared in include/gila.h."""
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "gila.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(gila_\w+)\s*\(([^;{]*?)\)\s*;", src):
        name, params = m.group(1), m.group(2).strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_the_header():
    """Every entry point the binding declares has the header's parameter count."""
    from paper_1606_02162_gb300 import gila as G
    arity = _declared_arity()
    sigs = list(G.SIGNATURES)
    for extra in ("SERVER_SIGNATURES",):
        sigs += list(getattr(G, extra, []))
    assert sigs
    for name, _res, args in sigs:
        assert name in arity, name
        assert len(args) == arity[name], (name, len(args), arity[name])
    # and every declared entry point has a binding
    assert set(arity) == {n for n, _, _ in sigs}
