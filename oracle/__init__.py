"""FP64 CPU oracle of the GiLA k-hop Fruchterman-Reingold step.

TEST INFRASTRUCTURE ONLY. This package restates, in plain C (gila_oracle.c,
FP64, OpenMP over vertices with a fixed per-vertex summation order), what
the paper defines: the k-neighbourhoods of Section 4.5, the forces of
Section 3.1, the synchronous capped move of Sections 3.1 and 4.5, and the
degree-one pruning and reinsertion of Sections 4.3 and 4.6. It is
used by the tests, the smoke check and the benchmark's CPU-baseline leg, and
by nothing else; it shares no code with the CUDA library.

Functions take graphs as (n, row_ptr int64[n+1], col_idx int32[nnz]) and
placements as float64[n, 2].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gila_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

SCHED_LINEAR = 0
SCHED_GEOM = 1


def build(force: bool = False) -> str:
    """Compile gila_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP,
    strict IEEE: no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I = ctypes.c_int
        D = ctypes.c_double
        lib.oracle_threads.restype = I
        lib.oracle_set_threads.argtypes = [I]
        lib.oracle_khop_count.restype = I64
        lib.oracle_khop_count.argtypes = [I64, P, P, I, P]
        lib.oracle_khop_fill.restype = I
        lib.oracle_khop_fill.argtypes = [I64, P, P, I, P, P]
        lib.oracle_khop_rows.restype = I64
        lib.oracle_khop_rows.argtypes = [I64, P, P, I, I64, P, P, P, I64]
        lib.oracle_forces.argtypes = [I64, P, P, P, P, P, D, I, I, I64, P, P]
        lib.oracle_step.argtypes = [I64, P, P, P, P, P, D, I, I, D, P, P]
        lib.oracle_temperature.restype = D
        lib.oracle_temperature.argtypes = [I, D, I, I]
        lib.oracle_default_t0.restype = D
        lib.oracle_default_t0.argtypes = [I, I64, D, P]
        lib.oracle_run.restype = I
        lib.oracle_run.argtypes = [I64, P, P, P, P, P, D, I, I, I, D, I, P]
        lib.oracle_metrics.argtypes = [I64, P, P, P, P, P, D, I, I, P]
        lib.oracle_forces_w.argtypes = [I64, P, P, P, P, P, P, D, I, I, I64, P, P]
        lib.oracle_step_w.argtypes = [I64, P, P, P, P, P, P, D, I, I, D, P, P]
        lib.oracle_run_w.argtypes = [I64, P, P, P, P, P, P, D, I, I, I, D, I, P]
        lib.oracle_run_w.restype = I
        lib.oracle_prune.argtypes = [I64, P, P, P, P, P]
        lib.oracle_prune.restype = I64
        lib.oracle_pruned_csr.argtypes = [I64, P, P, P, P, P]
        lib.oracle_pruned_csr.restype = I64
        lib.oracle_reinsert.argtypes = [I64, P, P, P, P, P, P, P, P, D, P]
        lib.oracle_components.argtypes = [I64, P, P, P]
        lib.oracle_components.restype = ctypes.c_int32
        lib.oracle_pack.argtypes = [ctypes.c_int32, P, P, D, P]
        lib.oracle_pack.restype = I
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(n, row_ptr, col_idx):
    row = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col_idx, dtype=np.int32)
    assert row.shape[0] == n + 1
    return row, col


def _pos(pos, n):
    p = np.ascontiguousarray(pos, dtype=np.float64).reshape(n, 2)
    return p


def threads() -> int:
    return _load().oracle_threads()


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def khop(n, row_ptr, col_idx, k):
    """k-hop lists N_v(k) (Section 4.5): (krow int64[n+1], kcol int32[nnz]),
    rows ascending, v excluded."""
    lib = _load()
    row, col = _csr(n, row_ptr, col_idx)
    counts = np.zeros(max(n, 1), dtype=np.int64)
    lib.oracle_khop_count(n, _p(row), _p(col), int(k), _p(counts))
    krow = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts[:n], out=krow[1:])
    kcol = np.zeros(max(int(krow[-1]), 1), dtype=np.int32)
    rc = lib.oracle_khop_fill(n, _p(row), _p(col), int(k), _p(krow), _p(kcol))
    if rc != 0:
        raise RuntimeError("oracle_khop_fill: inconsistent row lengths")
    return krow, kcol[: int(krow[-1])]


def khop_rows(n, row_ptr, col_idx, k, sources):
    """N_v(k) for the listed sources only: (counts int64[s], concatenated
    sorted rows int32[sum counts])."""
    lib = _load()
    row, col = _csr(n, row_ptr, col_idx)
    src = np.ascontiguousarray(sources, dtype=np.int64)
    counts = np.zeros(max(src.shape[0], 1), dtype=np.int64)
    total = lib.oracle_khop_rows(n, _p(row), _p(col), int(k), src.shape[0], _p(src),
                                 _p(counts), None, 0)
    out = np.zeros(max(total, 1), dtype=np.int32)
    got = lib.oracle_khop_rows(n, _p(row), _p(col), int(k), src.shape[0], _p(src),
                               _p(counts), _p(out), total)
    if got != total:
        raise RuntimeError("oracle_khop_rows: size mismatch")
    return counts[: src.shape[0]], out[:total]


def _wt(wt, n):
    if wt is None:
        return None, None
    w = np.ascontiguousarray(wt, dtype=np.float64)
    assert w.shape == (n,)
    return w, _p(w)


def forces(n, row_ptr, col_idx, krow, kcol, pos, d=1.0, p=2, q=1, sel=None, wt=None):
    """Resultant force F(u) (Section 3.1 over N_u(k)) for all u, or for the
    vertices in sel: float64[len, 2]. wt (float64[n], optional): the
    repulsion exerted by v is multiplied by wt[v] (Section 4.6)."""
    lib = _load()
    row, col = _csr(n, row_ptr, col_idx)
    kr, kc = _csr(n, krow, kcol)
    P = _pos(pos, n)
    w, wp = _wt(wt, n)
    if sel is None:
        F = np.zeros((n, 2), dtype=np.float64)
        lib.oracle_forces_w(n, _p(row), _p(col), _p(kr), _p(kc), wp, _p(P), float(d), int(p),
                            int(q), 0, None, _p(F))
    else:
        s = np.ascontiguousarray(sel, dtype=np.int64)
        F = np.zeros((s.shape[0], 2), dtype=np.float64)
        lib.oracle_forces_w(n, _p(row), _p(col), _p(kr), _p(kc), wp, _p(P), float(d), int(p),
                            int(q), s.shape[0], _p(s), _p(F))
    return F


def step(n, row_ptr, col_idx, krow, kcol, pos, t, d=1.0, p=2, q=1, wt=None):
    """One synchronous capped iteration: (new positions, displacements)."""
    lib = _load()
    row, col = _csr(n, row_ptr, col_idx)
    kr, kc = _csr(n, krow, kcol)
    P = _pos(pos, n)
    w, wp = _wt(wt, n)
    out = np.zeros((n, 2), dtype=np.float64)
    disp = np.zeros((n, 2), dtype=np.float64)
    lib.oracle_step_w(n, _p(row), _p(col), _p(kr), _p(kc), wp, _p(P), float(d), int(p), int(q),
                      float(t), _p(out), _p(disp))
    return out, disp


def temperature(schedule, t0, i, iters) -> float:
    return _load().oracle_temperature(int(schedule), float(t0), int(i), int(iters))


def default_t0(schedule, n, d, pos) -> float:
    P = _pos(pos, n)
    return _load().oracle_default_t0(int(schedule), n, float(d), _p(P))


def run(n, row_ptr, col_idx, krow, kcol, pos0, iters, d=1.0, p=2, q=1,
        schedule=SCHED_LINEAR, t0=0.0, wt=None):
    """`iters` iterations from pos0; returns the final float64[n, 2]."""
    lib = _load()
    row, col = _csr(n, row_ptr, col_idx)
    kr, kc = _csr(n, krow, kcol)
    P = _pos(pos0, n)
    w, wp = _wt(wt, n)
    out = np.zeros((n, 2), dtype=np.float64)
    rc = lib.oracle_run_w(n, _p(row), _p(col), _p(kr), _p(kc), wp, _p(P), float(d), int(p),
                          int(q), int(schedule), float(t0), int(iters), _p(out))
    if rc != 0:
        raise MemoryError("oracle_run")
    return out


def metrics(n, row_ptr, col_idx, krow, kcol, pos, d=1.0, p=2, q=1) -> dict:
    """Edge-length mean/std/CV and the repulsive/attractive totals and ratio."""
    lib = _load()
    row, col = _csr(n, row_ptr, col_idx)
    kr, kc = _csr(n, krow, kcol)
    P = _pos(pos, n)
    out = np.zeros(6, dtype=np.float64)
    lib.oracle_metrics(n, _p(row), _p(col), _p(kr), _p(kc), _p(P), float(d), int(p), int(q),
                       _p(out))
    return {"edge_mean": out[0], "edge_std": out[1], "edge_cv": out[2],
            "rep_total": out[3], "att_total": out[4], "rep_att_ratio": out[5]}


def prune(n, row_ptr, col_idx):
    """Degree-one pruning (Section 4.3): (anchor int32[n], w int32[n],
    newid int32[n], kept) -- anchor[v] the neighbour a removed v hangs on
    (else -1), w[v] the number of removed neighbours of v, newid[v] the index
    of a kept v in the pruned graph (else -1)."""
    lib = _load()
    row, col = _csr(n, row_ptr, col_idx)
    anchor = np.zeros(max(n, 1), dtype=np.int32)
    w = np.zeros(max(n, 1), dtype=np.int32)
    newid = np.zeros(max(n, 1), dtype=np.int32)
    kept = lib.oracle_prune(n, _p(row), _p(col), _p(anchor), _p(w), _p(newid))
    return anchor[:n], w[:n], newid[:n], int(kept)


def pruned_csr(n, row_ptr, col_idx, newid, kept):
    """The subgraph induced by the kept vertices, renumbered by newid:
    (prow int64[kept+1], pcol int32[nnz])."""
    lib = _load()
    row, col = _csr(n, row_ptr, col_idx)
    nid = np.ascontiguousarray(newid, dtype=np.int32)
    prow = np.zeros(kept + 1, dtype=np.int64)
    pcol = np.zeros(max(col.shape[0], 1), dtype=np.int32)
    e = lib.oracle_pruned_csr(n, _p(row), _p(col), _p(nid), _p(prow), _p(pcol))
    return prow, pcol[:e]


def reinsert(n, row_ptr, col_idx, newid, anchor, w, prow, pcol, ppos, d=1.0):
    """Reinsertion (Section 4.6): the full placement float64[n, 2] from the
    placement ppos of the pruned graph."""
    lib = _load()
    row, col = _csr(n, row_ptr, col_idx)
    kept = prow.shape[0] - 1
    nid = np.ascontiguousarray(newid, dtype=np.int32)
    anc = np.ascontiguousarray(anchor, dtype=np.int32)
    ww = np.ascontiguousarray(w, dtype=np.int32)
    pr = np.ascontiguousarray(prow, dtype=np.int64)
    pc = np.ascontiguousarray(pcol, dtype=np.int32)
    P = _pos(ppos, kept)
    out = np.zeros((n, 2), dtype=np.float64)
    lib.oracle_reinsert(n, _p(row), _p(col), _p(nid), _p(anc), _p(ww), _p(pr), _p(pc), _p(P),
                        float(d), _p(out))
    return out


def pipeline(n, row_ptr, col_idx, pos0, k, iters, d=1.0, p=2, q=1, schedule=SCHED_LINEAR,
             t0=0.0):
    """Prune (Section 4.3), lay out the pruned graph with repulsion weights
    1 + w (Sections 4.5, 4.6; default t0 from the pruned graph), reinsert
    (Section 4.6). pos0 is the full initial placement; the kept vertices
    start from their own rows of it. Returns the full final placement."""
    anchor, w, newid, kept = prune(n, row_ptr, col_idx)
    prow, pcol = pruned_csr(n, row_ptr, col_idx, newid, kept)
    keep = newid >= 0
    ppos0 = np.ascontiguousarray(np.asarray(pos0, dtype=np.float64).reshape(n, 2)[keep])
    wt = 1.0 + w[keep].astype(np.float64)
    krow, kcol = khop(kept, prow, pcol, k)
    ppos = run(kept, prow, pcol, krow, kcol, ppos0, iters, d, p, q, schedule, t0, wt=wt)
    return reinsert(n, row_ptr, col_idx, newid, anchor, w, prow, pcol, ppos, d)


def components(n, row_ptr, col_idx):
    """Connected components (Section 4.6): (label int32[n], count), numbered
    in the order of their smallest vertex id."""
    lib = _load()
    row, col = _csr(n, row_ptr, col_idx)
    label = np.zeros(max(n, 1), dtype=np.int32)
    count = lib.oracle_components(n, _p(row), _p(col), _p(label))
    if count < 0:
        raise MemoryError("oracle_components")
    return label[:n], int(count)


def pack(bbox, size, gap):
    """Shelf packing of component boxes (float64[c, 4]: xmin, ymin, xmax,
    ymax) by decreasing size: the translations float64[c, 2]."""
    lib = _load()
    bb = np.ascontiguousarray(bbox, dtype=np.float64).reshape(-1, 4)
    sz = np.ascontiguousarray(size, dtype=np.int64)
    c = bb.shape[0]
    off = np.zeros((max(c, 1), 2), dtype=np.float64)
    if lib.oracle_pack(c, _p(bb), _p(sz), float(gap), _p(off)) != 0:
        raise MemoryError("oracle_pack")
    return off[:c]


def components_layout(n, row_ptr, col_idx, pos0, k, iters, d=1.0, p=2, q=1,
                      schedule=SCHED_LINEAR, t0=0.0, gap=0.0):
    """Every connected component laid out on its own (its own default initial
    temperature from its own n and initial frame, Section 5.1), then the
    drawings packed into rows (Section 4.6). gap <= 0 means d. Returns the
    full final placement."""
    row, col = _csr(n, row_ptr, col_idx)
    P0 = _pos(pos0, n)
    label, count = components(n, row, col)
    out = np.zeros((n, 2), dtype=np.float64)
    bbox = np.zeros((count, 4), dtype=np.float64)
    size = np.bincount(label, minlength=count).astype(np.int64)
    order = np.argsort(label, kind="stable")  # vertices by component, ascending ids
    starts = np.concatenate([[0], np.cumsum(size)])
    local = np.zeros(n, dtype=np.int64)
    for c in range(count):
        vs = order[starts[c]:starts[c + 1]]
        local[vs] = np.arange(len(vs))
    for c in range(count):
        vs = order[starts[c]:starts[c + 1]]
        # the component's CSR in local ids (rows stay ascending)
        lens = row[vs + 1] - row[vs]
        crow = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        ccol = local[np.concatenate([col[row[v]:row[v + 1]] for v in vs])] \
            if crow[-1] > 0 else np.zeros(0, dtype=np.int64)
        ccol = ccol.astype(np.int32)
        krow, kcol = khop(len(vs), crow, ccol, k)
        res = run(len(vs), crow, ccol, krow, kcol, P0[vs], iters, d, p, q, schedule, t0)
        out[vs] = res
        bbox[c] = [res[:, 0].min(), res[:, 1].min(), res[:, 0].max(), res[:, 1].max()]
    off = pack(bbox, size, d if gap <= 0 else gap)
    return out + off[label]
