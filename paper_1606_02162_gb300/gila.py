"""Python binding of libgila (ctypes): argument marshalling only.

Every function here has the name of the C entry point it calls (see
include/gila.h) and does no arithmetic of the method: all compute runs in
the CUDA kernels of the library. Device placements are torch CUDA tensors
(float32 [n, 2] in the FP32 modes, float64 [n, 2] in FP64); work is issued
on torch's current CUDA stream. There is no CPU fallback: if libgila.so is
missing the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgila.so")

GILA_OK = 0
GILA_EINVAL = 1
GILA_ENOMEM = 2
GILA_EBUDGET = 3
GILA_ETIMEDOUT = 4
GILA_ECUDA = 5
GILA_EBUSY = 6
GILA_ESTATE = 7

GILA_FP32 = 0
GILA_FP64 = 1
GILA_FP32_COMPENSATED = 2
GILA_FP64_ORDERED = 3

GILA_COOL_LINEAR = 0
GILA_COOL_GEOMETRIC = 1

GILA_GRAPH_VALIDATE = 1
GILA_GRAPH_SIMPLIFY = 2

_STATUS = {0: "GILA_OK", 1: "GILA_EINVAL", 2: "GILA_ENOMEM", 3: "GILA_EBUDGET",
           4: "GILA_ETIMEDOUT", 5: "GILA_ECUDA", 6: "GILA_EBUSY", 7: "GILA_ESTATE"}


class gila_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("iters", ctypes.c_int32), ("d", ctypes.c_double),
                ("t0", ctypes.c_double), ("schedule", ctypes.c_int32), ("p", ctypes.c_int32),
                ("q", ctypes.c_int32), ("precision", ctypes.c_int32)]


class gila_metrics(ctypes.Structure):
    _fields_ = [("edge_mean", ctypes.c_double), ("edge_std", ctypes.c_double),
                ("edge_cv", ctypes.c_double), ("rep_total", ctypes.c_double),
                ("att_total", ctypes.c_double), ("rep_att_ratio", ctypes.c_double)]


class gila_tuning(ctypes.Structure):
    _fields_ = [("tiled", ctypes.c_int32), ("tile_vertices", ctypes.c_int32),
                ("min_segment", ctypes.c_int32), ("small_max", ctypes.c_int32),
                ("warp_max", ctypes.c_int32), ("block_max", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("bank_spread", ctypes.c_int32), ("step_schedule", ctypes.c_int32)]


class gila_batch_tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("group4_max", ctypes.c_int32), ("group8_max", ctypes.c_int32),
                ("group16_max", ctypes.c_int32)]


class GilaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every exported entry point
P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
D = ctypes.c_double
PP = ctypes.POINTER(gila_params)
SIGNATURES = [
    ("gila_params_default", None, [PP]),
    ("gila_csr_validate", ctypes.c_int, [I64, P, P]),
    ("gila_graph_create", ctypes.c_int, [I64, P, P, I32, ctypes.POINTER(P)]),
    ("gila_graph_destroy", None, [P]),
    ("gila_graph_set_stream", ctypes.c_int, [P, P]),
    ("gila_graph_info", ctypes.c_int, [P, P, P, P, P]),
    ("gila_graph_tune", ctypes.c_int, [P, ctypes.POINTER(gila_tuning)]),
    ("gila_graph_get_tuning", ctypes.c_int, [P, ctypes.POINTER(gila_tuning)]),
    ("gila_build_khop", ctypes.c_int, [P, I32, ctypes.POINTER(I64)]),
    ("gila_khop_reset", ctypes.c_int, [P]),
    ("gila_khop_export", ctypes.c_int, [P, P, P]),
    ("gila_khop_export_rows", ctypes.c_int, [P, I64, P, P, P, I64]),
    ("gila_layout_step", ctypes.c_int, [P, PP, D, P, P, P]),
    ("gila_layout_run_device", ctypes.c_int, [P, PP, P]),
    ("gila_layout_run", ctypes.c_int, [P, PP, P, P, P]),
    ("gila_layout_metrics", ctypes.c_int, [P, PP, P, ctypes.POINTER(gila_metrics)]),
    ("gila_temperature", D, [PP, D, I32]),
    ("gila_profile_enable", ctypes.c_int, [P, I32]),
    ("gila_profile_read", ctypes.c_int, [P, P, P, P, P]),
    ("gila_profile_read_kernel", ctypes.c_int, [P, P, P, ctypes.c_char_p, I32]),
    ("gila_last_error", ctypes.c_char_p, []),
    ("gila_kernel_launches", ctypes.c_int64, []),
    ("gila_khop_count_noalloc", ctypes.c_int, [I64, P, P, I32, P, ctypes.POINTER(I64), P]),
    ("gila_batch_create", ctypes.c_int, [I32, P, P, P, I32, ctypes.POINTER(P)]),
    ("gila_batch_destroy", None, [P]),
    ("gila_batch_set_stream", ctypes.c_int, [P, P]),
    ("gila_batch_info", ctypes.c_int, [P, P, P, P]),
    ("gila_batch_build_khop", ctypes.c_int, [P, I32, ctypes.POINTER(I64)]),
    ("gila_batch_khop_reset", ctypes.c_int, [P]),
    ("gila_batch_khop_export", ctypes.c_int, [P, P, P]),
    ("gila_batch_tune", ctypes.c_int, [P, ctypes.POINTER(gila_batch_tuning)]),
    ("gila_batch_get_tuning", ctypes.c_int, [P, I32, ctypes.POINTER(gila_batch_tuning)]),
    ("gila_batch_autotune", ctypes.c_int, [P, PP, P, I32, ctypes.POINTER(gila_batch_tuning)]),
    ("gila_layout_batch_device", ctypes.c_int, [P, PP, P]),
    ("gila_layout_batch_run", ctypes.c_int, [P, PP, P, P]),
    ("gila_layout_batch", ctypes.c_int, [P, I32, PP, P, P]),
    ("gila_graph_set_repulsion_weights", ctypes.c_int, [P, P]),
    ("gila_prune_degree_one", ctypes.c_int, [P, ctypes.POINTER(P)]),
    ("gila_pruned_destroy", None, [P]),
    ("gila_pruned_graph", P, [P]),
    ("gila_pruned_info", ctypes.c_int, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
    ("gila_pruned_export", ctypes.c_int, [P, P, P, P]),
    ("gila_pruned_gather", ctypes.c_int, [P, I32, P, P]),
    ("gila_reinsert_degree_one", ctypes.c_int, [P, PP, P, P]),
    ("gila_layout_pruned_run_device", ctypes.c_int, [P, PP, P]),
    ("gila_layout_pruned_run", ctypes.c_int, [P, PP, P, P]),
    ("gila_graph_components", ctypes.c_int, [P, P, ctypes.POINTER(I32)]),
    ("gila_graph_set_wait_test", ctypes.c_int, [P, I32]),
    ("gila_layout_components_run", ctypes.c_int, [P, PP, D, P, P, ctypes.POINTER(I32)]),
]


def load(path: str | None = None):
    """Load libgila.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"libgila.so not found at {p}: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(p)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int):
    if status != GILA_OK:
        raise GilaError(status, load().gila_last_error().decode(errors="replace"))


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t) -> int:
    """Device address of a torch tensor or an int address."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _torch_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def params(k=2, iters=300, d=1.0, t0=0.0, schedule=GILA_COOL_LINEAR, p=2, q=1,
           precision=GILA_FP32) -> gila_params:
    return gila_params(int(k), int(iters), float(d), float(t0), int(schedule), int(p), int(q),
                       int(precision))


def gila_params_default() -> gila_params:
    prm = gila_params()
    load().gila_params_default(ctypes.byref(prm))
    return prm


def gila_csr_validate(n, row_ptr, col_idx) -> int:
    """Host-only CSR check; returns the status (0 = valid)."""
    row = _np(row_ptr, np.int64)
    col = _np(col_idx, np.int32)
    return load().gila_csr_validate(int(n), _ptr(row), _ptr(col))


def gila_kernel_launches() -> int:
    return load().gila_kernel_launches()


def gila_khop_count_noalloc(n, row_ptr_dev, col_idx_dev, k, counts_dev, stream=None) -> int:
    """|N_v(k)| of every vertex into counts_dev (int64 device tensor of n),
    from caller-owned device CSR arrays, with no allocation inside the
    library; returns the total. stream: cudaStream_t address, None = torch's
    current stream."""
    total = I64()
    s = _torch_stream() if stream is None else stream
    _check(load().gila_khop_count_noalloc(int(n), _dev_ptr(row_ptr_dev), _dev_ptr(col_idx_dev),
                                          int(k), _dev_ptr(counts_dev), ctypes.byref(total), s))
    return total.value


def gila_last_error() -> str:
    return load().gila_last_error().decode(errors="replace")


def gila_graph_create(n, row_ptr, col_idx, flags=0) -> int:
    row = _np(row_ptr, np.int64)
    col = _np(col_idx, np.int32)
    h = ctypes.c_void_p()
    _check(load().gila_graph_create(int(n), _ptr(row), _ptr(col), int(flags), ctypes.byref(h)))
    return h.value


def gila_graph_destroy(g) -> None:
    if g:
        load().gila_graph_destroy(g)


def gila_graph_set_stream(g, stream=None) -> None:
    """stream: a cudaStream_t address (int); None = torch's current stream."""
    s = _torch_stream() if stream is None else stream
    _check(load().gila_graph_set_stream(g, s))


def gila_graph_info(g) -> dict:
    n, nnz, kb, nk = I64(), I64(), I32(), I64()
    _check(load().gila_graph_info(g, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(kb),
                                  ctypes.byref(nk)))
    return {"n": n.value, "nnz_adj": nnz.value, "k_built": kb.value, "nnz_khop": nk.value}


def gila_graph_tune(g, tiled=-1, tile_vertices=0, min_segment=0, small_max=0, warp_max=0,
                    block_max=0, chunk=0, ctas_per_sm=0, bank_spread=0,
                    step_schedule=0) -> None:
    t = gila_tuning(int(tiled), int(tile_vertices), int(min_segment), int(small_max),
                    int(warp_max), int(block_max), int(chunk), int(ctas_per_sm),
                    int(bank_spread), int(step_schedule))
    _check(load().gila_graph_tune(g, ctypes.byref(t)))


def gila_graph_get_tuning(g) -> dict:
    t = gila_tuning()
    _check(load().gila_graph_get_tuning(g, ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in gila_tuning._fields_}


def gila_build_khop(g, k) -> int:
    nnz = I64()
    _check(load().gila_build_khop(g, int(k), ctypes.byref(nnz)))
    return nnz.value


def gila_khop_reset(g) -> None:
    _check(load().gila_khop_reset(g))


def gila_khop_export(g):
    info = gila_graph_info(g)
    krow = np.zeros(info["n"] + 1, dtype=np.int64)
    kcol = np.zeros(max(info["nnz_khop"], 1), dtype=np.int32)
    _check(load().gila_khop_export(g, _ptr(krow), _ptr(kcol)))
    return krow, kcol[: info["nnz_khop"]]


def gila_khop_export_rows(g, sel):
    """Rows of the selected vertices: (counts int64[s], concatenated int32 rows)."""
    sel = _np(sel, np.int64)
    counts = np.zeros(max(len(sel), 1), dtype=np.int64)
    _check(load().gila_khop_export_rows(g, len(sel), _ptr(sel), _ptr(counts), None, 0))
    total = int(counts[: len(sel)].sum())
    cols = np.zeros(max(total, 1), dtype=np.int32)
    _check(load().gila_khop_export_rows(g, len(sel), _ptr(sel), _ptr(counts), _ptr(cols), total))
    return counts[: len(sel)], cols[:total]


def gila_layout_step(g, prm, t, pos_in, pos_out, disp_out=None) -> None:
    _check(load().gila_layout_step(g, ctypes.byref(prm), float(t), _dev_ptr(pos_in),
                                   _dev_ptr(pos_out), _dev_ptr(disp_out)))


def gila_layout_run_device(g, prm, pos) -> None:
    _check(load().gila_layout_run_device(g, ctypes.byref(prm), _dev_ptr(pos)))


def gila_layout_run(g, prm, pos_in, pos_out=None, metrics=False):
    """Host placement in (float64 [n, 2]), host placement out; with
    metrics=True also the quality figures of the result: (placement, dict)."""
    src = _np(pos_in, np.float64)
    out = np.empty_like(src) if pos_out is None else pos_out
    m = gila_metrics() if metrics else None
    _check(load().gila_layout_run(g, ctypes.byref(prm), _ptr(src), _ptr(out),
                                  ctypes.byref(m) if metrics else None))
    if metrics:
        return out, {f: getattr(m, f) for f, _ in gila_metrics._fields_}
    return out


def gila_layout_metrics(g, prm, pos) -> dict:
    m = gila_metrics()
    _check(load().gila_layout_metrics(g, ctypes.byref(prm), _dev_ptr(pos), ctypes.byref(m)))
    return {f: getattr(m, f) for f, _ in gila_metrics._fields_}


def gila_temperature(prm, t0, i) -> float:
    return load().gila_temperature(ctypes.byref(prm), float(t0), int(i))


def gila_profile_enable(g, on=True) -> None:
    """on: False/0 off, True/1 builds and iteration sequences, 2 also each
    iteration's repulsion kernel on its own."""
    _check(load().gila_profile_enable(g, int(on)))


def gila_profile_read(g) -> dict:
    b, bms, it, ims = I64(), D(), I64(), D()
    _check(load().gila_profile_read(g, ctypes.byref(b), ctypes.byref(bms), ctypes.byref(it),
                                    ctypes.byref(ims)))
    return {"builds": b.value, "build_ms": bms.value, "iter_launches": it.value,
            "iter_ms": ims.value}


def gila_profile_read_kernel(g) -> dict:
    n, ms = I64(), D()
    name = ctypes.create_string_buffer(64)
    _check(load().gila_profile_read_kernel(g, ctypes.byref(n), ctypes.byref(ms), name, 64))
    return {"launches": n.value, "ms": ms.value, "name": name.value.decode()}


class Graph:
    """Owning wrapper of a gila_graph handle bound to torch's current stream."""

    def __init__(self, n, row_ptr, col_idx, flags=0):
        self.n = int(n)
        self.handle = gila_graph_create(n, row_ptr, col_idx, flags)
        gila_graph_set_stream(self.handle)

    @classmethod
    def from_inputs(cls, g, flags=0):
        return cls(g.n, g.row_ptr, g.col_idx, flags)

    def close(self):
        if self.handle:
            gila_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------------ batches

def _ptr_array(arrs, ctype):
    return (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs]) if arrs else None


def gila_batch_create(graphs, flags=0) -> int:
    """graphs: sequence of objects with n, row_ptr, col_idx (host arrays)."""
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    rows = [_np(g.row_ptr, np.int64) for g in graphs]
    cols = [_np(g.col_idx, np.int32) for g in graphs]
    rp = _ptr_array(rows, ctypes.c_int64)
    cp = _ptr_array(cols, ctypes.c_int32)
    h = ctypes.c_void_p()
    _check(load().gila_batch_create(len(graphs), _ptr(ns) if len(graphs) else None,
                                    ctypes.cast(rp, P) if rp else None,
                                    ctypes.cast(cp, P) if cp else None, int(flags),
                                    ctypes.byref(h)))
    return h.value


def gila_batch_destroy(b) -> None:
    if b:
        load().gila_batch_destroy(b)


def gila_batch_set_stream(b, stream=None) -> None:
    s = _torch_stream() if stream is None else stream
    _check(load().gila_batch_set_stream(b, s))


def gila_batch_info(b) -> dict:
    c, n, k = I32(), I64(), I64()
    _check(load().gila_batch_info(b, ctypes.byref(c), ctypes.byref(n), ctypes.byref(k)))
    return {"count": c.value, "total_n": n.value, "nnz_khop": k.value}


def gila_batch_build_khop(b, k) -> int:
    nnz = I64()
    _check(load().gila_batch_build_khop(b, int(k), ctypes.byref(nnz)))
    return nnz.value


def gila_batch_khop_reset(b) -> None:
    _check(load().gila_batch_khop_reset(b))


def gila_batch_khop_export(b):
    """The whole batch's k-hop lists (union numbering): (krow, kcol)."""
    info = gila_batch_info(b)
    krow = np.zeros(info["total_n"] + 1, dtype=np.int64)
    kcol = np.zeros(max(info["nnz_khop"], 1), dtype=np.int32)
    _check(load().gila_batch_khop_export(b, _ptr(krow), _ptr(kcol)))
    return krow, kcol[: info["nnz_khop"]]


def gila_batch_tune(b, threads=0, ctas_per_sm=0, group4_max=0, group8_max=0,
                    group16_max=0) -> None:
    t = gila_batch_tuning(int(threads), int(ctas_per_sm), int(group4_max), int(group8_max),
                          int(group16_max))
    _check(load().gila_batch_tune(b, ctypes.byref(t)))


def gila_batch_get_tuning(b, precision=GILA_FP32) -> dict:
    t = gila_batch_tuning()
    _check(load().gila_batch_get_tuning(b, int(precision), ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in gila_batch_tuning._fields_}


def gila_batch_autotune(b, prm, pos, probe_iters=5) -> dict:
    t = gila_batch_tuning()
    _check(load().gila_batch_autotune(b, ctypes.byref(prm), _dev_ptr(pos), int(probe_iters),
                                      ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in gila_batch_tuning._fields_}


def gila_layout_batch_device(b, prm, pos) -> None:
    _check(load().gila_layout_batch_device(b, ctypes.byref(prm), _dev_ptr(pos)))


def gila_layout_batch_run(b, prm, pos_in, pos_out=None) -> np.ndarray:
    src = _np(pos_in, np.float64)
    out = np.empty_like(src) if pos_out is None else pos_out
    _check(load().gila_layout_batch_run(b, ctypes.byref(prm), _ptr(src), _ptr(out)))
    return out


def gila_layout_batch(graph_handles, prm, pos_in_list):
    """Lay out already-created graphs together; returns a list of host placements."""
    ins = [_np(p, np.float64) for p in pos_in_list]
    outs = [np.empty_like(p) for p in ins]
    handles = list(graph_handles)
    hs = (ctypes.c_void_p * len(handles))(*handles) if handles else None
    ip = _ptr_array(ins, ctypes.c_double)
    op = _ptr_array(outs, ctypes.c_double)
    _check(load().gila_layout_batch(ctypes.cast(hs, P) if hs else None, len(ins),
                                    ctypes.byref(prm), ctypes.cast(ip, P) if ip else None,
                                    ctypes.cast(op, P) if op else None))
    return outs


class Batch:
    """Owning wrapper of a gila_batch bound to torch's current stream."""

    def __init__(self, graphs, flags=0):
        self.graphs = list(graphs)
        self.handle = gila_batch_create(self.graphs, flags)
        gila_batch_set_stream(self.handle)
        self.offsets = np.concatenate([[0], np.cumsum([g.n for g in self.graphs])]).astype(np.int64)

    def close(self):
        if self.handle:
            gila_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------------ serving

class gila_job_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("nnz_khop", ctypes.c_int64),
                ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]


class gila_server_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("running", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_size_t), ("bytes_peak", ctypes.c_size_t),
                ("budget", ctypes.c_size_t)]


SIGNATURES += [
    ("gila_server_create", ctypes.c_int, [ctypes.c_size_t, I32, ctypes.POINTER(P)]),
    ("gila_server_destroy", None, [P]),
    ("gila_server_submit", ctypes.c_int, [P, I64, P, P, PP, P, ctypes.POINTER(ctypes.c_uint64)]),
    ("gila_server_wait", ctypes.c_int, [P, ctypes.c_uint64, I32, P,
                                        ctypes.POINTER(gila_job_info)]),
    ("gila_server_poll", ctypes.c_int, [P, ctypes.c_uint64, ctypes.POINTER(I32)]),
    ("gila_server_get_stats", ctypes.c_int, [P, ctypes.POINTER(gila_server_stats)]),
]


def gila_server_create(budget_bytes, max_slots) -> int:
    h = ctypes.c_void_p()
    _check(load().gila_server_create(int(budget_bytes), int(max_slots), ctypes.byref(h)))
    return h.value


def gila_server_destroy(s) -> None:
    if s:
        load().gila_server_destroy(s)


def gila_server_submit(s, n, row_ptr, col_idx, prm, pos_in) -> int:
    row = _np(row_ptr, np.int64)
    col = _np(col_idx, np.int32)
    pos = _np(pos_in, np.float64)
    t = ctypes.c_uint64()
    _check(load().gila_server_submit(s, int(n), _ptr(row), _ptr(col), ctypes.byref(prm),
                                     _ptr(pos), ctypes.byref(t)))
    return t.value


def gila_server_wait(s, ticket, n, timeout_ms=-1):
    """Returns (placement float64[n, 2], info dict); raises GilaError on
    failure or timeout (status GILA_ETIMEDOUT)."""
    out = np.empty((n, 2), dtype=np.float64)
    info = gila_job_info()
    _check(load().gila_server_wait(s, ctypes.c_uint64(ticket), int(timeout_ms), _ptr(out),
                                   ctypes.byref(info)))
    return out, {f: getattr(info, f) for f, _ in gila_job_info._fields_}


def gila_server_poll(s, ticket) -> bool:
    d = I32()
    _check(load().gila_server_poll(s, ctypes.c_uint64(ticket), ctypes.byref(d)))
    return bool(d.value)


def gila_server_get_stats(s) -> dict:
    st = gila_server_stats()
    _check(load().gila_server_get_stats(s, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in gila_server_stats._fields_}


class Server:
    """Owning wrapper of a gila_server; remembers each ticket's vertex count."""

    def __init__(self, budget_bytes, max_slots):
        self.handle = gila_server_create(budget_bytes, max_slots)
        self._n = {}

    def submit(self, graph, pos, prm) -> int:
        t = gila_server_submit(self.handle, graph.n, graph.row_ptr, graph.col_idx, prm, pos)
        self._n[t] = graph.n
        return t

    def wait(self, ticket, timeout_ms=-1):
        # unknown tickets go to the library, which reports GILA_EINVAL
        out = gila_server_wait(self.handle, ticket, self._n.get(ticket, 0), timeout_ms)
        self._n.pop(ticket, None)
        return out

    def poll(self, ticket) -> bool:
        return gila_server_poll(self.handle, ticket)

    def stats(self) -> dict:
        return gila_server_get_stats(self.handle)

    def close(self):
        if self.handle:
            gila_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------------ pruning

def gila_graph_set_repulsion_weights(g, weights) -> None:
    """Per-vertex repulsion weights (float64[n]) or None to remove them."""
    if weights is None:
        _check(load().gila_graph_set_repulsion_weights(g, None))
        return
    w = _np(weights, np.float64)
    _check(load().gila_graph_set_repulsion_weights(g, _ptr(w)))


def gila_prune_degree_one(g) -> int:
    out = P()
    _check(load().gila_prune_degree_one(g, ctypes.byref(out)))
    return out.value


def gila_pruned_destroy(p) -> None:
    load().gila_pruned_destroy(p)


def gila_pruned_graph(p) -> int:
    return load().gila_pruned_graph(p)


def gila_pruned_info(p) -> dict:
    k, r = I64(), I64()
    _check(load().gila_pruned_info(p, ctypes.byref(k), ctypes.byref(r)))
    return {"kept": k.value, "removed": r.value}


def gila_pruned_export(p, n):
    """(anchor, w, newid), each int32[n] over the original ids."""
    a = np.empty(n, dtype=np.int32)
    w = np.empty(n, dtype=np.int32)
    i = np.empty(n, dtype=np.int32)
    _check(load().gila_pruned_export(p, _ptr(a), _ptr(w), _ptr(i)))
    return a, w, i


def gila_pruned_gather(p, precision, pos_full, pos_pruned) -> None:
    _check(load().gila_pruned_gather(p, int(precision), _dev_ptr(pos_full), _dev_ptr(pos_pruned)))


def gila_reinsert_degree_one(p, prm, pos_pruned, pos_full) -> None:
    _check(load().gila_reinsert_degree_one(p, ctypes.byref(prm), _dev_ptr(pos_pruned),
                                           _dev_ptr(pos_full)))


def gila_layout_pruned_run_device(p, prm, pos_full) -> None:
    _check(load().gila_layout_pruned_run_device(p, ctypes.byref(prm), _dev_ptr(pos_full)))


def gila_layout_pruned_run(p, prm, pos_in, pos_out=None) -> np.ndarray:
    src = _np(pos_in, np.float64)
    out = np.empty_like(src) if pos_out is None else pos_out
    _check(load().gila_layout_pruned_run(p, ctypes.byref(prm), _ptr(src), _ptr(out)))
    return out


class Pruned:
    """Owning wrapper of a gila_pruned made from a Graph (which must outlive it)."""

    def __init__(self, graph: "Graph"):
        self.graph = graph
        self.handle = gila_prune_degree_one(graph.handle)
        info = gila_pruned_info(self.handle)
        self.kept, self.removed = info["kept"], info["removed"]

    @property
    def pruned_graph(self) -> int:
        return gila_pruned_graph(self.handle)

    def close(self):
        if self.handle:
            gila_pruned_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# --------------------------------------------------------------- components

def gila_graph_components(g, n):
    """(label int32[n], count) of the connected components."""
    label = np.zeros(max(n, 1), dtype=np.int32)
    c = I32()
    _check(load().gila_graph_components(g, _ptr(label), ctypes.byref(c)))
    return label[:n], c.value


def gila_layout_components_run(g, prm, pos_in, gap=0.0, pos_out=None):
    """Per-component layout and packing: (placement float64[n, 2], count)."""
    src = _np(pos_in, np.float64)
    out = np.empty_like(src) if pos_out is None else pos_out
    c = I32()
    _check(load().gila_layout_components_run(g, ctypes.byref(prm), float(gap), _ptr(src),
                                             _ptr(out), ctypes.byref(c)))
    return out, c.value


def gila_graph_set_wait_test(g, on) -> None:
    """Failure-detection test hook (see include/gila.h)."""
    _check(load().gila_graph_set_wait_test(g, 1 if on else 0))
