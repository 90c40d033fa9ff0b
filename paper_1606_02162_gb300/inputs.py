"""Seeded synthetic inputs: graphs in CSR form and initial placements.

This module is shared by the CUDA path, the tests and the benchmark. It holds
no arithmetic of the layout method itself: it only builds graphs and random
coordinates. Every generator is a pure function of its arguments and seed
(numpy's PCG64 stream), so the same call gives the same arrays on x86_64 and
aarch64.

Graph families follow the workloads of Section 5.2 (Synth-Random:
Erdos-Renyi; Synth-ScaleFree: Barabasi-Albert; density 2-3) plus the shapes
used for the scaled configurations: a 2D grid, a triangulated mesh, a
Chung-Lu power-law graph and a mix of small trees, grids and random graphs.
As in Table 1 of the paper, graphs are simple and undirected: self-loops and
parallel edges are removed, and every edge is stored in both directions.
"""
from __future__ import annotations

import heapq
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Graph:
    """Undirected simple graph in symmetric CSR form.

    row_ptr: int64[n+1]; col_idx: int32[2E]. Row u lists the neighbours of
    u in ascending order. No self-loops, no repeated entries.
    """

    name: str
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def num_edges(self) -> int:
        return int(self.col_idx.shape[0] // 2)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def edge_list(self) -> tuple[np.ndarray, np.ndarray]:
        """Undirected edges (u, v) with u < v, in CSR order."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))
        dst = self.col_idx.astype(np.int64)
        keep = src < dst
        return src[keep], dst[keep]


def csr_from_edges(n: int, u, v, name: str = "graph", meta=None) -> Graph:
    """Symmetric, deduplicated CSR from an undirected edge list.

    Self-loops and repeated pairs are dropped; each remaining edge is stored
    as (u, v) and (v, u); rows come out sorted ascending.
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if u.size:
        if u.min() < 0 or v.min() < 0 or u.max() >= n or v.max() >= n:
            raise ValueError("edge endpoint out of range")
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.minimum(u, v)
    b = np.maximum(u, v)
    key = np.unique(a * n + b)
    a = key // n
    b = key % n
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    order = np.lexsort((dst, src))
    src = src[order]
    dst = dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, src + 1, 1)
    np.cumsum(row_ptr, out=row_ptr)
    return Graph(name, int(n), row_ptr, dst.astype(np.int32), dict(meta or {}))


# --------------------------------------------------------------------------
# Deterministic families
# --------------------------------------------------------------------------

def grid(rows: int, cols: int) -> Graph:
    """rows x cols 4-neighbour grid; vertex (i, j) has id i*cols + j."""
    ids = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    us = [ids[:, :-1].ravel(), ids[:-1, :].ravel()]
    vs = [ids[:, 1:].ravel(), ids[1:, :].ravel()]
    return csr_from_edges(rows * cols, np.concatenate(us), np.concatenate(vs),
                          f"grid{rows}x{cols}", {"rows": rows, "cols": cols})


def tri_mesh(rows: int, cols: int) -> Graph:
    """rows x cols grid with each unit square split by its (i,j)-(i+1,j+1)
    diagonal: a triangulated planar mesh, interior degree 6."""
    ids = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    us = [ids[:, :-1].ravel(), ids[:-1, :].ravel(), ids[:-1, :-1].ravel()]
    vs = [ids[:, 1:].ravel(), ids[1:, :].ravel(), ids[1:, 1:].ravel()]
    return csr_from_edges(rows * cols, np.concatenate(us), np.concatenate(vs),
                          f"trimesh{rows}x{cols}", {"rows": rows, "cols": cols})


def path(n: int) -> Graph:
    a = np.arange(n - 1)
    return csr_from_edges(n, a, a + 1, f"path{n}")


def cycle(n: int) -> Graph:
    a = np.arange(n)
    return csr_from_edges(n, a, (a + 1) % n, f"cycle{n}")


def star(n: int) -> Graph:
    """Vertex 0 joined to vertices 1..n-1."""
    return csr_from_edges(n, np.zeros(n - 1, dtype=np.int64), np.arange(1, n), f"star{n}")


def complete(n: int) -> Graph:
    a, b = np.triu_indices(n, 1)
    return csr_from_edges(n, a, b, f"complete{n}")


def near_square_grid(n: int) -> Graph:
    """A grid with about n vertices: r = round(sqrt n) rows, round(n / r) columns."""
    r = max(1, int(round(math.sqrt(n))))
    c = max(1, int(round(n / r)))
    g = grid(r, c)
    g.name = f"nsgrid{r}x{c}"
    return g


# --------------------------------------------------------------------------
# Random families
# --------------------------------------------------------------------------

def barabasi_albert(n: int, m: int, seed: int) -> Graph:
    """Barabasi-Albert preferential attachment (Section 5.2, Synth-ScaleFree).

    Start from the clique on vertices 0..m; every later vertex v picks m
    distinct earlier targets, each drawn with probability proportional to its
    current degree (uniform draw from the list of edge endpoints), then joins
    them. E = m(m+1)/2 + m(n-m-1) exactly.
    """
    if n <= m:
        raise ValueError("need n > m")
    rng = np.random.default_rng(seed)
    E = m * (m + 1) // 2 + m * (n - m - 1)
    ends = np.empty(2 * E, dtype=np.int64)
    L = 0
    for a in range(m + 1):
        for b in range(a + 1, m + 1):
            ends[L] = a
            ends[L + 1] = b
            L += 2
    src = np.empty(E, dtype=np.int64)
    dst = np.empty(E, dtype=np.int64)
    e = L // 2
    src[:e] = ends[0:L:2]
    dst[:e] = ends[1:L:2]
    buf = rng.random(4 * m * n + 64)
    bi = 0
    ends_l = ends  # local alias
    for v in range(m + 1, n):
        chosen = []
        while len(chosen) < m:
            if bi >= buf.shape[0]:
                buf = rng.random(4 * m * n + 64)
                bi = 0
            t = int(ends_l[int(buf[bi] * L)])
            bi += 1
            if t not in chosen:
                chosen.append(t)
        for t in chosen:
            ends_l[L] = v
            ends_l[L + 1] = t
            L += 2
            src[e] = v
            dst[e] = t
            e += 1
    assert e == E
    return csr_from_edges(n, src, dst, f"ba_n{n}_m{m}_s{seed}", {"m": m, "seed": seed})


def barabasi_albert_fast(n: int, m: int, seed: int) -> Graph:
    """Preferential attachment without the per-vertex loop (for long request
    streams). Every new vertex v draws m endpoint slots uniformly from the
    2E_v slots that exist before it (a slot holds one end of an earlier
    edge, so a vertex is drawn in proportion to its degree); a slot that holds
    the far end of an earlier edge is resolved by following that edge's own
    draw (pointer jumping). Repeated picks by the same vertex are dropped, so
    E is slightly below m(m+1)/2 + m(n-m-1)."""
    if n <= m:
        raise ValueError("need n > m")
    rng = np.random.default_rng(seed)
    e0 = m * (m + 1) // 2
    E = e0 + m * (n - m - 1)
    src = np.empty(E, dtype=np.int64)
    dst = np.full(E, -1, dtype=np.int64)
    a, b = np.triu_indices(m + 1, 1)
    src[:e0] = a
    dst[:e0] = b
    v = np.repeat(np.arange(m + 1, n, dtype=np.int64), m)
    src[e0:] = v
    slots_before = 2 * (e0 + (v - m - 1) * m)
    r = (rng.random(E - e0) * slots_before).astype(np.int64)
    even = (r & 1) == 0
    idx = np.arange(e0, E)
    dst[idx[even]] = src[r[even] >> 1]
    ptr = np.full(E, -1, dtype=np.int64)
    ptr[idx[~even]] = (r[~even] - 1) >> 1
    pending = idx[~even]
    while pending.size:
        tgt = ptr[pending]
        known = dst[tgt] >= 0
        dst[pending[known]] = dst[tgt[known]]
        pending = pending[~known]
        ptr[pending] = ptr[ptr[pending]]
    return csr_from_edges(n, src, dst, f"bafast_n{n}_m{m}_s{seed}", {"m": m, "seed": seed})


def _sample_unique_pairs(rng, weights_cdf, n: int, num_edges: int, uniform: bool):
    """Draw endpoint pairs until num_edges distinct non-loop pairs exist;
    keep the first num_edges in draw order."""
    keys = np.empty(0, dtype=np.int64)
    first = np.empty(0, dtype=np.int64)
    drawn = 0
    while True:
        need = num_edges - keys.shape[0]
        if need <= 0:
            break
        batch = int(need * 1.3) + 1024
        if uniform:
            a = rng.integers(0, n, batch, dtype=np.int64)
            b = rng.integers(0, n, batch, dtype=np.int64)
        else:
            a = np.searchsorted(weights_cdf, rng.random(batch), side="right").astype(np.int64)
            b = np.searchsorted(weights_cdf, rng.random(batch), side="right").astype(np.int64)
            np.minimum(a, n - 1, out=a)
            np.minimum(b, n - 1, out=b)
        ok = a != b
        lo = np.minimum(a, b)[ok]
        hi = np.maximum(a, b)[ok]
        k_new = lo * n + hi
        order_new = drawn + np.nonzero(ok)[0]
        drawn += batch
        allk = np.concatenate([keys, k_new])
        allo = np.concatenate([first, order_new])
        uk, idx = np.unique(allk, return_index=True)
        fo = allo[idx]
        srt = np.argsort(fo, kind="stable")
        keys = uk[srt]
        first = fo[srt]
    keys = keys[:num_edges]
    return keys // n, keys % n


def chung_lu(n: int, gamma: float, mean_degree: float, num_edges: int, seed: int) -> Graph:
    """Chung-Lu power-law graph.

    Weights w_i = (i+1)^(-1/(gamma-1)), scaled to mean `mean_degree` and
    capped at sqrt(sum w). Endpoints are drawn independently with
    probability proportional to w; self-loops and repeats are dropped until
    `num_edges` distinct edges exist. Vertices left with degree 0 stay in
    the graph (their k-hop sets are empty).
    """
    rng = np.random.default_rng(seed)
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    w *= mean_degree / w.mean()
    w = np.minimum(w, math.sqrt(w.sum()))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    a, b = _sample_unique_pairs(rng, cdf, n, num_edges, uniform=False)
    g = csr_from_edges(n, a, b, f"chunglu_n{n}_g{gamma}_E{num_edges}_s{seed}",
                       {"gamma": gamma, "seed": seed})
    g.meta["isolated"] = int((np.diff(g.row_ptr) == 0).sum())
    return g


def erdos_renyi(n: int, avg_degree: float, seed: int) -> Graph:
    """G(n, p) with p = avg_degree / (n - 1): the edge count is drawn from
    Binomial(n(n-1)/2, p), then that many distinct pairs uniformly."""
    rng = np.random.default_rng(seed)
    if n < 2:
        return csr_from_edges(n, [], [], f"er_n{n}")
    pairs = n * (n - 1) // 2
    p = min(1.0, avg_degree / (n - 1))
    m = int(rng.binomial(pairs, p))
    m = min(m, pairs)
    if m == pairs:
        a, b = np.triu_indices(n, 1)
    else:
        a, b = _sample_unique_pairs(rng, None, n, m, uniform=True)
    return csr_from_edges(n, a, b, f"er_n{n}_s{seed}", {"seed": seed})


def random_tree(n: int, seed: int) -> Graph:
    """Uniform random labelled tree on n vertices (Pruefer sequence)."""
    if n <= 1:
        return csr_from_edges(max(n, 1), [], [], f"tree{n}")
    if n == 2:
        return csr_from_edges(2, [0], [1], "tree2")
    rng = np.random.default_rng(seed)
    seq = rng.integers(0, n, n - 2).tolist()
    degree = [1] * n
    for x in seq:
        degree[x] += 1
    leaves = [i for i in range(n) if degree[i] == 1]
    heapq.heapify(leaves)
    us, vs = [], []
    for x in seq:
        leaf = heapq.heappop(leaves)
        us.append(leaf)
        vs.append(x)
        degree[x] -= 1
        if degree[x] == 1:
            heapq.heappush(leaves, x)
    a = heapq.heappop(leaves)
    b = heapq.heappop(leaves)
    us.append(a)
    vs.append(b)
    return csr_from_edges(n, us, vs, f"tree_n{n}_s{seed}", {"seed": seed})


def batch_mix(count: int, nmin: int, nmax: int, seed: int) -> list[Graph]:
    """Mix of small graphs: n ~ round(exp U[ln nmin, ln nmax]); the family
    is uniform over {random tree, near-square grid, G(n, 4/(n-1))}."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), count))).astype(np.int64)
    kinds = rng.integers(0, 3, count)
    seeds = rng.integers(0, 2**31 - 1, count)
    out = []
    for n, kind, s in zip(sizes.tolist(), kinds.tolist(), seeds.tolist()):
        if kind == 0:
            out.append(random_tree(n, s))
        elif kind == 1:
            out.append(near_square_grid(n))
        else:
            out.append(erdos_renyi(n, 4.0, s))
    return out


# --------------------------------------------------------------------------
# Placements
# --------------------------------------------------------------------------

def uniform_positions(n: int, seed: int, side: float | None = None) -> np.ndarray:
    """Initial placement: float64[n, 2], uniform in [0, side]^2, side defaults
    to sqrt(n). Row u holds (x_u, y_u)."""
    rng = np.random.default_rng(seed)
    s = math.sqrt(n) if side is None else float(side)
    return rng.random((n, 2)) * s


def serving_requests(count: int, seed: int, emin: float = 1e3, emax: float = 1e6,
                     m: int = 3):
    """Layout-request stream for the serving workload: each request is a
    Barabasi-Albert graph (m = 3) with edge count log-uniform in
    [emin, emax], k drawn from {2, 3} with equal odds. Returns a list of
    dicts with the vertex count, k and a per-request seed; arrival times are
    left to the caller (Poisson at a chosen rate)."""
    rng = np.random.default_rng(seed)
    E = np.exp(rng.uniform(math.log(emin), math.log(emax), count))
    ks = rng.integers(2, 4, count)
    seeds = rng.integers(0, 2**31 - 1, count)
    reqs = []
    for e, k, s in zip(E.tolist(), ks.tolist(), seeds.tolist()):
        n = int(round((e - m * (m + 1) / 2) / m)) + m + 1
        reqs.append({"n": max(n, m + 2), "k": int(k), "seed": int(s)})
    return reqs


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival offsets in seconds of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, count))


# --------------------------------------------------------------------------
# Named workloads (Section 5.2 shapes at the sizes the benchmarks use)
# --------------------------------------------------------------------------

def workload(name: str) -> tuple[Graph, np.ndarray]:
    """Graph and initial placement of a named workload.

    grid32      : 32x32 grid, positions U[0, 32]^2, seed 1
    ba100k      : Barabasi-Albert n=100,000, m=3, seed 2, U[0, sqrt n]^2
    chunglu250k : Chung-Lu gamma=2.3, n=250,000, E=1,000,000, seed 3
    chunglu40k  : Chung-Lu gamma=2.3, n=40,000, E=160,000, seed 3 (profiling size)
    mesh1000    : 1000x1000 triangulated mesh, seed 3
    ba1m        : Barabasi-Albert n=333,334, m=3 (999,996 edges), seed 12, U[0, sqrt n]^2
    """
    if name == "grid32":
        g = grid(32, 32)
        return g, uniform_positions(g.n, 1)
    if name == "ba100k":
        g = barabasi_albert(100_000, 3, 2)
        return g, uniform_positions(g.n, 2)
    if name == "chunglu250k":
        g = chung_lu(250_000, 2.3, 8.0, 1_000_000, 3)
        return g, uniform_positions(g.n, 3)
    if name == "chunglu40k":
        g = chung_lu(40_000, 2.3, 8.0, 160_000, 3)
        return g, uniform_positions(g.n, 3)
    if name == "mesh1000":
        g = tri_mesh(1000, 1000)
        return g, uniform_positions(g.n, 3)
    if name == "ba1m":
        g = barabasi_albert(333_334, 3, 12)
        return g, uniform_positions(g.n, 12)
    raise KeyError(name)
