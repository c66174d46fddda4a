"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module draws graphs, views and initial layouts. It holds none of the
PPRviz arithmetic (no PageRank, no DPPR, no PDist, no stress): both sides
receive the same arrays from here and nothing else is shared between them.

Randomness is a counter-based SplitMix64 (Steele, Lea, Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): output number i of
stream (seed, tag) is mix64(base + (i + 1) * GOLDEN) with base derived from
(seed, tag). Everything is vectorised with numpy uint64 arithmetic, so a draw
depends only on its counter and never on how the work is blocked.

Workload shapes follow the paper's setting (Sec. 6, dataset table): the paper
benchmarks on real scale-free graphs; Chung-Lu power-law graphs with degree
exponent in [2, 3] (the range its complexity analysis assumes, Appendix,
Tau-Push expected cost) stand in for them, and stochastic-block-model views
stand in for the clusters of its supergraph hierarchy (Sec. 5).
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

__all__ = [
    "mix64", "uniform", "chung_lu_weights", "chung_lu", "sbm", "dense_clustered",
    "uniform_x0", "sample_view", "sbm_views", "Graph", "directed_from", "random_leaf_sets",
]


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _base(seed: int, tag: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GOLDEN + np.uint64(tag & 0xFFFFFFFFFFFFFFFF)
        return mix64(np.array([s], dtype=np.uint64))[0]


def uniform(seed: int, tag: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) for the given uint64 counters of stream (seed, tag)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = mix64(_base(seed, tag) + (c + np.uint64(1)) * GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


class Graph:
    """Graph in CSR form, columns sorted: undirected (both directions stored)
    unless `directed`, then each row lists the node's out-neighbours.

    row_ptr: int64[n + 1]; col: int32[nnz]; weight: float32[nnz] or None.
    """

    def __init__(self, n, row_ptr, col, weight=None, directed=False):
        self.n = int(n)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.weight = None if weight is None else np.ascontiguousarray(weight, dtype=np.float32)
        self.directed = bool(directed)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def __repr__(self):
        return f"Graph(n={self.n}, nnz={self.nnz}, weighted={self.weight is not None})"


def _csr_from_pairs(n: int, u: np.ndarray, v: np.ndarray, w: np.ndarray | None = None) -> Graph:
    """Symmetric CSR from undirected pairs u < v (each pair listed once)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    order = np.lexsort((dst, src))
    src = src[order]
    dst = dst[order]
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    wt = None
    if w is not None:
        w = np.asarray(w, dtype=np.float32)
        wt = np.concatenate([w, w])[order]
    return Graph(n, row_ptr, dst.astype(np.int32), wt)


def chung_lu_weights(n: int, mean_degree: float, exponent: float) -> np.ndarray:
    """Expected degrees w_i = C (i + 1)^(-1/(exponent - 1)), descending in i.

    Scaled so that the mean is `mean_degree`, with every weight capped at
    sqrt(sum w) so that w_i w_j / sum(w) <= 1; scale and cap alternate until
    they agree (a few rounds).
    """
    i = np.arange(n, dtype=np.float64)
    w = (i + 1.0) ** (-1.0 / (exponent - 1.0))
    for _ in range(50):
        w = w * (mean_degree * n / w.sum())
        cap = np.sqrt(w.sum())
        if w.max() <= cap * (1 + 1e-12):
            break
        w = np.minimum(w, cap)
    return w


def chung_lu(n: int, mean_degree: float, exponent: float = 2.5, seed: int = 0) -> Graph:
    """Undirected Chung-Lu graph: edge {i, j}, i < j, present with probability
    min(1, w_i w_j / sum(w)), no self-loops, unit weights.

    Node ids are in descending expected degree. Exact pairwise sampling for
    n <= 20,000 (one uniform per pair, counter i*n + j); for larger n the
    geometric skip sampler of Miller and Hagberg ("Efficient generation of
    networks with given expected degrees", WAW 2011), vectorised over all
    source nodes at once.
    """
    w = chung_lu_weights(n, mean_degree, exponent)
    S = w.sum()
    if n <= 20000:
        us, vs = [], []
        block = max(1, 4_000_000 // max(n, 1))
        for i0 in range(0, n, block):
            i1 = min(n, i0 + block)
            ii = np.arange(i0, i1, dtype=np.int64)[:, None]
            jj = np.arange(n, dtype=np.int64)[None, :]
            mask_upper = jj > ii
            p = np.minimum(1.0, w[i0:i1, None] * w[None, :] / S)
            r = uniform(seed, 1, (ii * n + jj).astype(np.uint64))
            hit = mask_upper & (r < p)
            a, b = np.nonzero(hit)
            us.append(a + i0)
            vs.append(b)
        return _csr_from_pairs(n, np.concatenate(us), np.concatenate(vs))
    return _chung_lu_skip(n, w, S, seed)


def _chung_lu_skip(n: int, w: np.ndarray, S: float, seed: int) -> Graph:
    us, vs = [], []
    u = np.arange(n - 1, dtype=np.int64)
    v = u + 1
    p = np.minimum(1.0, w[u] * w[v] / S)
    draw = np.zeros_like(u)
    active = p > 0
    u, v, p, draw = u[active], v[active], p[active], draw[active]
    while u.size:
        # geometric skip with success probability p
        r = uniform(seed, 2, (u.astype(np.uint64) << np.uint64(22)) + draw.astype(np.uint64))
        draw = draw + 1
        with np.errstate(divide="ignore"):
            skip = np.where(p >= 1.0, 0.0, np.floor(np.log1p(-r) / np.log1p(-np.minimum(p, 1 - 1e-16))))
        v = v + np.minimum(skip, n).astype(np.int64)
        inb = v < n
        u, v, p, draw = u[inb], v[inb], p[inb], draw[inb]
        if not u.size:
            break
        q = np.minimum(1.0, w[u] * w[v] / S)
        r2 = uniform(seed, 3, (u.astype(np.uint64) << np.uint64(22)) + draw.astype(np.uint64))
        draw = draw + 1
        acc = r2 < q / p
        us.append(u[acc])
        vs.append(v[acc])
        p = q
        v = v + 1
        keep = (v < n) & (p > 0)
        u, v, p, draw = u[keep], v[keep], p[keep], draw[keep]
    return _csr_from_pairs(n, np.concatenate(us) if us else np.zeros(0, np.int64),
                           np.concatenate(vs) if vs else np.zeros(0, np.int64))


def sbm(sizes, p_in: float, p_out: float, seed: int = 0, tag: int = 4) -> Graph:
    """Undirected stochastic block model with the given block sizes; isolated
    nodes are kept. Pair {i, j}, i < j, uses counter i*n + j of stream tag."""
    sizes = np.asarray(sizes, dtype=np.int64)
    n = int(sizes.sum())
    block_of = np.repeat(np.arange(len(sizes)), sizes)
    us, vs = [], []
    block = max(1, 4_000_000 // max(n, 1))
    for i0 in range(0, n, block):
        i1 = min(n, i0 + block)
        ii = np.arange(i0, i1, dtype=np.int64)[:, None]
        jj = np.arange(n, dtype=np.int64)[None, :]
        same = block_of[i0:i1, None] == block_of[None, :]
        p = np.where(same, p_in, p_out)
        r = uniform(seed, tag, (ii * n + jj).astype(np.uint64))
        hit = (jj > ii) & (r < p)
        a, b = np.nonzero(hit)
        us.append(a + i0)
        vs.append(b)
    return _csr_from_pairs(n, np.concatenate(us), np.concatenate(vs))


def dense_clustered(n: int, blocks: int = 20, density: float = 0.15, seed: int = 0,
                    in_out_ratio: float = 8.0) -> Graph:
    """Dense weighted clustered view: an SBM with `blocks` equal blocks whose
    in/out edge probabilities (ratio `in_out_ratio`) give the requested
    overall density, and symmetric lognormal(0, 1) edge weights (Box-Muller on
    two uniforms per pair)."""
    sizes = np.full(blocks, n // blocks, dtype=np.int64)
    sizes[: n - sizes.sum()] += 1
    f_in = float((sizes * (sizes - 1)).sum()) / (n * (n - 1))
    p_out = density / (f_in * in_out_ratio + (1 - f_in))
    p_in = min(1.0, in_out_ratio * p_out)
    g = sbm(sizes, p_in, p_out, seed=seed, tag=5)
    # weights: one lognormal per undirected pair, keyed by (min, max) counter
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.row_ptr))
    dst = g.col.astype(np.int64)
    lo = np.minimum(src, dst)
    hi = np.maximum(src, dst)
    key = (lo * n + hi).astype(np.uint64)
    u1 = uniform(seed, 6, key)
    u2 = uniform(seed, 7, key)
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    g.weight = np.exp(z).astype(np.float32)
    return g


def uniform_x0(k: int, seed: int = 0, tag: int = 8) -> np.ndarray:
    """Initial layout: k x 2 float32 uniform on [-1, 1]^2, row-major."""
    r = uniform(seed, tag, np.arange(2 * k, dtype=np.uint64))
    return (2.0 * r - 1.0).astype(np.float32).reshape(k, 2)


def sample_view(n: int, k: int, seed: int = 0, tag: int = 9) -> np.ndarray:
    """k distinct node ids drawn uniformly without replacement (sorted by
    their random keys, so the order is random but reproducible)."""
    if k > n:
        raise ValueError("view larger than graph")
    keys = mix64(_base(seed, tag) + (np.arange(n, dtype=np.uint64) + np.uint64(1)) * GOLDEN)
    return np.argsort(keys, kind="stable")[:k].astype(np.int32)


def sbm_views(count: int, seed: int = 0, n_min: int = 50, n_max: int = 5000,
              b_min: int = 4, b_max: int = 16, p_in: float = 0.1, p_out: float = 0.002):
    """`count` independent SBM views with n_v ~ U{n_min..n_max} and
    b_v ~ U{b_min..b_max} near-equal blocks (the batched-views workload)."""
    r = uniform(seed, 10, np.arange(2 * count, dtype=np.uint64)).reshape(count, 2)
    out = []
    for v in range(count):
        nv = n_min + int(r[v, 0] * (n_max - n_min + 1))
        bv = b_min + int(r[v, 1] * (b_max - b_min + 1))
        sizes = np.full(bv, nv // bv, dtype=np.int64)
        sizes[: nv - sizes.sum()] += 1
        out.append(sbm(sizes, p_in, p_out, seed=seed * 1000003 + v, tag=11))
    return out


def directed_from(g: Graph, p_both: float = 0.3, dangling: float = 0.02, seed: int = 0, tag: int = 11) -> Graph:
    """A directed graph drawn from an undirected one: each edge {u, v} keeps
    both directions with probability p_both, else one direction chosen
    uniformly; then a `dangling` fraction of the nodes lose all out-edges
    (dangling nodes). Weights, if any, follow their edges."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    dst = g.col.astype(np.int64)
    up = src < dst
    u, v = src[up], dst[up]
    w = None if g.weight is None else g.weight[up]
    idx = np.arange(len(u), dtype=np.uint64)
    r1 = uniform(seed, tag, idx)
    r2 = uniform(seed, tag + 1, idx)
    both = r1 < p_both
    fwd = both | (r2 < 0.5)
    bwd = both | (r2 >= 0.5)
    s2 = np.concatenate([u[fwd], v[bwd]])
    d2 = np.concatenate([v[fwd], u[bwd]])
    w2 = None if w is None else np.concatenate([w[fwd], w[bwd]])
    drop = uniform(seed, tag + 2, np.arange(g.n, dtype=np.uint64)) < dangling
    keep = ~drop[s2]
    s2, d2 = s2[keep], d2[keep]
    if w2 is not None:
        w2 = w2[keep]
    order = np.lexsort((d2, s2))
    s2, d2 = s2[order], d2[order]
    row_ptr = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(np.bincount(s2, minlength=g.n), out=row_ptr[1:])
    return Graph(g.n, row_ptr, d2.astype(np.int32), None if w2 is None else w2[order], directed=True)


def random_leaf_sets(n: int, sizes, seed: int = 0, tag: int = 12):
    """Disjoint leaf sets of the given sizes drawn uniformly from 0..n-1 (the
    children of a randomly chosen supernode, the case the paper's expected
    Tau-Push cost is stated for). Returns (leaf_ptr int64, leaf_idx int32)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    total = int(sizes.sum())
    ids = sample_view(n, total, seed=seed, tag=tag)
    leaf_ptr = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=leaf_ptr[1:])
    return leaf_ptr, np.ascontiguousarray(ids.astype(np.int32))
