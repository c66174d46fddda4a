"""Plain FP64 CPU oracle for the PPRviz hot path. TEST INFRASTRUCTURE ONLY.

Who may use this module: the tests, the smoke check in __graft_entry__ and the
CPU-baseline leg of bench.py. Nothing in the product (the C-ABI library under
paper_2112_14944_gb300/ and its Python binding) imports or runs it, and it
shares no code with the CUDA path; the only common inputs are the arrays drawn
by the seeded generators in `synth`.

Every function states the passage of the paper (Zhang et al., "Effective and
Efficient PageRank-based Positioning for Graph Visualization", SIGMOD 2023,
arXiv 2112.14944) that it follows. Everything is FP64, written for a reader to
check against the paper by eye: no blocking, no fusion, no reordering. Library
primitives used as single steps: scipy sparse matrix products, numpy dense
LU/Cholesky solves.

Readings where the paper is silent (each also listed in the design notes):
  * dangling nodes (out-degree 0): the walk stays where it is (a self-loop in
    the transition matrix) and d(v) = 0, so the node's DPPR row is zero;
  * weighted graphs: P[i, j] = w_ij / s_i and d(i) := s_i = sum_j w_ij;
  * m = sum_v d(v) (both directions of an undirected edge are counted);
  * PDist with z = 0 is 2 ln n_clamp, the diagonal of PDist is 0 and unused;
  * "(L^w)^-1" in Eq. (10) is the Moore-Penrose solution: the pinned solve
    followed by centring;
  * Tau-Push (Sec. 4): the readings are listed above gfp() below.

Parity status: every function here is pinned by a test in
tests/test_oracle_pins.py (closed forms, a direct linear solve, invariants,
the paper's forward- and backward-push examples, the error bounds of
Lemmas 2 and 3 and Theorem 3 against a direct solve, finite differences).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
import scipy.sparse as sp

__all__ = [
    "degrees", "transition_matrix", "ppr_direct", "ppr_rows", "ppr_cols", "dppr_rows",
    "pdist_from_z", "pdist_from_dppr", "stress", "stress_grad", "stress_grad_pdist",
    "lw_matrix", "ly_matrix", "smacof_step", "smacof", "forward_push",
    "residual_certificate", "power_sweeps_needed", "level_dppr", "node_distribution", "ulcv",
    "backward_push", "dpr", "dpr_power", "gfp", "gbp", "tau_push", "level_dppr_rows_power",
]


# ----------------------------------------------------------------------------
# Sec. 2.1 / Table 1: the graph, out-degrees d(v), and the random walk.
# ----------------------------------------------------------------------------
def degrees(n, row_ptr, col, weight=None):
    """Out-degree d(v) (Table 1); strength sum_j w_vj for weighted graphs."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    if weight is None:
        return np.diff(row_ptr).astype(np.float64)
    w = np.asarray(weight, dtype=np.float64)
    d = np.zeros(n, dtype=np.float64)
    for v in range(n):
        d[v] = w[row_ptr[v]:row_ptr[v + 1]].sum()
    return d


def transition_matrix(n, row_ptr, col, weight=None):
    """Row-stochastic walk matrix P of Sec. 3.1: from v_i step to an
    out-neighbour v_j with probability w_ij / d(v_i) (1 / d(v_i) unweighted).
    A node without out-edges keeps the walk (P[i, i] = 1)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    vals = np.ones(len(col)) if weight is None else np.asarray(weight, dtype=np.float64)
    A = sp.csr_matrix((vals, col, row_ptr), shape=(n, n))
    d = np.asarray(A.sum(axis=1)).ravel()
    dangling = d == 0
    inv = np.where(dangling, 0.0, 1.0 / np.where(dangling, 1.0, d))
    P = sp.diags(inv) @ A
    if dangling.any():
        idx = np.nonzero(dangling)[0]
        P = P + sp.csr_matrix((np.ones(len(idx)), (idx, idx)), shape=(n, n))
    return sp.csr_matrix(P)


# ----------------------------------------------------------------------------
# Sec. 3.1: PPR pi(v_i, v_j) of a random walk with restart probability alpha.
# Summing over walk lengths, the ending distribution from v_i is
#   pi(v_i, .) = alpha * sum_t (1 - alpha)^t e_i P^t,
# i.e. Pi = alpha (I - (1 - alpha) P)^-1 as a matrix.
# ----------------------------------------------------------------------------
def ppr_direct(P, alpha):
    """Pi = alpha (I - (1 - alpha) P)^-1 by a dense LU solve (tiny graphs)."""
    Pd = P.toarray() if sp.issparse(P) else np.asarray(P, dtype=np.float64)
    n = Pd.shape[0]
    return alpha * np.linalg.solve((np.eye(n) - (1 - alpha) * Pd).T, np.eye(n)).T


def power_sweeps_needed(alpha, tol):
    """Smallest T with (1 - alpha)^(T + 1) <= tol: after T sweeps of the power
    iteration the walk mass not yet ended is (1 - alpha)^(T + 1)."""
    c = 1.0 - alpha
    return max(0, math.ceil(math.log(tol) / math.log(c)) - 1)


def ppr_rows(P, sources, alpha, tol=1e-15):
    """PPR rows pi(s, .) for each s in `sources` by power iteration (the
    paper's near-exact baseline of Sec. 3.3, run far below its 1e-9):
        x_0 = alpha e_s,   x_{t+1} = alpha e_s + (1 - alpha) x_t P,
    stopped once the unended walk mass (1 - alpha)^(t+1) is at most `tol`.
    Returns a dense (len(sources), n) array."""
    n = P.shape[0]
    c = 1.0 - alpha
    sources = np.asarray(sources, dtype=np.int64)
    B = np.zeros((len(sources), n))
    B[np.arange(len(sources)), sources] = alpha
    PT = sp.csr_matrix(P.T)
    X = B.copy()
    for _ in range(power_sweeps_needed(alpha, tol)):
        X = B + c * (PT @ X.T).T
    return X


def ppr_cols(P, targets, alpha, tol=1e-15):
    """PPR columns pi(., t): y_0 = alpha e_t, y_{k+1} = alpha e_t + (1 - alpha) P y_k.
    Returns a dense (n, len(targets)) array."""
    n = P.shape[0]
    c = 1.0 - alpha
    targets = np.asarray(targets, dtype=np.int64)
    B = np.zeros((n, len(targets)))
    B[targets, np.arange(len(targets))] = alpha
    Y = B.copy()
    for _ in range(power_sweeps_needed(alpha, tol)):
        Y = B + c * (P @ Y)
    return Y


def dppr_rows(pi_rows, d, sources):
    """Definition 1: pi_d(v_i, v_j) = pi(v_i, v_j) * d(v_i)."""
    return pi_rows * np.asarray(d, dtype=np.float64)[np.asarray(sources)][:, None]


def residual_certificate(P, x_rows, sources, d, alpha):
    """Error bound of an approximate PPR row x (Eq. (3), the push invariant):
    with res = alpha e_s - x (I - (1 - alpha) P), the exact row is
    x + res Pi / alpha, and since 0 <= Pi <= 1 entrywise,
        max_t |pi_d(s, t) - d(s) x_t| <= d(s) * ||res||_1 / alpha."""
    n = P.shape[0]
    c = 1.0 - alpha
    sources = np.asarray(sources, dtype=np.int64)
    B = np.zeros((len(sources), n))
    B[np.arange(len(sources)), sources] = alpha
    res = B - x_rows + c * (sp.csr_matrix(P.T) @ x_rows.T).T
    return np.asarray(d, dtype=np.float64)[sources] * np.abs(res).sum(axis=1) / alpha


# ----------------------------------------------------------------------------
# Sec. 3.1, Eq. (1): PDist.
#   Delta[i, j] = min(max(1 - ln(pi_d(v_i, v_j) + pi_d(v_j, v_i)), 2), 2 ln n)
# ----------------------------------------------------------------------------
def pdist_from_z(z, n_clamp):
    """Eq. (1) applied to z_ij = pi_d(i, j) + pi_d(j, i) (natural log, Sec. 3.1).
    z = 0 gives the upper clamp 2 ln n_clamp (ln 0 = -inf, never NaN)."""
    z = np.asarray(z, dtype=np.float64)
    upper = 2.0 * math.log(n_clamp) if n_clamp > 0 else float("nan")
    with np.errstate(divide="ignore"):
        raw = 1.0 - np.log(z)
    raw = np.where(z > 0, raw, np.inf)
    return np.minimum(np.maximum(raw, 2.0), upper)


def pdist_from_dppr(D, n_clamp):
    """Full k x k PDist from a k x k DPPR matrix (rows = sources); the
    diagonal is set to 0 (the paper defines no self distance)."""
    D = np.asarray(D, dtype=np.float64)
    Delta = pdist_from_z(D + D.T, n_clamp)
    np.fill_diagonal(Delta, 0.0)
    return Delta


# ----------------------------------------------------------------------------
# Sec. 5, Eq. (7): the stress energy L(X | Delta) = sum_{i<j} (1 - |X_i - X_j| / Delta_ij)^2
# ----------------------------------------------------------------------------
def _pair_dist(X):
    X = np.asarray(X, dtype=np.float64)
    diff = X[:, None, :] - X[None, :, :]
    return diff, np.sqrt((diff ** 2).sum(axis=-1))


def stress(X, Delta):
    """Eq. (7) summed over the upper triangle i < j."""
    _, dist = _pair_dist(X)
    Delta = np.asarray(Delta, dtype=np.float64)
    iu = np.triu_indices(len(Delta), 1)
    return float(((1.0 - dist[iu] / Delta[iu]) ** 2).sum())


def stress_grad(X, Delta):
    """dL/dX_i = sum_{j != i} 2 (d_ij - Delta_ij) / (Delta_ij^2 d_ij) (X_i - X_j),
    the derivative of Eq. (7); a pair at zero distance contributes 0 (the
    subgradient the paper's L^Y convention also takes, Appendix A.1)."""
    diff, dist = _pair_dist(X)
    Delta = np.asarray(Delta, dtype=np.float64)
    k = len(Delta)
    coef = np.zeros((k, k))
    off = ~np.eye(k, dtype=bool)
    ok = off & (dist > 0)
    coef[ok] = 2.0 * (dist[ok] - Delta[ok]) / (Delta[ok] ** 2 * dist[ok])
    return (coef[:, :, None] * diff).sum(axis=1)


def stress_grad_pdist(X, Delta):
    """Derivative of Eq. (7) with respect to each entry of a k x k PDist
    matrix when the energy is read as (1/2) sum_{i != j}, which equals Eq. (7)
    for symmetric Delta: dL/dDelta_ij = (1 - d_ij / Delta_ij) d_ij / Delta_ij^2
    for i != j, and 0 on the diagonal."""
    _, dist = _pair_dist(X)
    Delta = np.asarray(Delta, dtype=np.float64)
    k = len(Delta)
    g = np.zeros((k, k))
    off = ~np.eye(k, dtype=bool)
    g[off] = (1.0 - dist[off] / Delta[off]) * dist[off] / Delta[off] ** 2
    return g


# ----------------------------------------------------------------------------
# Appendix A.1, stress majorization: L^w, L^Y and Eq. (10) X = (L^w)^-1 L^Y Y.
# ----------------------------------------------------------------------------
def lw_matrix(Delta):
    """L^w[i, j] = -1 / Delta_ij^2 (i != j), L^w[i, i] = sum_{k != i} 1 / Delta_ik^2."""
    Delta = np.asarray(Delta, dtype=np.float64)
    k = len(Delta)
    L = np.zeros((k, k))
    off = ~np.eye(k, dtype=bool)
    L[off] = -1.0 / Delta[off] ** 2
    np.fill_diagonal(L, -L.sum(axis=1))
    return L


def ly_matrix(Y, Delta):
    """L^Y[i, j] = -1 / (Delta_ij |Y_i - Y_j|) if i != j and Y_i != Y_j, else 0;
    L^Y[i, i] = -sum_{k != i} L^Y[i, k]."""
    _, dist = _pair_dist(Y)
    Delta = np.asarray(Delta, dtype=np.float64)
    k = len(Delta)
    L = np.zeros((k, k))
    ok = (~np.eye(k, dtype=bool)) & (dist > 0)
    L[ok] = -1.0 / (Delta[ok] * dist[ok])
    np.fill_diagonal(L, -L.sum(axis=1))
    return L


def smacof_step(Y, Delta):
    """One stress-majorization update, Eq. (10): solve L^w X = L^Y(Y) Y.
    L^w is a Laplacian (singular), so the solve pins node 0 at the origin
    (a dense Cholesky solve of L^w without row/column 0) and then centres X,
    which is the minimum-norm (Moore-Penrose) solution."""
    Lw = lw_matrix(Delta)
    b = ly_matrix(Y, Delta) @ np.asarray(Y, dtype=np.float64)
    k = len(Lw)
    X = np.zeros((k, b.shape[1]))
    if k > 1:
        cf = scipy.linalg.cho_factor(Lw[1:, 1:], lower=True)
        X[1:] = scipy.linalg.cho_solve(cf, b[1:])
    return X - X.mean(axis=0)


def smacof(X0, Delta, iters):
    """`iters` updates of Eq. (10) from X0; returns (X, stress after each update)."""
    X = np.asarray(X0, dtype=np.float64).copy()
    hist = []
    for _ in range(iters):
        X = smacof_step(X, Delta)
        hist.append(stress(X, Delta))
    return X, np.array(hist)


# ----------------------------------------------------------------------------
# Sec. 3.3: Forward-Push with reserve and residue, in a caller-given order
# (used to check the running example and the invariant Eq. (3)).
# ----------------------------------------------------------------------------
def forward_push(n, row_ptr, col, d, source, alpha, order):
    """Initial residue r(s, s) = d(s) (DPPR scaling, Sec. 3.3). Each push at
    v_k moves alpha * r(v_k) to the estimate and spreads (1 - alpha) r(v_k)
    evenly over the out-neighbours, then zeroes r(v_k). `order` lists the
    nodes to push, in turn. Returns (estimate, residue)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    est = np.zeros(n)
    r = np.zeros(n)
    r[source] = d[source]
    for v in order:
        rv = r[v]
        est[v] += alpha * rv
        nb = col[row_ptr[v]:row_ptr[v + 1]]
        for u in nb:
            r[u] += (1 - alpha) * rv / len(nb)
        r[v] = 0.0
    return est, r


# ----------------------------------------------------------------------------
# Sec. 3.2, Eq. (2): level-l DPPR between supernodes (leaf-set averages).
# ----------------------------------------------------------------------------
def level_dppr(dppr_full, leaf_sets):
    """pi_d(V_i, V_j) = sum_{s in F(V_i), t in F(V_j)} pi_d(s, t) / (|F(V_i)| |F(V_j)|)."""
    k = len(leaf_sets)
    out = np.zeros((k, k))
    for i, Fi in enumerate(leaf_sets):
        for j, Fj in enumerate(leaf_sets):
            out[i, j] = dppr_full[np.ix_(Fi, Fj)].sum() / (len(Fi) * len(Fj))
    return out


def level_dppr_rows_power(P, d, leaf_sets, sources, alpha, tol=1e-15):
    """Rows `sources` of Eq. (2) without the dense matrix. By linearity
    sum_{s in F(V_i)} d(s) pi(s, .) / |F(V_i)| is the power iteration from the
    group start b = d(s) / |F(V_i)| on F(V_i) (the initial residues of
    Algorithm 2): y_0 = alpha b, y_{t+1} = alpha b + (1 - alpha) y_t P, stopped
    once the unended walk mass is at most `tol` times the start's; entry j of
    row i is the mean of y over F(V_j). Returns (len(sources), k)."""
    n = P.shape[0]
    d = np.asarray(d, dtype=np.float64)
    PT = sp.csr_matrix(P.T)
    Bm = np.zeros((n, len(sources)))
    for c, i in enumerate(sources):
        Fi = np.asarray(leaf_sets[i], dtype=np.int64)
        Bm[Fi, c] = d[Fi] / len(Fi)
    Y = alpha * Bm
    for _ in range(power_sweeps_needed(alpha, tol)):
        Y = alpha * Bm + (1 - alpha) * (PT @ Y)
    out = np.zeros((len(sources), len(leaf_sets)))
    for j, Fj in enumerate(leaf_sets):
        out[:, j] = Y[np.asarray(Fj, dtype=np.int64), :].mean(axis=0)
    return out


# ----------------------------------------------------------------------------
# Sec. 2 (visualization quality): node distribution and uniform length
# coefficient variance of a layout.
# ----------------------------------------------------------------------------
def node_distribution(X):
    """ND(X) = sum_{i<j} 1 / |X_i - X_j|^2 (the node-distribution definition of
    Sec. 2); a coincident pair makes it infinite."""
    _, dist = _pair_dist(X)
    iu = np.triu_indices(len(dist), 1)
    d2 = dist[iu] ** 2
    if np.any(d2 == 0):
        return float("inf")
    return float((1.0 / d2).sum())


def ulcv(X, edges):
    """ULCV(X) = l_sigma / l_mu over the edge lengths (Sec. 2), with the
    population standard deviation; `edges` lists each undirected edge (u, v)
    once, u, v indexing the rows of X."""
    X = np.asarray(X, dtype=np.float64)
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    lengths = np.sqrt(((X[e[:, 0]] - X[e[:, 1]]) ** 2).sum(axis=1))
    mu = lengths.mean()
    sigma = np.sqrt(((lengths - mu) ** 2).mean())
    return float(sigma / mu)


# ----------------------------------------------------------------------------
# Sec. 4.1: backward push (the conventional single-target form, PPR units), in
# a caller-given order (used to check the paper's backward-push example).
# ----------------------------------------------------------------------------
def backward_push(P, target, alpha, order):
    """Initial residue r(t) = 1 at the target t. A push at v_k moves
    alpha * r(v_k) to the estimate of v_k and gives every in-neighbour v_i of
    v_k the amount (1 - alpha) * r(v_k) * P[i, k] (= (1 - alpha) r(v_k) / d(v_i)
    unweighted), then zeroes r(v_k). The residue is read and zeroed before it
    is spread. Returns (estimate, residue) with pi(s, t) = estimate_s +
    sum_k pi(s, k) r_k (the backward invariant)."""
    n = P.shape[0]
    PT = sp.csr_matrix(P.T)  # row k lists the in-neighbours i of k with P[i, k]
    est = np.zeros(n)
    r = np.zeros(n)
    r[target] = 1.0
    for v in order:
        rv = r[v]
        est[v] += alpha * rv
        r[v] = 0.0
        for q in range(PT.indptr[v], PT.indptr[v + 1]):
            r[PT.indices[q]] += (1 - alpha) * rv * PT.data[q]
    return est, r


# ----------------------------------------------------------------------------
# Sec. 4, Eq. (dnpr-dnppr): degree-normalised PageRank (DPR) of single nodes,
#   tau_t = (1 / m) sum_k pi_d(v_k, v_t);
# a supernode's tau_j is the mean of tau_t over its leaves.
# ----------------------------------------------------------------------------
def dpr(P, d, alpha):
    """tau_t from the dense PPR matrix (the definition; tiny graphs)."""
    d = np.asarray(d, dtype=np.float64)
    Pi = ppr_direct(P, alpha)
    return (d[:, None] * Pi).sum(axis=0) / d.sum()


def dpr_power(P, d, alpha, tol=1e-15):
    """The index precompute of Sec. 4.3: a global PageRank whose start vector
    has entry d(v_k) / m at v_k, by power iteration,
        x_0 = alpha s,   x_{t+1} = alpha s + (1 - alpha) x_t P,   s = d / m,
    stopped once the unended walk mass (1 - alpha)^(t+1) is at most `tol`.
    Summing sum_k d(v_k) pi(v_k, .) / m this is the same vector as dpr()."""
    d = np.asarray(d, dtype=np.float64)
    s = d / d.sum()
    PT = sp.csr_matrix(P.T)
    x = alpha * s
    for _ in range(power_sweeps_needed(alpha, tol)):
        x = alpha * s + (1 - alpha) * (PT @ x)
    return x


# ----------------------------------------------------------------------------
# Sec. 4.2: Group Forward-Push (Algorithm 2) and Group Backward-Push
# (Algorithm 3); Sec. 4.1: Tau-Push (Algorithm 1).
#
# Readings (the paper is silent on these):
#   * "while some residue is above its threshold" takes the nodes first in,
#     first out: a node joins the queue when its residue rises above the
#     threshold and is pushed when it reaches the front;
#   * a push reads and zeroes the residue before spreading it;
#   * a node without out-edges keeps the walk (P[v, v] = 1, the dangling
#     reading above); a push there takes the sum of its endless repeats:
#     forward, the whole residue goes to the estimate; backward, the estimate
#     gains d(v) r = 0 and each other in-neighbour x of v receives
#     (1 - alpha) r P[x, v] / alpha;
#   * Eq. (brmax)'s maximum over the other supernodes: with no other supernode
#     (a single child) the target's own mean degree is used, and a maximum of 0
#     (no source can reach anything) means no backward push at all.
# ----------------------------------------------------------------------------
def _owners(n, leaf_sets):
    owner = np.full(n, -1, dtype=np.int64)
    for j, F in enumerate(leaf_sets):
        owner[np.asarray(F, dtype=np.int64)] = j
    return owner


def gfp(P, d, leaf_sets, i, alpha, r_max):
    """Algorithm 2 from source supernode V_i: initial residue d(v) / |F(V_i)|
    on each leaf of V_i; while some v_k has r(v_k) > d(v_k) r_max, add
    alpha r(v_k) / |F(V_j)| to the estimate of the supernode V_j holding v_k
    (if any) and give each out-neighbour v_j the share (1 - alpha) r(v_k) P[k, j].
    Returns the estimates of every supernode (length len(leaf_sets))."""
    n = P.shape[0]
    d = np.asarray(d, dtype=np.float64)
    owner = _owners(n, leaf_sets)
    size = np.array([len(F) for F in leaf_sets], dtype=np.float64)
    Pc = sp.csr_matrix(P)
    est = np.zeros(len(leaf_sets))
    r = np.zeros(n)
    Fi = np.asarray(leaf_sets[i], dtype=np.int64)
    r[Fi] = d[Fi] / len(Fi)
    queue = [int(v) for v in Fi if r[v] > d[v] * r_max]
    head = 0
    while head < len(queue):
        v = queue[head]
        head += 1
        rv = r[v]
        r[v] = 0.0
        dangling = Pc.indptr[v + 1] - Pc.indptr[v] == 1 and Pc.indices[Pc.indptr[v]] == v and d[v] == 0
        j = owner[v]
        if dangling:
            if j >= 0:
                est[j] += rv / size[j]
            continue
        if j >= 0:
            est[j] += alpha * rv / size[j]
        for q in range(Pc.indptr[v], Pc.indptr[v + 1]):
            u = Pc.indices[q]
            thr = d[u] * r_max
            before = r[u]
            r[u] += (1 - alpha) * rv * Pc.data[q]
            if before <= thr < r[u]:
                queue.append(int(u))
    return est


def gbp(P, d, leaf_sets, j, alpha, rb_max):
    """Algorithm 3 towards target supernode V_j: initial residue 1 / |F(V_j)| on
    each leaf of V_j; while some v_k has r(v_k) > rb_max, add
    alpha d(v_k) r(v_k) / |F(V_i)| to the estimate of the supernode V_i holding
    v_k (if any) and give each in-neighbour v_i the share
    (1 - alpha) r(v_k) P[i, k] (= (1 - alpha) r(v_k) / d(v_i) unweighted).
    Returns the estimates pi_d(V_i, V_j) of every source supernode."""
    n = P.shape[0]
    d = np.asarray(d, dtype=np.float64)
    owner = _owners(n, leaf_sets)
    size = np.array([len(F) for F in leaf_sets], dtype=np.float64)
    Pc = sp.csr_matrix(P)
    PT = sp.csr_matrix(P.T)
    est = np.zeros(len(leaf_sets))
    r = np.zeros(n)
    Fj = np.asarray(leaf_sets[j], dtype=np.int64)
    r[Fj] = 1.0 / len(Fj)
    queue = [int(v) for v in Fj if r[v] > rb_max]
    head = 0
    while head < len(queue):
        v = queue[head]
        head += 1
        rv = r[v]
        r[v] = 0.0
        dangling = Pc.indptr[v + 1] - Pc.indptr[v] == 1 and Pc.indices[Pc.indptr[v]] == v and d[v] == 0
        i = owner[v]
        if i >= 0:
            est[i] += (d[v] * rv if dangling else alpha * d[v] * rv) / size[i]
        share = (1 - alpha) * rv / alpha if dangling else (1 - alpha) * rv
        for q in range(PT.indptr[v], PT.indptr[v + 1]):
            x = PT.indices[q]
            if dangling and x == v:
                continue
            before = r[x]
            r[x] += share * PT.data[q]
            if before <= rb_max < r[x]:
                queue.append(int(x))
    return est


def tau_push(P, d, leaf_sets, alpha, eps, delta, dpr_nodes, tau=None):
    """Algorithm 1: (eps, delta)-approximate level-l DPPR between the children
    V_0 .. V_{k-1} of a supernode (k = len(leaf_sets)).
      1. tau = 1 / sqrt(k n) unless given;
      2. r_max = eps delta / (m tau)  (Eq. (rmax));
      3. row i = gfp from V_i with r_max, for every i;
      4. for every V_j whose DPR tau_j (mean of dpr_nodes over F(V_j)) exceeds
         tau: column j = gbp towards V_j with
         rb_max = eps delta / max_{i != j} mean_{v in F(V_i)} d(v)  (Eq. (brmax)).
    Returns (estimates k x k with row = source, tau, r_max, {refined target j:
    its rb_max})."""
    n = P.shape[0]
    d = np.asarray(d, dtype=np.float64)
    k = len(leaf_sets)
    m = d.sum()
    if tau is None:
        tau = 1.0 / math.sqrt(k * n)
    r_max = eps * delta / (m * tau)
    est = np.zeros((k, k))
    for i in range(k):
        est[i, :] = gfp(P, d, leaf_sets, i, alpha, r_max)
    dpr_nodes = np.asarray(dpr_nodes, dtype=np.float64)
    davg = np.array([d[np.asarray(F)].mean() for F in leaf_sets])
    tau_j = np.array([dpr_nodes[np.asarray(F)].mean() for F in leaf_sets])
    refined = {}
    for j in range(k):
        if tau_j[j] > tau:
            others = [davg[i] for i in range(k) if i != j]
            dmax = max(others) if others else davg[j]
            rb_max = eps * delta / dmax if dmax > 0 else math.inf
            est[:, j] = gbp(P, d, leaf_sets, j, alpha, rb_max)
            refined[j] = rb_max
    return est, tau, r_max, refined
