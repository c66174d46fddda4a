"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, a direct linear solve, invariants proved in the paper, the paper's
worked Forward-Push example, finite differences, and special cases with a
known answer. None of them needs a GPU.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALPHA = 0.15
C = 1.0 - ALPHA


def _graph_P(g):
    return O.transition_matrix(g.n, g.row_ptr, g.col, g.weight)


def _csr_from_edges(n, edges, undirected):
    pairs = list(edges) + ([(b, a) for a, b in edges] if undirected else [])
    pairs = sorted(set(pairs))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    for a, _ in pairs:
        row_ptr[a + 1] += 1
    row_ptr = np.cumsum(row_ptr)
    col = np.array([b for _, b in pairs], dtype=np.int32)
    return row_ptr, col


# --------------------------------------------------------------------------
# PPR (Sec. 3.1) and DPPR (Definition 1)
# --------------------------------------------------------------------------
def test_power_iteration_matches_direct_solve_small_graphs():
    graphs = [
        synth.chung_lu(150, 8, 2.5, seed=3),
        synth.sbm([30, 30, 40], 0.15, 0.01, seed=5),          # has isolated nodes
        synth.dense_clustered(90, blocks=3, density=0.2, seed=2),  # weighted
    ]
    for g in graphs:
        P = _graph_P(g)
        Pi = O.ppr_direct(P, ALPHA)
        rows = O.ppr_rows(P, np.arange(g.n), ALPHA)
        cols = O.ppr_cols(P, np.arange(g.n), ALPHA)
        assert np.abs(rows - Pi).max() < 1e-13
        assert np.abs(cols - Pi).max() < 1e-13


def test_complete_graph_closed_form():
    # K_n: P = (J - I)/(n - 1) has eigenvalue 1 on the ones vector and
    # -1/(n-1) elsewhere, so Pi = J/n + q (I - J/n), q = alpha (n-1)/(n-1+c).
    n = 7
    edges = [(i, j) for i in range(n) for j in range(i + 1, n)]
    rp, col = _csr_from_edges(n, edges, True)
    P = O.transition_matrix(n, rp, col)
    q = ALPHA * (n - 1) / (n - 1 + C)
    Pi = O.ppr_rows(P, np.arange(n), ALPHA)
    assert np.allclose(np.diag(Pi), q * (1 - 1 / n) + 1 / n, atol=1e-14, rtol=0)
    off = ~np.eye(n, dtype=bool)
    assert np.allclose(Pi[off], 1 / n - q / n, atol=1e-14, rtol=0)


def test_star_closed_form_and_pdist():
    # centre 0 with L leaves: pi(leaf, centre) = a, pi(centre, centre) = b with
    # b = alpha + c a and a = c b, so a = c / (1 + c); by symmetry of pi_d the
    # centre-leaf DPPR is c/(1+c) both ways and leaf-leaf is c^2 / (L (1+c)).
    L = 9
    n = L + 1
    rp, col = _csr_from_edges(n, [(0, i) for i in range(1, n)], True)
    P = O.transition_matrix(n, rp, col)
    d = O.degrees(n, rp, col)
    D = O.dppr_rows(O.ppr_rows(P, np.arange(n), ALPHA), d, np.arange(n))
    assert abs(D[0, 3] - C / (1 + C)) < 1e-14
    assert abs(D[3, 0] - C / (1 + C)) < 1e-14
    assert abs(D[2, 5] - C * C / (L * (1 + C))) < 1e-14
    Delta = O.pdist_from_dppr(D, n)
    # leaf-leaf: 1 - ln(2 c^2 / (L (1 + c))) = 3.4443009 at alpha = 0.15, L = 9
    assert abs(Delta[2, 5] - (1 - math.log(2 * C * C / (L * (1 + C))))) < 1e-13
    assert abs(Delta[2, 5] - 3.4443009) < 1e-7
    assert Delta[0, 4] == 2.0                           # clamped at the lower bound
    assert np.all(np.diag(Delta) == 0)


def test_single_edge_closed_form():
    rp, col = _csr_from_edges(2, [(0, 1)], True)
    Pi = O.ppr_rows(O.transition_matrix(2, rp, col), [0, 1], ALPHA)
    assert abs(Pi[0, 0] - 1 / (1 + C)) < 1e-15
    assert abs(Pi[0, 1] - C / (1 + C)) < 1e-15


def _weighted_csr_from_edges(n, wedges):
    """Symmetric weighted CSR from (a, b, w) undirected edges."""
    pairs = sorted({(a, b): w for a, b, w in wedges}.items() | {(b, a): w for a, b, w in wedges}.items())
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    for (a, _), _ in pairs:
        row_ptr[a + 1] += 1
    row_ptr = np.cumsum(row_ptr)
    col = np.array([b for (_, b), _ in pairs], dtype=np.int32)
    w = np.array([x for _, x in pairs], dtype=np.float32)
    return row_ptr, col, w


def test_weighted_star_closed_form():
    # Weighted reading of Sec. 3.1 / Definition 1: a walk at v steps to u with
    # probability w_vu / s_v and d(v) = s_v (the strength). Star: centre 0,
    # leaves j with edge weights w_j, W = sum_j w_j. From the recursion
    # pi(s, t) = alpha [s = t] + c sum_u P(s, u) pi(u, t):
    #   pi(centre, centre) = 1 / (1 + c),  pi(leaf_j, centre) = c / (1 + c),
    #   pi(centre, leaf_j) = c w_j / (W (1 + c)),
    #   pi(leaf_i, leaf_j) = alpha [i = j] + c^2 w_j / (W (1 + c)),
    # so pi_d(centre, leaf_j) = pi_d(leaf_j, centre) = c w_j / (1 + c) and
    # pi_d(leaf_i, leaf_j) = c^2 w_i w_j / (W (1 + c)). With d = edge count
    # or P normalised by the count instead, these values (and the symmetry)
    # do not hold, since the weights below differ.
    wts = [0.5, 1.0, 2.0, 3.5, 7.25]
    L = len(wts)
    n = L + 1
    rp, col, w = _weighted_csr_from_edges(n, [(0, j + 1, wts[j]) for j in range(L)])
    W = float(sum(wts))
    d = O.degrees(n, rp, col, w)
    assert abs(d[0] - W) < 1e-12 and np.allclose(d[1:], wts, atol=1e-12, rtol=0)
    P = O.transition_matrix(n, rp, col, w)
    Pi = O.ppr_rows(P, np.arange(n), ALPHA)
    assert abs(Pi[0, 0] - 1 / (1 + C)) < 1e-14
    for j in range(L):
        assert abs(Pi[j + 1, 0] - C / (1 + C)) < 1e-14
        assert abs(Pi[0, j + 1] - C * wts[j] / (W * (1 + C))) < 1e-14
        for i in range(L):
            exp = (ALPHA if i == j else 0.0) + C * C * wts[j] / (W * (1 + C))
            assert abs(Pi[i + 1, j + 1] - exp) < 1e-14
    D = O.dppr_rows(Pi, d, np.arange(n))
    for j in range(L):
        assert abs(D[0, j + 1] - C * wts[j] / (1 + C)) < 1e-13
        assert abs(D[j + 1, 0] - C * wts[j] / (1 + C)) < 1e-13
    assert abs(D[1, 4] - C * C * wts[0] * wts[3] / (W * (1 + C))) < 1e-14
    # the same star read with d = edge count breaks the symmetry of pi_d
    dc = O.degrees(n, rp, col)
    Dc = O.dppr_rows(Pi, dc, np.arange(n))
    assert np.abs(Dc - Dc.T).max() > 1e-2


def test_weighted_graph_invariants():
    # On a symmetric weighted graph the strength-weighted walk is reversible
    # (s_v P(v, u) = w_vu = s_u P(u, v)), so pi_d is symmetric, every PPR row
    # is a distribution, and sum_{s,t} pi_d(s, t) = sum_s d(s) = sum of all
    # stored weights (Eq. (11) with m = sum_v d(v)).
    g = synth.dense_clustered(120, blocks=4, density=0.2, seed=6)
    assert g.weight is not None and np.ptp(g.weight) > 1.0
    P = _graph_P(g)
    d = O.degrees(g.n, g.row_ptr, g.col, g.weight)
    Pi = O.ppr_direct(P, ALPHA)
    D = O.dppr_rows(Pi, d, np.arange(g.n))
    assert np.abs(Pi.sum(axis=1) - 1).max() < 1e-13
    assert np.abs(D - D.T).max() < 1e-12 * max(1.0, np.abs(D).max())
    m = float(np.asarray(g.weight, dtype=np.float64).sum())
    assert abs(D.sum() - m) < 1e-11 * m
    # P[i, j] = w_ij / s_i row by row
    Pd = P.toarray()
    for v in (0, 7, 63, 119):
        lo, hi = g.row_ptr[v], g.row_ptr[v + 1]
        if hi > lo:
            ww = np.asarray(g.weight[lo:hi], dtype=np.float64)
            assert np.allclose(Pd[v, g.col[lo:hi]], ww / ww.sum(), atol=1e-15, rtol=0)


def test_invariants_on_random_graph():
    g = synth.chung_lu(300, 10, 2.5, seed=1)
    P = _graph_P(g)
    d = O.degrees(g.n, g.row_ptr, g.col)
    Pi = O.ppr_rows(P, np.arange(g.n), ALPHA)
    D = O.dppr_rows(Pi, d, np.arange(g.n))
    assert np.abs(Pi.sum(axis=1) - 1).max() < 1e-13              # each row is a distribution
    assert np.all(np.diag(Pi) >= ALPHA - 1e-15)                    # ends at once w.p. alpha
    assert np.abs(D - D.T).max() < 1e-13                           # reversibility (undirected)
    m = g.nnz
    assert abs(D.sum() - m) < 1e-9 * m                             # Eq. (11): sum z = 2m
    Delta = O.pdist_from_dppr(D, g.n)
    # Theorem 2: every edge has Delta <= 1 - ln(2 alpha (1 - alpha))
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    bound = 1 - math.log(2 * ALPHA * (1 - ALPHA))
    assert Delta[src, g.col].max() <= bound + 1e-12
    # Theorem 1: ND = sum_{i<j} 1/Delta^2 <= 0.215 e m + 0.0175 n^2
    iu = np.triu_indices(g.n, 1)
    assert (1 / Delta[iu] ** 2).sum() <= 0.215 * math.e * m + 0.0175 * g.n ** 2
    assert Delta[iu].min() >= 2.0 and Delta[iu].max() <= 2 * math.log(g.n) + 1e-12


def test_dangling_node_reading():
    # an isolated node keeps its walk: pi(v, v) = 1, d(v) = 0 so its DPPR row
    # is zero, and every PDist entry with it is the upper clamp 2 ln n.
    g = synth.sbm([5, 5, 1], 0.9, 0.0, seed=7)
    iso = 10
    assert g.row_ptr[iso + 1] == g.row_ptr[iso]
    P = _graph_P(g)
    Pi = O.ppr_rows(P, np.arange(g.n), ALPHA)
    assert abs(Pi[iso, iso] - 1) < 1e-15
    d = O.degrees(g.n, g.row_ptr, g.col)
    D = O.dppr_rows(Pi, d, np.arange(g.n))
    assert np.all(D[iso] == 0)
    Delta = O.pdist_from_dppr(D, g.n)
    others = [j for j in range(g.n) if j != iso]
    assert np.all(Delta[iso, others] == 2 * math.log(g.n))


def test_pdist_clamps_and_zero():
    n = 100
    z = np.array([0.0, 1e-300, math.e ** -1, 1.0, 5.0, math.e ** (1 - 2 * math.log(n)) * 1.5])
    out = O.pdist_from_z(z, n)
    assert out[0] == 2 * math.log(n) and out[1] == 2 * math.log(n)
    assert out[2] == 2.0 and out[3] == 2.0 and out[4] == 2.0
    assert abs(out[5] - (2 * math.log(n) - math.log(1.5))) < 1e-12


def test_forward_push_running_example():
    with open(os.path.join(GOLDEN, "forward_push_example.json")) as f:
        ex = json.load(f)
    n = ex["n"]
    rp, col = _csr_from_edges(n, [tuple(e) for e in ex["edges"]], False)
    d = O.degrees(n, rp, col)
    a = ex["alpha"]
    est, r = O.forward_push(n, rp, col, d, ex["source"], a, ex["after_first_push"]["order"])
    for v, val in ex["after_first_push"]["estimate"].items():
        assert abs(est[int(v)] - val) < 1e-12
    for v, val in ex["after_first_push"]["residue"].items():
        assert abs(r[int(v)] - val) < 1e-12
    est, r = O.forward_push(n, rp, col, d, ex["source"], a, ex["after_second_hop"]["order"])
    for v, val in ex["after_second_hop"]["residue"].items():
        assert abs(r[int(v)] - val) < 1e-12
    # Eq. (3): pi_d(s, t) = estimate_t + sum_k r_k pi(k, t)  (r in DPPR units)
    P = O.transition_matrix(n, rp, col)
    Pi = O.ppr_direct(P, a)
    lhs = d[ex["source"]] * Pi[ex["source"]]
    rhs = est + r @ Pi
    assert np.abs(lhs - rhs).max() < 1e-14


def test_residual_certificate_bounds_error_and_matches_closed_form():
    g = synth.chung_lu(200, 8, 2.5, seed=4)
    P = _graph_P(g)
    d = O.degrees(g.n, g.row_ptr, g.col)
    Pi = O.ppr_direct(P, ALPHA)
    src = np.arange(0, g.n, 17)
    for T in (5, 20, 40):
        B = np.zeros((len(src), g.n)); B[np.arange(len(src)), src] = ALPHA
        X = B.copy()
        for _ in range(T):
            X = B + C * (sp.csr_matrix(P.T) @ X.T).T
        cert = O.residual_certificate(P, X, src, d, ALPHA)
        err = (d[src][:, None] * np.abs(X - Pi[src])).max(axis=1)
        assert np.all(err <= cert * (1 + 1e-9))
        # power iteration leaves exactly (1 - alpha)^(T+1) walk mass unended
        assert np.allclose(cert, d[src] * C ** (T + 1), rtol=1e-9, atol=0)
    assert O.power_sweeps_needed(ALPHA, 1e-15) == 212


# --------------------------------------------------------------------------
# Stress (Eq. (7)) and stress majorization (Appendix A.1, Eq. (10))
# --------------------------------------------------------------------------
def _random_delta(k, seed):
    r = synth.uniform(seed, 77, np.arange(k * k, dtype=np.uint64)).reshape(k, k)
    D = 2.0 + 4.0 * (r + r.T) / 2
    np.fill_diagonal(D, 0.0)
    return D


def test_stress_gradient_finite_differences():
    k = 12
    D = _random_delta(k, 1)
    X = synth.uniform_x0(k, seed=2).astype(np.float64) * 3
    g = O.stress_grad(X, D)
    h = 1e-6
    num = np.zeros_like(X)
    for i in range(k):
        for a in range(2):
            Xp = X.copy(); Xp[i, a] += h
            Xm = X.copy(); Xm[i, a] -= h
            num[i, a] = (O.stress(Xp, D) - O.stress(Xm, D)) / (2 * h)
    assert np.abs(num - g).max() < 1e-7 * max(1, np.abs(g).max())
    gD = O.stress_grad_pdist(X, D)
    i, j = 3, 8
    Dp = D.copy(); Dp[i, j] += h; Dp[j, i] += h
    Dm = D.copy(); Dm[i, j] -= h; Dm[j, i] -= h
    fd = (O.stress(X, Dp) - O.stress(X, Dm)) / (2 * h)
    assert abs(fd - (gD[i, j] + gD[j, i])) < 1e-7


def test_stress_invariances_and_zero_for_realisable_delta():
    k = 9
    pts = synth.uniform_x0(k, seed=5).astype(np.float64) * 4
    D = np.sqrt(((pts[:, None] - pts[None]) ** 2).sum(-1))
    assert O.stress(pts, D) < 1e-28
    X = synth.uniform_x0(k, seed=6).astype(np.float64)
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    e0 = O.stress(X, D)
    assert abs(O.stress(X @ R.T + np.array([3.0, -1.0]), D) - e0) < 1e-12 * e0
    # stress majorization drives a realisable Delta to zero stress from a
    # start in the basin of the realising configuration
    Xs, hist = O.smacof(pts + 0.3 * X, D, 400)
    assert hist[-1] < 1e-10


def test_smacof_step_properties():
    k = 25
    D = _random_delta(k, 3)
    X = synth.uniform_x0(k, seed=4).astype(np.float64)
    e_prev = O.stress(X, D)
    for _ in range(30):
        X = O.smacof_step(X, D)
        e = O.stress(X, D)
        assert e <= e_prev * (1 + 1e-12)            # majorization: never increases
        assert np.abs(X.mean(axis=0)).max() < 1e-13  # centred
        e_prev = e
    # the pinned Cholesky solve equals the pseudo-inverse form of Eq. (10)
    Y = X + 0.1 * synth.uniform_x0(k, seed=9)
    ref = np.linalg.pinv(O.lw_matrix(D)) @ (O.ly_matrix(Y, D) @ Y)
    assert np.abs(O.smacof_step(Y, D) - ref).max() < 1e-11
    # the update is the Guttman form X = Y - (L^w)^+ grad / 2 (gradient = 2 (L^w Y - L^Y Y))
    gstep = Y - np.linalg.pinv(O.lw_matrix(D)) @ O.stress_grad(Y, D) / 2
    assert np.abs(O.smacof_step(Y, D) - (gstep - gstep.mean(0))).max() < 1e-10


def test_smacof_two_points_reach_target_in_one_step():
    D = np.array([[0.0, 3.7], [3.7, 0.0]])
    X = np.array([[0.2, -0.4], [0.9, 0.1]])
    Xn = O.smacof_step(X, D)
    assert abs(np.linalg.norm(Xn[0] - Xn[1]) - 3.7) < 1e-14
    assert O.stress(Xn, D) < 1e-28


def test_level_dppr_reduces_to_node_dppr_for_singletons():
    g = synth.chung_lu(60, 6, 2.5, seed=8)
    P = _graph_P(g)
    d = O.degrees(g.n, g.row_ptr, g.col)
    D = O.dppr_rows(O.ppr_direct(P, ALPHA), d, np.arange(g.n))
    sets = [[i] for i in range(g.n)]
    assert np.abs(O.level_dppr(D, sets) - D).max() == 0
    sets = [list(range(0, 20)), list(range(20, 60))]
    lv = O.level_dppr(D, sets)
    assert abs(lv[0, 1] - D[:20, 20:].mean()) < 1e-14


def test_level_dppr_star_closed_form():
    # Definition 2 on the star (centre 0, L leaves) with supernodes A = {0} and
    # B = {1..L}: every pi_d(centre, leaf) = pi_d(leaf, centre) = c / (1 + c),
    # so both cross averages are c / (1 + c); within B, pi_d(s, s) =
    # alpha + c^2 / (L (1 + c)) and pi_d(s, t) = c^2 / (L (1 + c)) (s != t), so
    # pi_d(B, B) = alpha / L + c^2 / (L (1 + c)); pi_d(A, A) = 1 / (1 + c) * L.
    L = 7
    n = L + 1
    rp, col = _csr_from_edges(n, [(0, i) for i in range(1, n)], True)
    P = O.transition_matrix(n, rp, col)
    d = O.degrees(n, rp, col)
    D = O.dppr_rows(O.ppr_direct(P, ALPHA), d, np.arange(n))
    lv = O.level_dppr(D, [[0], list(range(1, n))])
    assert abs(lv[0, 1] - C / (1 + C)) < 1e-14
    assert abs(lv[1, 0] - C / (1 + C)) < 1e-14
    assert abs(lv[1, 1] - (ALPHA / L + C * C / (L * (1 + C)))) < 1e-14
    assert abs(lv[0, 0] - L / (1 + C)) < 1e-13


def test_node_distribution_and_ulcv_hand_values():
    # unit square: four sides of length 1 and two diagonals of length sqrt(2):
    # ND = 4 * 1 + 2 * 1/2 = 5; a coincident pair makes ND infinite
    sq = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    assert abs(O.node_distribution(sq) - 5.0) < 1e-14
    assert O.node_distribution(np.array([[0.0, 0.0], [1.0, 2.0], [0.0, 0.0]])) == float("inf")
    # equal edge lengths: ULCV = 0; lengths 1 and 3: mean 2, population std 1
    assert O.ulcv(sq, [(0, 1), (1, 2), (2, 3), (3, 0)]) < 1e-15
    pts = np.array([[0.0, 0.0], [1.0, 0.0], [4.0, 0.0]])
    assert abs(O.ulcv(pts, [(0, 1), (1, 2)]) - 0.5) < 1e-15
    # invariances: ND and ULCV do not change under rotation and translation;
    # scaling X by s multiplies ND by 1/s^2 and leaves ULCV unchanged
    X = synth.uniform_x0(20, seed=4).astype(np.float64) * 3
    th = 0.4
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    E = [(i, (i * 7 + 3) % 20) for i in range(20) if i != (i * 7 + 3) % 20]
    assert abs(O.node_distribution(X @ R.T + 2.0) - O.node_distribution(X)) < 1e-9 * O.node_distribution(X)
    assert abs(O.node_distribution(2.0 * X) - O.node_distribution(X) / 4.0) < 1e-12 * O.node_distribution(X)
    assert abs(O.ulcv(X @ R.T - 1.0, E) - O.ulcv(X, E)) < 1e-12
    assert abs(O.ulcv(5.0 * X, E) - O.ulcv(X, E)) < 1e-12


def test_directed_walk_closed_forms():
    # Sec. 2.1's directed setting. Cycle a -> b -> c -> a: the walk from a is at
    # step t on node t mod 3, so pi(a, .) = alpha (1, c, c^2) / (1 - c^3).
    rp, col = _csr_from_edges(3, [(0, 1), (1, 2), (2, 0)], False)
    Pi = O.ppr_rows(O.transition_matrix(3, rp, col), [0], ALPHA)
    z = 1 - C ** 3
    assert np.allclose(Pi[0], [ALPHA / z, ALPHA * C / z, ALPHA * C * C / z], atol=1e-15, rtol=0)
    # a -> b with b dangling (reading 2: the walk stays on b): pi(a, a) = alpha,
    # pi(a, b) = c, pi(b, b) = 1; d(b) = 0 so b's DPPR row is 0
    rp, col = _csr_from_edges(2, [(0, 1)], False)
    P = O.transition_matrix(2, rp, col)
    Pi = O.ppr_rows(P, [0, 1], ALPHA)
    assert np.allclose(Pi, [[ALPHA, C], [0.0, 1.0]], atol=1e-15, rtol=0)
    d = O.degrees(2, rp, col)
    D = O.dppr_rows(Pi, d, [0, 1])
    assert np.all(D[1] == 0.0) and abs(D[0, 1] - C) < 1e-15
    # the direct solve agrees on a random directed graph with dangling nodes,
    # and every PPR row is a distribution
    g = synth.directed_from(synth.chung_lu(150, 8, 2.5, seed=3), seed=4)
    P = O.transition_matrix(g.n, g.row_ptr, g.col)
    rows = O.ppr_rows(P, np.arange(g.n), ALPHA)
    assert np.abs(rows - O.ppr_direct(P, ALPHA)).max() < 1e-13
    assert np.abs(rows.sum(axis=1) - 1).max() < 1e-13


# --------------------------------------------------------------------------
# Sec. 4: backward push, DPR (Eq. (dnpr-dnppr)), GFP / GBP / Tau-Push
# (Algorithms 1-3) against the exact level-l DPPR of a direct solve
# --------------------------------------------------------------------------
def test_backward_push_example():
    with open(os.path.join(GOLDEN, "backward_push_example.json")) as f:
        ex = json.load(f)
    n, a, t = ex["n"], ex["alpha"], ex["target"]
    rp, col = _csr_from_edges(n, [tuple(e) for e in ex["edges"]], False)
    P = O.transition_matrix(n, rp, col)
    est, r = O.backward_push(P, t, a, ex["after_first_push"]["order"])
    for v, val in ex["after_first_push"]["estimate"].items():
        assert abs(est[int(v)] - val) < 1e-15
    for v, val in ex["after_first_push"]["residue"].items():
        assert abs(r[int(v)] - val) < 1e-15
    assert np.count_nonzero(r) == 2 and np.count_nonzero(est) == 1
    # the backward invariant pi(s, t) = est_s + sum_k pi(s, k) r_k holds for
    # every s after any sequence of pushes
    Pi = O.ppr_direct(P, a)
    for order in ([10], [10, 5, 6], [10, 6, 5, 9, 10]):
        est, r = O.backward_push(P, t, a, order)
        assert np.abs(Pi[:, t] - (est + Pi @ r)).max() < 1e-15


def _tp_graphs():
    """Small graphs covering the unweighted, weighted and directed (with
    dangling nodes) walks."""
    g_u = synth.sbm([14, 12, 10, 9], 0.35, 0.04, seed=21)
    rng = np.random.default_rng(5)
    wedges = []
    for u in range(g_u.n):
        for q in range(g_u.row_ptr[u], g_u.row_ptr[u + 1]):
            v = int(g_u.col[q])
            if u < v:
                wedges.append((u, v, float(np.exp(rng.normal()))))
    rp_w, col_w, w_w = _weighted_csr_from_edges(g_u.n, wedges)
    g_d = synth.directed_from(g_u, p_both=0.3, dangling=0.08, seed=6)
    out = [("unweighted", g_u.n, g_u.row_ptr, g_u.col, None),
           ("weighted", g_u.n, rp_w, col_w, w_w),
           ("directed", g_d.n, g_d.row_ptr, g_d.col, None)]
    return out


def _tp_exact(n, rp, col, w, leaf_sets, alpha):
    P = O.transition_matrix(n, rp, col, w)
    d = O.degrees(n, rp, col, w)
    full = d[:, None] * O.ppr_direct(P, alpha)
    return P, d, O.level_dppr(full, leaf_sets)


def _tp_leaf_sets(n, sizes, seed):
    perm = np.argsort(synth.uniform(seed, 31, np.arange(n)))
    out, at = [], 0
    for s in sizes:
        out.append([int(v) for v in perm[at:at + s]])
        at += s
    return out


def test_dpr_closed_form_and_definition():
    """Undirected: pi_d is symmetric, so sum_k pi_d(v_k, t) = d(t) and
    tau_t = d(t) / m. Directed: the index precompute (PageRank from d / m)
    equals the definition; either way sum_t tau_t = 1."""
    for name, n, rp, col, w in _tp_graphs():
        P = O.transition_matrix(n, rp, col, w)
        d = O.degrees(n, rp, col, w)
        t_def = O.dpr(P, d, ALPHA)
        t_pow = O.dpr_power(P, d, ALPHA)
        assert np.abs(t_def - t_pow).max() < 1e-15, name
        assert abs(t_def.sum() - 1.0) < 1e-13, name
        if name != "directed":
            assert np.abs(t_def - d / d.sum()).max() < 1e-15, name
        else:
            assert np.abs(t_def - d / d.sum()).max() > 1e-3  # the closed form is undirected-only


def test_gfp_meets_its_error_bound():
    """Lemma 2 (with Lemma 4's invariant): GFP underestimates, by at most
    r_max m tau_j for target V_j; with a tiny r_max it reaches Eq. (2)."""
    for name, n, rp, col, w in _tp_graphs():
        leaf_sets = _tp_leaf_sets(n, [1, 3, 5, 2, 7], seed=3)
        P, d, exact = _tp_exact(n, rp, col, w, leaf_sets, ALPHA)
        tau_nodes = O.dpr(P, d, ALPHA)
        tau_j = np.array([tau_nodes[F].mean() for F in leaf_sets])
        m = d.sum()
        for r_max in (3e-3, 2e-4):
            for i in range(len(leaf_sets)):
                est = O.gfp(P, d, leaf_sets, i, ALPHA, r_max)
                err = exact[i] - est
                assert np.all(err >= -1e-15), (name, i, err)
                assert np.all(err <= r_max * m * tau_j + 1e-15), (name, i, err, r_max * m * tau_j)
        for i in range(len(leaf_sets)):
            est = O.gfp(P, d, leaf_sets, i, ALPHA, 1e-15)
            assert np.abs(exact[i] - est).max() < 1e-12, name


def test_gbp_meets_its_error_bound():
    """Lemma 3 (with its invariant): GBP towards V_j underestimates
    pi_d(V_i, V_j) by at most rb_max times the mean leaf degree of V_i; with a
    tiny rb_max it reaches Eq. (2)."""
    for name, n, rp, col, w in _tp_graphs():
        leaf_sets = _tp_leaf_sets(n, [2, 1, 4, 6, 3], seed=4)
        P, d, exact = _tp_exact(n, rp, col, w, leaf_sets, ALPHA)
        davg = np.array([d[F].mean() for F in leaf_sets])
        for rb_max in (2e-2, 1e-3):
            for j in range(len(leaf_sets)):
                est = O.gbp(P, d, leaf_sets, j, ALPHA, rb_max)
                err = exact[:, j] - est
                assert np.all(err >= -1e-15), (name, j, err)
                assert np.all(err <= rb_max * davg + 1e-15), (name, j, err, rb_max * davg)
        for j in range(len(leaf_sets)):
            est = O.gbp(P, d, leaf_sets, j, ALPHA, 1e-16)
            assert np.abs(exact[:, j] - est).max() < 1e-12, name


def test_tau_push_is_eps_delta_approximate():
    """Theorem 3: every off-diagonal estimate meets Definition 3 (absolute
    eps delta below delta, relative eps above), whichever targets the DPR
    threshold sends to GBP: the paper's tau = 1 / sqrt(k n), none, all."""
    eps, delta = 1 - 1 / math.e, 0.01
    for name, n, rp, col, w in _tp_graphs():
        leaf_sets = _tp_leaf_sets(n, [3, 1, 4, 2, 5, 2], seed=5)
        k = len(leaf_sets)
        P, d, exact = _tp_exact(n, rp, col, w, leaf_sets, ALPHA)
        tau_nodes = O.dpr(P, d, ALPHA)
        tau_j = np.array([tau_nodes[F].mean() for F in leaf_sets])
        for tau, want in ((None, None), (10.0, []), (1e-12, list(range(k)))):
            est, t, r_max, refined = O.tau_push(P, d, leaf_sets, ALPHA, eps, delta, tau_nodes, tau)
            assert t == (1 / math.sqrt(k * n) if tau is None else tau)
            assert abs(r_max - eps * delta / (d.sum() * t)) <= 1e-18
            assert list(refined) == [j for j in range(k) if tau_j[j] > t]
            if want is not None:
                assert list(refined) == want
            # Lemma 3's condition: rb_max is the largest threshold whose bound
            # rb_max * (mean leaf degree of V_i) stays within eps delta for
            # every source V_i other than the target
            davg = np.array([d[F].mean() for F in leaf_sets])
            for j, rb in refined.items():
                worst = max(rb * davg[i] for i in range(k) if i != j)
                assert abs(worst - eps * delta) <= 1e-15, (j, worst)
            off = ~np.eye(k, dtype=bool)
            err = np.abs(est - exact)[off]
            ex = exact[off]
            bound = np.where(ex < delta, eps * delta, eps * ex)
            assert np.all(err <= bound + 1e-15), (name, tau, err.max())
            assert np.all(est <= exact + 1e-15)
        # tight eps delta: both phases reach Eq. (2)
        est, *_ = O.tau_push(P, d, leaf_sets, ALPHA, 1e-7, 1e-7, tau_nodes, 1e-12)
        assert np.abs(est - exact)[~np.eye(k, dtype=bool)].max() < 1e-13
        est, *_ = O.tau_push(P, d, leaf_sets, ALPHA, 1e-7, 1e-7, tau_nodes, 10.0)
        assert np.abs(est - exact).max() < 1e-10


def test_level_dppr_rows_power_matches_the_definition():
    """The group-start power iteration gives the rows of Eq. (2) as the
    leaf-set average of the dense DPPR matrix does."""
    for name, n, rp, col, w in _tp_graphs():
        leaf_sets = _tp_leaf_sets(n, [4, 1, 6, 3], seed=7)
        P, d, exact = _tp_exact(n, rp, col, w, leaf_sets, ALPHA)
        rows = O.level_dppr_rows_power(P, d, leaf_sets, [0, 2, 3], ALPHA)
        assert np.abs(rows - exact[[0, 2, 3]]).max() < 1e-13, name


# --------------------------------------------------------------------------
# Louvain+ hierarchy (Sec. 5 preprocessing; Appendix A merge rules)
# --------------------------------------------------------------------------
def test_louvain_gain_is_the_change_of_newman_modularity():
    """Q^(S, T) summed from the appendix's q(V_i, T) must equal the change of
    the partition's modularity (Newman's definition, brute force over the
    leaf edges) when S is merged into T, for level nodes that are groups of
    leaves and for S and T that are groups of level nodes."""
    rng = np.random.default_rng(3)
    for trial in range(12):
        n = int(rng.integers(8, 30))
        edges = {(int(a), int(b)) for a, b in rng.integers(0, n, size=(3 * n, 2)) if a != b}
        row_ptr, col = _csr_from_edges(n, edges, undirected=True)
        if row_ptr[-1] == 0:
            continue
        # level nodes: random groups of leaves; supernodes S, T: random sets of level nodes
        nl = int(rng.integers(3, min(n, 10) + 1))
        level_of_leaf = [int(x) for x in rng.permutation(np.arange(n) % nl)]
        leaves_of = {A: [u for u in range(n) if level_of_leaf[u] == A] for A in range(nl)}
        nodes = [int(x) for x in rng.permutation(nl)]
        cut = int(rng.integers(1, nl))
        S = set(nodes[:cut])
        T = set(nodes[cut:cut + int(rng.integers(1, nl - cut + 1))])
        # partition of the leaves before (each level node alone, T as one community) and after
        def part_of(merge):
            part = []
            for u in range(n):
                A = level_of_leaf[u]
                if A in T or (merge and A in S):
                    part.append(-1)
                elif A in S:
                    part.append(-2)  # S as one community before the merge
                else:
                    part.append(A)
            return part
        before = O.modularity(row_ptr, col, part_of(False))
        after = O.modularity(row_ptr, col, part_of(True))
        gain = O.louvain_gain(S, T, leaves_of, row_ptr, col, level_of_leaf)
        assert gain == after - before, trial


def test_louvain_plus_splits_two_cliques_at_the_bridge():
    """Two 4-cliques joined by one edge: modularity's textbook optimum puts
    each clique in its own community (k = 4 forbids nothing else)."""
    edges = [(a, b) for a in range(4) for b in range(a + 1, 4)]
    edges += [(a + 4, b + 4) for a, b in edges] + [(3, 4)]
    row_ptr, col = _csr_from_edges(8, edges, undirected=True)
    levels = O.louvain_plus(8, row_ptr, col, 4)
    assert len(levels) == 1
    assert levels[0].tolist() == [0, 0, 0, 0, 1, 1, 1, 1]
    assert O.louvain_plus(8, row_ptr, col, 8) == []  # n <= k: the leaves fit one view


def _ring_of_cliques(c, q):
    edges = []
    for b in range(q):
        base = b * c
        edges += [(base + i, base + j) for i in range(c) for j in range(i + 1, c)]
        edges.append((base + c - 1, ((b + 1) % q) * c))
    return _csr_from_edges(c * q, edges, undirected=True)


def test_louvain_plus_finds_the_cliques_of_a_ring():
    """A ring of six 5-cliques, each joined to the next by one edge: the
    partition into the cliques is modularity's optimum (Q = 0.742 here;
    the ring is far below the resolution limit), and it is level 1 for k = 5
    and k = 7 (for k = 7 also the top: 6 <= k)."""
    row_ptr, col = _ring_of_cliques(5, 6)
    cliques = np.repeat(np.arange(6), 5)
    for k in (5, 7):
        levels = O.louvain_plus(30, row_ptr, col, k)
        assert levels[0].tolist() == cliques.tolist()
    assert len(O.louvain_plus(30, row_ptr, col, 7)) == 1
    q = O.modularity(row_ptr, col, cliques)
    assert abs(float(q) - (60 / 66 - 6 * (22 / 132) ** 2)) < 1e-15


def test_louvain_plus_rule_i_on_a_star_and_a_path():
    """Rule (i) by hand. Star of 6 leaves, k = 4: every leaf's only neighbour
    is the hub, which takes leaves 1-3 (cap 4); leaves 4-6 stay alone.
    Path 0-..-5, k = 2: the ends join their neighbours by rule (i), the
    middle pair by rule (ii) (gain 2m - 2*2*2 > 0); at level 2 the first
    pair takes the middle pair (rule (i)), the last pair is left by the cap."""
    row_ptr, col = _csr_from_edges(7, [(0, i) for i in range(1, 7)], undirected=True)
    levels = O.louvain_plus(7, row_ptr, col, 4)
    assert [p.tolist() for p in levels] == [[0, 0, 0, 0, 1, 2, 3]]
    row_ptr, col = _csr_from_edges(6, [(i, i + 1) for i in range(5)], undirected=True)
    levels = O.louvain_plus(6, row_ptr, col, 2)
    assert [p.tolist() for p in levels] == [[0, 0, 1, 1, 2, 2], [0, 0, 1]]


@pytest.mark.parametrize("k", [3, 8])
def test_louvain_plus_hierarchy_invariants(k):
    """On a connected power-law graph: every supernode has at most k
    children, every level is onto 0..n_l-1 and numbered by smallest child,
    every level is smaller than the one below, and the top has at most k
    supernodes."""
    g = synth.chung_lu(160, 5, 2.5, seed=2)
    # keep the largest connected component's guarantee simple: join the graph by a path
    edges = {(u, int(v)) for u in range(g.n) for v in g.col[g.row_ptr[u]:g.row_ptr[u + 1]] if u < v}
    edges |= {(i, i + 1) for i in range(g.n - 1)}
    row_ptr, col = _csr_from_edges(g.n, edges, undirected=True)
    levels = O.louvain_plus(g.n, row_ptr, col, k)
    assert levels
    n_prev = g.n
    for p in levels:
        assert len(p) == n_prev
        n_l = int(p.max()) + 1
        assert n_l < n_prev
        counts = np.bincount(p, minlength=n_l)
        assert counts.min() >= 1 and counts.max() <= k
        first = [int(p[np.flatnonzero(p == s)[0]]) for s in range(n_l)]
        firsts = [int(np.flatnonzero(p == s)[0]) for s in range(n_l)]
        assert first == list(range(n_l)) and firsts == sorted(firsts)
        n_prev = n_l
    assert n_prev <= k
