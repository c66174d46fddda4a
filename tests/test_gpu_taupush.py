"""GPU parity of Tau-Push (Sec. 4, Algorithms 1-3) and its DPR index
(Eq. (dnpr-dnppr), Sec. 4.3) against the FP64 oracle, through the C ABI
(pprviz_tau_push, pprviz_dpr).

The GPU pushes in synchronous rounds, the oracle one node at a time (first
in, first out), so the two push in different orders and their estimates
differ; several results are correct. What is unique is checked exactly: the
DPR threshold tau, r_max and the set of refined targets. The rest is checked
for validity against the exact level-l DPPR of Eq. (2) (a direct solve, or
the oracle's group-start power iteration at full size): every estimate is at
most the exact value and misses it by at most Lemma 2's r_max m tau_j
(forward columns) or Lemma 3's rb_max d_i (refined columns), which gives
Theorem 3's (eps, delta) guarantee; the GPU and oracle estimates then lie
within that same bound of each other. Slack for rounding: 1e-12 absolute.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu
ALPHA = 0.15
EPS_P = 1 - 1 / math.e  # the paper's eps (Sec. 6 settings)
SLACK = 1e-12


@pytest.fixture(scope="module")
def ctx():
    import paper_2112_14944_gb300 as P
    c = P.Context(0)
    yield c
    c.close()


def _weighted(g, seed):
    """Symmetric lognormal(0, 1) weights on an undirected graph's edges."""
    u = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    v = g.col.astype(np.int64)
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    key = lo * g.n + hi
    z = synth.uniform(seed, 41, key.astype(np.uint64))
    z2 = synth.uniform(seed, 42, key.astype(np.uint64))
    w = np.exp(np.sqrt(-2 * np.log1p(-z)) * np.cos(2 * np.pi * z2)).astype(np.float32)
    return synth.Graph(g.n, g.row_ptr, g.col, w)


def _graphs():
    g_u = synth.sbm([300, 250, 200, 150, 100], 0.04, 0.002, seed=31)
    return [("unweighted", g_u), ("weighted", _weighted(g_u, 3)),
            ("directed", synth.directed_from(g_u, p_both=0.3, dangling=0.03, seed=7))]


def _oracle_setup(g, leaf_sets):
    P = O.transition_matrix(g.n, g.row_ptr, g.col, g.weight)
    d = O.degrees(g.n, g.row_ptr, g.col, g.weight)
    full = d[:, None] * O.ppr_direct(P, ALPHA)
    return P, d, O.level_dppr(full, leaf_sets)


def _bounds(d, leaf_sets, dpr_nodes, tau, r_max, eps, delta):
    """Per entry (i, j): the error bound of the phase that produced it."""
    k = len(leaf_sets)
    m = d.sum()
    davg = np.array([d[F].mean() for F in leaf_sets])
    tau_j = np.array([dpr_nodes[F].mean() for F in leaf_sets])
    bound = np.tile(r_max * m * tau_j, (k, 1))
    refined = [j for j in range(k) if tau_j[j] > tau]
    for j in refined:
        others = [davg[i] for i in range(k) if i != j]
        dmax = max(others) if others else davg[j]
        rb = eps * delta / dmax if dmax > 0 else math.inf
        bound[:, j] = rb * davg if math.isfinite(rb) else np.inf
    return bound, refined


def _check_valid(est, exact, bound, tag):
    err = exact - est
    assert np.all(err >= -SLACK), (tag, err.min())
    assert np.all(err <= bound + SLACK), (tag, np.max(err - bound))


def _leaf_sets(ptr, idx):
    return [idx[ptr[i]:ptr[i + 1]].astype(np.int64) for i in range(len(ptr) - 1)]


def test_dpr_undirected_closed_form(ctx):
    """Undirected graphs: tau_t = d(t) / m (pi_d is symmetric), for an
    unweighted power-law graph and a weighted SBM; the L1 error is within the
    returned bound."""
    for g in (synth.chung_lu(20000, 12, seed=5), _weighted(synth.sbm([400, 300, 300], 0.05, 0.003, seed=9), 1)):
        G = ctx.upload_graph(g)
        dpr, cert = ctx.dpr(G, ALPHA, 1e-12)
        d = O.degrees(g.n, g.row_ptr, g.col, g.weight)
        ref = d / d.sum()
        assert cert <= 1e-12
        assert np.abs(dpr - ref).sum() <= cert + 1e-13
        assert np.abs(dpr - ref).max() <= 1e-13


def test_dpr_directed_matches_oracle(ctx):
    """Directed graph with dangling nodes: the GPU DPR against the oracle's
    index precompute (itself pinned to the definition)."""
    g = synth.directed_from(synth.chung_lu(3000, 8, seed=2), p_both=0.3, dangling=0.03, seed=4)
    G = ctx.upload_graph(g)
    dpr, cert = ctx.dpr(G, ALPHA, 1e-13)
    P = O.transition_matrix(g.n, g.row_ptr, g.col)
    d = O.degrees(g.n, g.row_ptr, g.col)
    ref = O.dpr_power(P, d, ALPHA)
    assert np.abs(dpr - ref).sum() <= cert + 1e-13
    assert abs(dpr.sum() - 1.0) <= cert + 1e-12


@pytest.mark.parametrize("tau", [0.0, 10.0, 1e-12])
def test_tau_push_matches_oracle_within_bounds(ctx, tau):
    """Unweighted, weighted and directed (dangling nodes) SBM graphs of 1,000
    nodes; six children of mixed leaf counts (1 to 40 leaves); the paper's
    eps and delta = 1 / (10 k) with the paper's tau, with no refined target
    and with every target refined."""
    sizes = [1, 5, 40, 12, 3, 25]
    k = len(sizes)
    delta = 1.0 / (10 * k)
    for name, g in _graphs():
        ptr, idx = synth.random_leaf_sets(g.n, sizes, seed=11)
        leaf_sets = _leaf_sets(ptr, idx)
        P, d, exact = _oracle_setup(g, leaf_sets)
        dpr_nodes = O.dpr(P, d, ALPHA)
        G = ctx.upload_graph(g)
        est, Pd, info = ctx.tau_push(G, ptr, idx, dpr_nodes, ALPHA, EPS_P, delta, tau)
        ref, t_ref, r_ref, refined = O.tau_push(P, d, leaf_sets, ALPHA, EPS_P, delta, dpr_nodes,
                                                None if tau == 0.0 else tau)
        assert info["tau"] == t_ref, (name, info)
        assert abs(info["r_max"] - r_ref) <= 1e-14 * r_ref, (name, info)  # m summed in another order
        assert info["backward_targets"] == len(refined), (name, info, refined)
        bound, refined_b = _bounds(d, leaf_sets, dpr_nodes, t_ref, r_ref, EPS_P, delta)
        assert refined_b == list(refined)
        _check_valid(est, exact, bound, (name, tau))
        assert np.all(np.abs(est - ref) <= bound + SLACK), (name, tau)
        # Definition 3 off the diagonal
        off = ~np.eye(k, dtype=bool)
        lim = np.where(exact < delta, EPS_P * delta, EPS_P * exact)
        assert np.all(np.abs(est - exact)[off] <= lim[off] + SLACK), name
        # PDist of the estimates (Algorithm 1, conversion step)
        assert np.allclose(Pd, O.pdist_from_dppr(est, g.n), rtol=0, atol=1e-12)
        if tau == 1e-12:
            assert info["bwd_pushes"] > 0
        if tau == 10.0:
            assert info["backward_targets"] == 0 and info["bwd_pushes"] == 0


def test_tau_push_tight_thresholds_reach_eq2(ctx):
    """With eps delta = 1e-14 both phases reach Eq. (2): forward only
    (tau = 10) everywhere, every target refined (tau = 1e-12) off the
    diagonal (Theorem 3 covers i != j)."""
    sizes = [2, 7, 1, 30]
    for name, g in _graphs():
        ptr, idx = synth.random_leaf_sets(g.n, sizes, seed=13)
        leaf_sets = _leaf_sets(ptr, idx)
        P, d, exact = _oracle_setup(g, leaf_sets)
        dpr_nodes = O.dpr(P, d, ALPHA)
        G = ctx.upload_graph(g)
        est, _, info = ctx.tau_push(G, ptr, idx, dpr_nodes, ALPHA, 1e-7, 1e-7, 10.0, want_pdist=False)
        assert np.abs(est - exact).max() <= 1e-10, (name, np.abs(est - exact).max())
        est, _, info = ctx.tau_push(G, ptr, idx, dpr_nodes, ALPHA, 1e-7, 1e-7, 1e-12, want_pdist=False)
        assert info["backward_targets"] == len(sizes)
        off = ~np.eye(len(sizes), dtype=bool)
        assert np.abs(est - exact)[off].max() <= 1e-10, name


def test_tau_push_degenerate_cases(ctx):
    """One child holding every node; singleton leaves (level 0); leaves of
    degree 0 (isolated nodes); thresholds so loose that nothing is pushed
    (every estimate 0, PDist at its upper clamp)."""
    base = synth.sbm([120, 100, 80], 0.06, 0.004, seed=17)
    # two isolated nodes appended
    n = base.n + 2
    rp = np.concatenate([base.row_ptr, [base.row_ptr[-1]] * 2]).astype(np.int64)
    g = synth.Graph(n, rp, base.col, None)
    G = ctx.upload_graph(g)
    P = O.transition_matrix(n, g.row_ptr, g.col)
    d = O.degrees(n, g.row_ptr, g.col)
    full = d[:, None] * O.ppr_direct(P, ALPHA)
    dpr_nodes = O.dpr(P, d, ALPHA)
    cases = {
        "one child": [np.arange(n)],
        "level 0": [np.array([v]) for v in (0, 5, 130, 250, 300, n - 1)],
        "isolated leaves": [np.array([n - 2, n - 1]), np.array([1, 2, 3]), np.array([n - 3])],
    }
    for name, leaf_sets in cases.items():
        ptr, idx = ctx.leaf_csr(leaf_sets)
        exact = O.level_dppr(full, leaf_sets)
        k = len(leaf_sets)
        for tau in (0.0, 1e-12):
            est, _, info = ctx.tau_push(G, ptr, idx, dpr_nodes, ALPHA, EPS_P, 1.0 / (10 * k), tau,
                                        want_pdist=False)
            ref, t_ref, r_ref, _ = O.tau_push(P, d, leaf_sets, ALPHA, EPS_P, 1.0 / (10 * k), dpr_nodes,
                                              None if tau == 0.0 else tau)
            bound, _ = _bounds(d, leaf_sets, dpr_nodes, t_ref, r_ref, EPS_P, 1.0 / (10 * k))
            _check_valid(est, exact, bound, (name, tau))
            assert np.all(np.abs(est - ref) <= bound + SLACK), (name, tau)
    # nothing above the thresholds: eps delta so large that r_max > 1 / |F|
    ptr, idx = ctx.leaf_csr(cases["level 0"])
    est, Pd, info = ctx.tau_push(G, ptr, idx, dpr_nodes, ALPHA, 1e6, 1e6, 10.0)
    assert info["fwd_pushes"] == 0 and np.all(est == 0)
    off = ~np.eye(6, dtype=bool)
    assert np.all(Pd[off] == 2 * math.log(n))


def test_tau_push_device_buffers_match_host(ctx):
    """The same query on device (torch) buffers: same thresholds and pushes
    within the bound of the host call's estimates."""
    torch = pytest.importorskip("torch")
    name, g = _graphs()[0]
    sizes = [3, 9, 1, 20]
    ptr, idx = synth.random_leaf_sets(g.n, sizes, seed=19)
    P = O.transition_matrix(g.n, g.row_ptr, g.col)
    d = O.degrees(g.n, g.row_ptr, g.col)
    dpr_nodes = O.dpr(P, d, ALPHA)
    G = ctx.upload_graph(g)
    est_h, pd_h, info_h = ctx.tau_push(G, ptr, idx, dpr_nodes, ALPHA, EPS_P, 0.025, 0.0)
    dev = torch.device("cuda", 0)
    k = len(sizes)
    out = torch.empty((k, k), dtype=torch.float64, device=dev)
    pdo = torch.empty((k, k), dtype=torch.float64, device=dev)
    est_d, pd_d, info_d = ctx.tau_push(G, torch.from_numpy(ptr).to(dev), torch.from_numpy(idx).to(dev),
                                       torch.from_numpy(dpr_nodes).to(dev), ALPHA, EPS_P, 0.025, 0.0,
                                       ldppr_out=out, pdist_out=pdo)
    torch.cuda.synchronize()
    assert info_d["tau"] == info_h["tau"] and info_d["r_max"] == info_h["r_max"]
    leaf_sets = _leaf_sets(ptr, idx)
    bound, _ = _bounds(d, leaf_sets, dpr_nodes, info_h["tau"], info_h["r_max"], EPS_P, 0.025)
    assert np.all(np.abs(out.cpu().numpy() - est_h) <= bound + SLACK)
    assert np.allclose(pdo.cpu().numpy(), O.pdist_from_dppr(out.cpu().numpy(), g.n), rtol=0, atol=1e-12)


def test_tau_push_rejects_bad_input(ctx):
    import paper_2112_14944_gb300 as P
    g = synth.sbm([60, 40], 0.1, 0.01, seed=3)
    G = ctx.upload_graph(g)
    ptr, idx = synth.random_leaf_sets(g.n, [3, 4], seed=1)
    dpr_nodes = np.full(g.n, 1.0 / g.n)
    for kw in ({"eps": 0.0}, {"delta": -1.0}, {"tau": math.inf}, {"alpha": 1.0}):
        args = dict(alpha=ALPHA, eps=EPS_P, delta=0.05, tau=0.0)
        args.update(kw)
        with pytest.raises(P.PPRVizError):
            ctx.tau_push(G, ptr, idx, dpr_nodes, **args)
    bad = dpr_nodes.copy()
    bad[7] = -1e-3
    with pytest.raises(P.PPRVizError):
        ctx.tau_push(G, ptr, idx, bad, ALPHA, EPS_P, 0.05)
    bad[7] = math.nan
    with pytest.raises(P.PPRVizError):
        ctx.tau_push(G, ptr, idx, bad, ALPHA, EPS_P, 0.05)
    with pytest.raises(P.PPRVizError):  # overlapping leaf sets
        ctx.tau_push(G, np.array([0, 2, 4], dtype=np.int64), np.array([1, 2, 2, 3], dtype=np.int32), dpr_nodes,
                     ALPHA, EPS_P, 0.05)


@pytest.mark.parametrize("per", [1, 25])
def test_tau_push_full_size_sampled(ctx, per):
    """The 2,000,000-node Chung-Lu graph (mean degree 10): a level-0 query
    (25 single nodes) and a level-1 query (25 children of 25 leaves), the
    paper's eps, delta and tau; two sampled source rows against the oracle's
    group-start power iteration (to 1e-9 of the walk mass); the DPR index
    from the GPU equals the closed form d / m."""
    g = synth.chung_lu(2_000_000, 10, seed=0)
    G = ctx.upload_graph(g)
    d = O.degrees(g.n, g.row_ptr, g.col)
    dpr_gpu, cert = ctx.dpr(G, ALPHA, 1e-12)
    dpr_nodes = d / d.sum()
    assert np.abs(dpr_gpu - dpr_nodes).max() <= 1e-13
    k = 25
    ptr, idx = synth.random_leaf_sets(g.n, [per] * k, seed=23)
    leaf_sets = _leaf_sets(ptr, idx)
    delta = 1.0 / (10 * k)
    est, _, info = ctx.tau_push(G, ptr, idx, dpr_gpu, ALPHA, EPS_P, delta, 0.0, want_pdist=False)
    assert info["tau"] == 1 / math.sqrt(k * g.n)
    assert info["fwd_pushes"] > 0
    P = O.transition_matrix(g.n, g.row_ptr, g.col)
    rows = [0, 17]
    exact = O.level_dppr_rows_power(P, d, leaf_sets, rows, ALPHA, tol=1e-9)
    bound, refined = _bounds(d, leaf_sets, dpr_nodes, info["tau"], info["r_max"], EPS_P, delta)
    assert info["backward_targets"] == len(refined)
    oracle_err = 1e-9 * max(d[leaf_sets[i]].mean() for i in rows)
    for c, i in enumerate(rows):
        err = exact[c] - est[i]
        assert np.all(err >= -oracle_err - SLACK), (i, err.min())
        assert np.all(err <= bound[i] + oracle_err + SLACK), (i, np.max(err - bound[i]))
