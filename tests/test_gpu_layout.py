"""GPU parity of the layout pass, Guttman solve, energy/gradients and the
batched-views path (P4-P7) against the FP64 oracle, through the C ABI.

Tolerances:
  FP64 layout: the whole trajectory, coordinates within 1e-4 * max(1, |x|)
               after the fixed iteration count from the same X0.
  FP32 layout: one update from the same X_t within 1e-4 * max(1, |X|_max)
               (a whole FP32 trajectory is not reproducible to 1e-4: the
               stress-majorization map amplifies a 6e-8 perturbation of its
               matrices to ~2e-4 within 300 updates even in FP64 arithmetic),
               plus trajectory properties: non-increasing stress, centred
               output, final stress within 1e-3 of the oracle's.
  Energy: relative 1e-12 (FP64), 1e-5 (FP32); gradients likewise.
  Batched vs single-view FP32 layout: the batched passes group a view's
               column sums by the CTA chunks of the whole batch, so they add
               the same FP32 terms in another order; one update agrees within
               1e-5 * max(1, |X|_max) and final stresses within 1e-4
               relative; after 40-200 updates (the same amplification) the
               final stresses agree within 1e-3 relative and both layouts are
               finite and centred. The batched propagation advances many views'
               sources in shared launches; each view's PDist is gated
               against the oracle with its own certificates.
  Batched FP32 layout vs the oracle: with a tight eps (1e-9) one batched
               update of each checked view matches the oracle's update on the
               oracle's PDist within 1e-4 * max(1, |X|_max), and (small views)
               the final stress after 40 updates within 1e-3 of the oracle's.
Every oracle input (PDist, coordinates) comes from the oracle or the seeded
generators, never from the GPU.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth
from _parity import check_pdist, oracle_dppr, oracle_pdist

pytestmark = pytest.mark.gpu
ALPHA = 0.15


@pytest.fixture(scope="module")
def ctx():
    import paper_2112_14944_gb300 as P
    c = P.Context(0)
    yield c
    c.close()


def _pdist_for(n, mean_deg, seed):
    """The oracle's FP64 PDist of a seeded Chung-Lu graph (exponent 2.5)."""
    return oracle_pdist(synth.chung_lu(n, mean_deg, 2.5, seed=seed), ALPHA)


def _rel(a, b):
    return np.abs(np.asarray(a, np.float64) - b) / np.maximum(1.0, np.abs(b))


def _same_layout(X1, Xb, s1, sb, tol):
    """Batched and single-view FP32 layouts of one view after one update: the
    same update up to FP32 summation order."""
    scale = max(1.0, float(np.abs(X1).max()))
    assert np.abs(np.asarray(Xb, np.float64) - X1).max() <= tol * scale
    assert abs(sb - s1) <= 1e-4 * abs(s1)


def _same_trajectory(X1, Xb, s1, sb):
    """Batched and single-view FP32 layouts of one view after many updates. The
    two runs add the same terms in another order, and stress majorization
    amplifies that rounding difference along the trajectory (to ~6e-3 of the
    layout's scale after a few hundred updates at n of a few thousand, even in
    FP64 arithmetic on FP32-rounded matrices), so coordinates are not compared
    one by one: the final stresses agree to 1e-3 relative, and both layouts
    are finite and centred."""
    Xb = np.asarray(Xb, np.float64)
    assert np.all(np.isfinite(Xb)) and np.all(np.isfinite(X1))
    assert np.abs(Xb.mean(0)).max() <= 1e-3 and np.abs(np.asarray(X1, np.float64).mean(0)).max() <= 1e-3
    assert abs(sb - s1) <= 1e-3 * abs(s1)


def test_layout_fp64_config_small_full_trajectory(ctx):
    """n = 1,000 Chung-Lu (mean degree 10), 300 updates from U[-1,1]^2, FP64."""
    import paper_2112_14944_gb300 as P
    Delta = _pdist_for(1000, 10, 0)
    x0 = synth.uniform_x0(1000, seed=0).astype(np.float64)
    X, stress = ctx.layout(Delta, x0, 300, P.FP64)
    Xr, hist = O.smacof(x0, Delta, 300)
    assert _rel(X, Xr).max() <= 1e-4
    assert abs(stress - hist[-1]) <= 1e-9 * hist[-1]


def test_layout_fp32_one_step_matches_oracle(ctx):
    import paper_2112_14944_gb300 as P
    Delta32 = _pdist_for(1500, 10, 3).astype(np.float32)
    D64 = Delta32.astype(np.float64)
    Xt, _ = O.smacof(synth.uniform_x0(1500, seed=1), D64, 15)
    X1, _ = ctx.layout(Delta32, Xt.astype(np.float32), 1, P.FP32)
    ref = O.smacof_step(Xt.astype(np.float32).astype(np.float64), D64)
    err = np.abs(X1 - ref).max() / max(1.0, np.abs(ref).max())
    assert err <= 1e-4, err


@pytest.mark.parametrize("n", [5000, 10000])
def test_layout_fp32_one_update_bench_scale(ctx, n):
    """One FP32 update at the benchmark's sizes against the oracle's update
    (Eq. (10), pinned Cholesky solve) on the oracle's PDist of the benchmark
    graph family (Chung-Lu, mean degree 20, exponent 2.5, seed 0). At
    n = 10,000 (kp = 10,112) the L^w inverse runs its 79 pivot steps with the
    lookahead, and each persistent layout-pass CTA streams ~21 of the 3,160
    upper tiles (column runs across chunk boundaries, L2-resident and streamed
    tiles, many run slots per reduce); at n = 5,000, 40 pivots. Two updates
    are checked: from the seeded U[-1,1]^2 start (the benchmark's first
    update) and from the oracle's first update."""
    import paper_2112_14944_gb300 as P
    D32 = _pdist_for(n, 20, 0).astype(np.float32)
    D64 = D32.astype(np.float64)
    X = synth.uniform_x0(n, seed=0).astype(np.float64)
    for _ in range(2):
        Xin = X.astype(np.float32)
        Xg, _ = ctx.layout(D32, Xin, 1, P.FP32)
        ref = O.smacof_step(Xin.astype(np.float64), D64)
        err = np.abs(Xg - ref).max() / max(1.0, np.abs(ref).max())
        assert err <= 1e-4, err
        X = ref


def test_layout_fp32_trajectory_properties(ctx):
    import paper_2112_14944_gb300 as P
    n = 800
    Delta32 = _pdist_for(n, 10, 4).astype(np.float32)
    x0 = synth.uniform_x0(n, seed=4)
    prev = math.inf
    for it in (0, 1, 5, 20, 60, 150):
        X, s = ctx.layout(Delta32, x0, it, P.FP32)
        assert np.abs(X.astype(np.float64).mean(axis=0)).max() <= 1e-5 * max(1.0, np.abs(X).max())
        assert s <= prev * (1 + 1e-6)
        prev = s
    _, hist = O.smacof(x0.astype(np.float64), Delta32.astype(np.float64), 150)
    assert abs(prev - hist[-1]) <= 1e-3 * hist[-1]


def test_layout_zero_iterations_only_centres(ctx):
    import paper_2112_14944_gb300 as P
    D = O.pdist_from_z(np.full((5, 5), 0.05), 5)
    np.fill_diagonal(D, 0)
    x0 = np.array([[1, 2], [3, 4], [0, 0], [5, -1], [2, 2]], dtype=np.float64)
    X, s = ctx.layout(D, x0, 0, P.FP64)
    assert np.allclose(X, x0 - x0.mean(axis=0), atol=1e-15)
    assert abs(s - O.stress(x0, D)) <= 1e-12 * s


def test_layout_two_points_one_step(ctx):
    import paper_2112_14944_gb300 as P
    D = np.array([[0.0, 3.7], [3.7, 0.0]])
    for prec, tol in ((P.FP64, 1e-13), (P.FP32, 1e-5)):
        dt = np.float64 if prec == P.FP64 else np.float32
        X, s = ctx.layout(D.astype(dt), np.array([[0.2, -0.4], [0.9, 0.1]], dt), 1, prec)
        assert abs(np.linalg.norm(X[0].astype(np.float64) - X[1]) - 3.7) <= tol * 3.7


def test_layout_rejects_bad_pdist(ctx):
    import paper_2112_14944_gb300 as P
    from paper_2112_14944_gb300 import _binding as B
    D = np.full((4, 4), 3.0, np.float32)
    D[1, 2] = -1.0
    with pytest.raises(P.PPRVizError) as ei:
        ctx.layout(D, np.zeros((4, 2), np.float32), 3, P.FP32)
    assert ei.value.status == B.PPRVIZ_E_INVALID_ARG
    D[1, 2] = np.inf
    with pytest.raises(P.PPRVizError):
        ctx.layout(D, np.zeros((4, 2), np.float32), 3, P.FP32)


@pytest.mark.parametrize("dt,tol", [(np.float64, 1e-11), (np.float32, 2e-5)])
def test_energy_and_gradients_match_oracle(ctx, dt, tol):
    k = 300
    Delta = _pdist_for(k, 8, 7)
    X = (synth.uniform_x0(k, seed=3).astype(np.float64) * 4.0)
    X[7] = X[8]  # a coincident pair: its gradient term is 0
    e, gx, gd = ctx.energy(Delta.astype(dt), X.astype(dt), grad_scale=0.5, grad_x=True, grad_pdist=True)
    Xd, Dd = X.astype(dt).astype(np.float64), Delta.astype(dt).astype(np.float64)
    e_ref = O.stress(Xd, Dd)
    assert abs(e - e_ref) <= tol * e_ref
    g_ref = 0.5 * O.stress_grad(Xd, Dd)
    assert np.abs(gx - g_ref).max() <= tol * max(1.0, np.abs(g_ref).max()) * 10
    gd_ref = 0.5 * O.stress_grad_pdist(Xd, Dd)
    assert np.abs(gd - gd_ref).max() <= tol * max(1.0, np.abs(gd_ref).max()) * 10


def test_autograd_function_gradcheck():
    torch = pytest.importorskip("torch")
    import paper_2112_14944_gb300 as P
    c = P.Context(0, torch_stream=True)
    k = 10
    D = torch.tensor(_pdist_for(30, 4, 8)[:k, :k], device="cuda")
    X = torch.tensor(synth.uniform_x0(k, seed=5).astype(np.float64) * 3, device="cuda")
    Xr = X.clone().requires_grad_(True)
    Dr = D.clone().requires_grad_(True)
    f = lambda x, d: P.StressEnergy.apply(x, d, c)  # noqa: E731
    assert torch.autograd.gradcheck(f, (Xr, Dr), eps=1e-6, atol=1e-7, rtol=1e-6)
    c.close()


def test_gradient_finite_differences_subview_512(ctx):
    """Energy backward against central finite differences of the energy on an
    n=512 sub-view (the differentiable-layout gradient check), FP64."""
    k = 512
    D = _pdist_for(2048, 10, 5)[:k, :k].copy()
    X = synth.uniform_x0(k, seed=6).astype(np.float64) * 5
    _, gx, _ = ctx.energy(D, X, grad_x=True)
    g_ref = O.stress_grad(X, D)
    assert np.abs(gx - g_ref).max() <= 1e-10 * np.abs(g_ref).max()
    h = 1e-5
    for (i, a) in [(0, 0), (17, 1), (255, 0), (511, 1)]:
        Xp = X.copy(); Xp[i, a] += h
        Xm = X.copy(); Xm[i, a] -= h
        ep, _, _ = ctx.energy(D, Xp)
        em, _, _ = ctx.energy(D, Xm)
        fd = (ep - em) / (2 * h)
        assert abs(fd - gx[i, a]) <= 1e-5 * max(1.0, abs(gx[i, a]))


def _views_oracle(g):
    return oracle_dppr(g, ALPHA)


def _batched_update_vs_oracle(ctx, graphs, G, x0, pick, eps=1e-9):
    """One batched FP32 update of each picked view against the oracle's update
    (Eq. (10)) from the same start on the oracle's PDist of the view. The
    batch computes its own PDist; with a tight eps its certified error is
    ~1e-5 or less on all but the entries near the upper clamp, far inside the
    layout gate, so the batched update must match the oracle's within
    1e-4 * max(1, |X|_max)."""
    torch_in = not isinstance(x0, np.ndarray)
    xb1, _, _, off, cert = ctx.views_batch(G, x0, ALPHA, eps, 1, want_pdist=False, want_cert=True)
    assert np.all(cert <= eps)
    xb1 = xb1.cpu().numpy() if torch_in else xb1
    x0h = x0.cpu().numpy() if torch_in else x0
    for v in pick:
        D64 = oracle_pdist(graphs[v], ALPHA).astype(np.float32).astype(np.float64)
        ref = O.smacof_step(x0h[off[v]:off[v + 1]].astype(np.float64), D64)
        err = np.abs(xb1[off[v]:off[v + 1]] - ref).max() / max(1.0, np.abs(ref).max())
        assert err <= 1e-4, (v, graphs[v].n, err)


def test_views_batch_matches_single_views(ctx):
    """5 SBM views (50..300 nodes): every view's batched PDist passes the
    certified oracle gate with its own certificates, and so does the
    single-view PDist; one batched update equals the single-view update of
    the same PDist up to FP32 summation order, and after 40 updates the final
    stresses agree."""
    import paper_2112_14944_gb300 as P
    graphs = synth.sbm_views(5, seed=3, n_min=50, n_max=300)
    G = [ctx.upload_graph(g) for g in graphs]
    x0 = np.concatenate([synth.uniform_x0(g.n, seed=10 + i) for i, g in enumerate(graphs)])
    xb, pdb, stress, off, cert = ctx.views_batch(G, x0, ALPHA, 1e-6, 40, want_pdist=True, want_cert=True)
    assert np.all(cert <= 1e-6)
    assert ctx.stats()["graph_launched"] == 1  # the 40 updates ran as one CUDA graph
    sq = 0
    for v, g in enumerate(graphs):
        n = g.n
        Dref = _views_oracle(g)
        Pd = pdb[sq:sq + n * n].reshape(n, n)
        check_pdist(Pd, Dref, cert[off[v]:off[v + 1]], n)
        _, Pd1, cert1, _ = ctx.dppr(G[v], np.arange(n, dtype=np.int32), ALPHA, 1e-6, P.FP32)
        check_pdist(Pd1, Dref, cert1, n)
        X1, s1 = ctx.layout(Pd.copy(), x0[off[v]:off[v + 1]].copy(), 40, P.FP32)
        _same_trajectory(X1, xb[off[v]:off[v + 1]], s1, stress[v])
        sq += n * n
    # one update: only the summation order differs
    xb1, _, stress1, _ = ctx.views_batch(G, x0, ALPHA, 1e-6, 1, want_pdist=False)
    sq = 0
    for v, g in enumerate(graphs):
        n = g.n
        X1, s1 = ctx.layout(pdb[sq:sq + n * n].reshape(n, n).copy(), x0[off[v]:off[v + 1]].copy(), 1, P.FP32)
        _same_layout(X1, xb1[off[v]:off[v + 1]], s1, stress1[v], 1e-5)
        sq += n * n
    # against the oracle: one update of every view, and after 40 updates the
    # final stress (the trajectory gate of the FP32 layout)
    _batched_update_vs_oracle(ctx, graphs, G, x0, range(len(graphs)))
    xt, _, st_t, _ = ctx.views_batch(G, x0, ALPHA, 1e-9, 40, want_pdist=False)
    for v, g in enumerate(graphs):
        D64 = oracle_pdist(g, ALPHA).astype(np.float32).astype(np.float64)
        _, hist = O.smacof(x0[off[v]:off[v + 1]].astype(np.float64), D64, 40)
        assert abs(st_t[v] - hist[-1]) <= 1e-3 * hist[-1], (v, st_t[v], hist[-1])


def test_views_batch_profiled_runs_launches_directly(ctx):
    """With kernel timing on, the batched updates go to the stream one by one
    (no CUDA graph: a recorded graph has no stream points to time), give the
    layout of the graph launch (up to the rounding of the propagation's
    reductions), and every timing event pair is readable."""
    graphs = synth.sbm_views(4, seed=5, n_min=60, n_max=200)
    G = [ctx.upload_graph(g) for g in graphs]
    x0 = np.concatenate([synth.uniform_x0(g.n, seed=20 + i) for i, g in enumerate(graphs)])
    ctx.views_batch(G, x0, ALPHA, 1e-6, 12, want_pdist=False)  # settles the tuned wave widths
    xg, _, sg, _, _ = ctx.views_batch(G, x0, ALPHA, 1e-6, 12, want_pdist=False, want_cert=True)
    assert ctx.stats()["graph_launched"] == 1
    ctx.profile(1)
    try:
        xp, _, sp, _, _ = ctx.views_batch(G, x0, ALPHA, 1e-6, 12, want_pdist=False, want_cert=True)
        assert ctx.stats()["graph_launched"] == 0
        kt = ctx.kernel_times()
    finally:
        ctx.profile(0)
    np.testing.assert_allclose(xp, xg, rtol=0, atol=1e-4 * max(1.0, np.abs(xg).max()))
    np.testing.assert_allclose(sp, sg, rtol=1e-4)
    assert sum(t for _, _, t in kt.values()) > 0
    assert all(t <= c for _, c, t in kt.values())


def test_views_batch_waves_edge_cases(ctx):
    """Batched propagation over views that exercise the wave plan: single
    nodes, a single edge, a star, many small SBM views sharing one wave, and
    a 3,000-node view whose sources take two groups. Each view's PDist passes
    the certified oracle gate; the closed forms of the single edge and the
    star hold."""
    import math
    from synth import Graph
    small = synth.sbm_views(40, seed=11, n_min=2, n_max=60)
    big = synth.sbm([750] * 4, 0.1, 0.002, seed=12)

    def csr(n, edges):
        rows = [[] for _ in range(n)]
        for a, b in edges:
            rows[a].append(b)
            rows[b].append(a)
        rp = np.zeros(n + 1, dtype=np.int64)
        for i, r in enumerate(rows):
            rp[i + 1] = rp[i] + len(r)
        col = np.array([c for r in rows for c in sorted(r)], dtype=np.int32)
        return Graph(n, rp, col, None)

    single = csr(1, [])
    edge = csr(2, [(0, 1)])
    star = csr(6, [(0, i) for i in range(1, 6)])
    graphs = [single, big, edge] + small + [star, csr(3, [])]
    G = [ctx.upload_graph(g) for g in graphs]
    x0 = np.concatenate([synth.uniform_x0(g.n, seed=300 + i) for i, g in enumerate(graphs)])
    xb, pdb, stress, off, cert = ctx.views_batch(G, x0, ALPHA, 1e-6, 5, want_pdist=True, want_cert=True)
    assert np.all(cert <= 1e-6)
    assert np.all(np.isfinite(xb))
    sq = np.concatenate([[0], np.cumsum([g.n * g.n for g in graphs])])
    for v, g in enumerate(graphs):
        n = g.n
        Pd = pdb[sq[v]:sq[v + 1]].reshape(n, n)
        check_pdist(Pd, _views_oracle(g), cert[off[v]:off[v + 1]], n)
    c = 1.0 - ALPHA
    # single edge: pi_d(a, b) = c / (1 + c), PDist clamped at 2 ln 2 < 2
    Pe = pdb[sq[2]:sq[3]].reshape(2, 2)
    assert abs(Pe[0, 1] - min(max(1.0 - math.log(2 * c / (1 + c)), 2.0), 2.0 * math.log(2.0))) <= 1e-5
    # star with 5 leaves (n = 6): leaf-leaf PDist from pi_d = c^2 / (L (1 + c))
    vs = len(graphs) - 2
    Ps = pdb[sq[vs]:sq[vs + 1]].reshape(6, 6)
    z = 2 * c * c / (5 * (1 + c))
    assert abs(Ps[1, 2] - min(max(1.0 - math.log(z), 2.0), 2.0 * math.log(6.0))) <= 1e-5


def test_views_batch_sbm_sample_of_the_batched_workload(ctx):
    """16 SBM views (sizes 50..1500, 4..16 blocks, p_in 0.1, p_out 0.002): the
    batched workload at reduced size. Every certificate is within eps; sampled
    views' batched PDists match the oracle under the certified gate; every
    view's final stress after 200 updates agrees with a single-view run's on
    the same PDist, and one update agrees up to FP32 summation order."""
    import paper_2112_14944_gb300 as P
    graphs = synth.sbm_views(16, seed=5, n_min=50, n_max=1500)
    G = [ctx.upload_graph(g) for g in graphs]
    x0 = np.concatenate([synth.uniform_x0(g.n, seed=100 + i) for i, g in enumerate(graphs)])
    xb, pdb, stress, off, cert = ctx.views_batch(G, x0, ALPHA, 1e-6, 200, want_pdist=True, want_cert=True)
    assert np.all(cert <= 1e-6)
    sq = np.concatenate([[0], np.cumsum([g.n * g.n for g in graphs])])
    big = int(np.argmax([g.n for g in graphs]))
    for v in sorted({0, big, len(graphs) - 1}):
        g, n = graphs[v], graphs[v].n
        Pd = pdb[sq[v]:sq[v + 1]].reshape(n, n)
        check_pdist(Pd, _views_oracle(g), cert[off[v]:off[v + 1]], n)
    for v, g in enumerate(graphs):
        X1, s1 = ctx.layout(pdb[sq[v]:sq[v + 1]].reshape(g.n, g.n).copy(), x0[off[v]:off[v + 1]].copy(), 200, P.FP32)
        _same_trajectory(X1, xb[off[v]:off[v + 1]], s1, stress[v])
    # one update: the same update up to summation order
    xb1, _, stress1, _ = ctx.views_batch(G, x0, ALPHA, 1e-6, 1, want_pdist=False)
    for v, g in enumerate(graphs):
        X1, s1 = ctx.layout(pdb[sq[v]:sq[v + 1]].reshape(g.n, g.n).copy(), x0[off[v]:off[v + 1]].copy(), 1, P.FP32)
        _same_layout(X1, xb1[off[v]:off[v + 1]], s1, stress1[v], 1e-5)
    _batched_update_vs_oracle(ctx, graphs, G, x0, sorted({0, big, len(graphs) - 1}))


def test_views_batch_full_size_sbm_workload_sampled(ctx):
    """The batched-views workload at full size: 256 SBM views, n_v ~ U{50..5000},
    4..16 blocks, p_in 0.1, p_out 0.002 (seed 0), DPPR, PDist and 200 FP32
    layout updates of every view in one call on device buffers. Every
    certificate is within eps and every layout is finite and centred; for
    sampled views (the smallest, the largest and two more) the batched PDist
    matches the oracle's direct solve under the certified gate, one batched
    update equals the single-view update on the same PDist up to FP32
    summation order, and after 200 updates the final stresses agree."""
    torch = pytest.importorskip("torch")
    import paper_2112_14944_gb300 as P
    graphs = synth.sbm_views(256, seed=0)
    G = [ctx.upload_graph(g) for g in graphs]
    x0 = np.concatenate([synth.uniform_x0(g.n, seed=1000 + i) for i, g in enumerate(graphs)])
    xb_d, pd_d, stress, off, cert = ctx.views_batch(G, torch.from_numpy(x0).cuda(), ALPHA, 1e-6, 200,
                                                    want_pdist=True, want_cert=True)
    xb = xb_d.cpu().numpy()
    assert np.all(cert <= 1e-6)
    assert np.all(np.isfinite(xb)) and np.all(np.isfinite(stress)) and np.all(stress > 0)
    for v in range(len(graphs)):
        assert np.abs(xb[off[v]:off[v + 1]].astype(np.float64).mean(0)).max() <= 1e-3
    sizes = np.array([g.n for g in graphs])
    sq = np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 2)])
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 200})
    xb1_d, _, stress1, _ = ctx.views_batch(G, torch.from_numpy(x0).cuda(), ALPHA, 1e-6, 1, want_pdist=False)
    xb1 = xb1_d.cpu().numpy()
    for v in pick:
        g, n = graphs[v], graphs[v].n
        Pd = pd_d[int(sq[v]):int(sq[v + 1])].cpu().numpy().reshape(n, n)
        check_pdist(Pd, _views_oracle(g), cert[off[v]:off[v + 1]], n)
        X1, s1 = ctx.layout(Pd, x0[off[v]:off[v + 1]].copy(), 200, P.FP32)
        _same_trajectory(X1, xb[off[v]:off[v + 1]], s1, stress[v])
        X1, s1 = ctx.layout(Pd, x0[off[v]:off[v + 1]].copy(), 1, P.FP32)
        _same_layout(X1, xb1[off[v]:off[v + 1]], s1, stress1[v], 1e-5)
    # one batched update of the sampled views against the oracle's update
    _batched_update_vs_oracle(ctx, graphs, G, torch.from_numpy(x0).cuda(), pick)
