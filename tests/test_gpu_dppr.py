"""GPU parity of graph ingest (P0), propagation + certificate (P1/P2) and
DPPR/PDist (P3) against the FP64 oracle, through the C ABI.

Tolerances (derived in the design notes from the paper's definitions):
  DPPR:  |got - ref| <= 1e-6 * max(1, |ref|) per entry; certificate <= eps.
  PDist: 1e-5 plus the certified propagation bound of Eq. (1) (tests/_parity.py);
         with a tight eps the flat 1e-5 gate holds everywhere.
  Degrees and other integer outputs: bit-exact.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth
from _parity import check_dppr, check_pdist

pytestmark = pytest.mark.gpu
ALPHA = 0.15
EPS = 1e-6


@pytest.fixture(scope="module")
def ctx():
    import paper_2112_14944_gb300 as P
    c = P.Context(0)
    yield c
    c.close()


def _oracle(g, view, alpha=ALPHA, direct=False):
    Pm = O.transition_matrix(g.n, g.row_ptr, g.col, g.weight)
    d = O.degrees(g.n, g.row_ptr, g.col, g.weight)
    view = np.asarray(view)
    if direct:
        rows = O.ppr_direct(Pm, alpha)[view]
    else:
        rows = O.ppr_rows(Pm, view, alpha)
    D = O.dppr_rows(rows, d, view)[:, view]
    return D, d


_check_dppr = check_dppr


def _check_pdist_flat(got, ref, tol=1e-5):
    err = np.abs(got.astype(np.float64) - ref)
    assert err.max() <= tol, f"max PDist error {err.max():.3e}"
    return err.max()


def _graphs():
    return {
        "chung_lu_400": synth.chung_lu(400, 10, 2.5, seed=11),
        "sbm_isolated": synth.sbm([40, 50, 60, 3, 1], 0.12, 0.01, seed=3),
        "weighted_dense": synth.dense_clustered(240, blocks=4, density=0.15, seed=5),
    }


# ---------------------------------------------------------------- P0
def test_degrees_bit_exact(ctx):
    for name, g in _graphs().items():
        G = ctx.upload_graph(g)
        deg, n, nnz, m = G.degrees()
        assert n == g.n and nnz == g.nnz
        ref = np.zeros(g.n)
        for v in range(g.n):  # d(v) summed in row order, the definition the kernel follows
            s = 0.0
            lo, hi = g.row_ptr[v], g.row_ptr[v + 1]
            if g.weight is None:
                s = float(hi - lo)
            else:
                for x in g.weight[lo:hi]:
                    s += float(x)
            ref[v] = s
        assert np.array_equal(deg, ref), name
        assert m == sum(ref.tolist())  # m = sum_v d(v), in node order


def _bad(ctx, n, rp, col, w=None, flags=None):
    import paper_2112_14944_gb300 as P
    from paper_2112_14944_gb300 import _binding as B
    f = B.PPRVIZ_UNDIRECTED | B.PPRVIZ_VALIDATE if flags is None else flags
    with pytest.raises(P.PPRVizError) as ei:
        B.pprviz_graph_upload(ctx.h, n, np.asarray(rp, np.int64), np.asarray(col, np.int32),
                              None if w is None else np.asarray(w, np.float32), f)
    return ei.value.status


def test_graph_validation_rejects_bad_csr(ctx):
    from paper_2112_14944_gb300 import _binding as B
    assert _bad(ctx, 2, [0, 1, 2], [1, 1]) == B.PPRVIZ_E_BAD_GRAPH          # asymmetric (1->1 self-loop too)
    assert _bad(ctx, 3, [0, 2, 3, 4], [2, 1, 0, 0]) == B.PPRVIZ_E_BAD_GRAPH  # unsorted row 0
    assert _bad(ctx, 2, [0, 1, 2], [5, 0]) == B.PPRVIZ_E_BAD_GRAPH          # column out of range
    assert _bad(ctx, 2, [0, 1, 2], [0, 1]) == B.PPRVIZ_E_BAD_GRAPH          # self-loops
    assert _bad(ctx, 2, [0, 1, 2], [1, 0], w=[1.0, -2.0]) == B.PPRVIZ_E_BAD_GRAPH  # negative weight
    assert _bad(ctx, 2, [0, 1, 2], [1, 0], w=[1.0, 2.0]) == B.PPRVIZ_E_BAD_GRAPH   # asymmetric weight
    assert _bad(ctx, 2, [0, 2, 1], [1, 0]) == B.PPRVIZ_E_BAD_GRAPH          # decreasing row_ptr
    assert _bad(ctx, 3, [0, 1, 1, 2], [2, 1]) == B.PPRVIZ_E_BAD_GRAPH       # 0->2 without 2->0
    assert _bad(ctx, 2, [0, 1, 1], [0], flags=B.PPRVIZ_VALIDATE) == B.PPRVIZ_E_BAD_GRAPH  # self-loop (directed)
    assert _bad(ctx, 2, [0, 2, 2], [1, 1], flags=B.PPRVIZ_VALIDATE) == B.PPRVIZ_E_BAD_GRAPH  # duplicate (directed)
    assert _bad(ctx, 0, [0], []) == B.PPRVIZ_E_INVALID_ARG


def test_view_and_scalar_errors(ctx):
    import paper_2112_14944_gb300 as P
    from paper_2112_14944_gb300 import _binding as B
    g = synth.chung_lu(50, 5, 2.5, seed=1)
    G = ctx.upload_graph(g)
    for view, kw in [
        (np.array([1, 2, 1], np.int32), {}),           # duplicate id
        (np.array([1, 60], np.int32), {}),             # out of range
        (np.array([-1], np.int32), {}),
        (np.array([1, 2], np.int32), {"alpha": 0.0}),
        (np.array([1, 2], np.int32), {"alpha": 1.0}),
        (np.array([1, 2], np.int32), {"eps": 0.0}),
        (np.array([1, 2], np.int32), {"precision": 7}),
        (np.array([1, 2], np.int32), {"n_clamp": 1}),
    ]:
        with pytest.raises(P.PPRVizError) as ei:
            ctx.dppr(G, view, **kw)
        assert ei.value.status == B.PPRVIZ_E_INVALID_ARG


# ---------------------------------------------------------------- P1-P3
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dppr_pdist_small_graphs(ctx, precision):
    import paper_2112_14944_gb300 as P
    prec = P.FP64 if precision == "fp64" else P.FP32
    for name, g in _graphs().items():
        G = ctx.upload_graph(g)
        for view in [np.arange(g.n, dtype=np.int32), synth.sample_view(g.n, g.n // 3, seed=2)]:
            Dref, _ = _oracle(g, view, direct=True)
            D, Delta, cert, st = ctx.dppr(G, view, ALPHA, EPS, prec)
            assert st == 0, name
            assert cert.max() <= EPS
            _check_dppr(D, Dref)
            check_pdist(Delta, Dref, cert, g.n)


def test_dppr_fp64_outputs_and_closed_forms(ctx):
    import paper_2112_14944_gb300 as P
    C = 1 - ALPHA
    # star: centre 0 with 9 leaves (closed forms pinned in the oracle tests)
    n = 10
    rp = np.array([0, 9] + list(range(10, 19)), dtype=np.int64)
    col = np.array(list(range(1, 10)) + [0] * 9, dtype=np.int32)
    G = ctx.upload(n, rp, col)
    D, Delta, cert, _ = ctx.dppr(G, np.arange(n, dtype=np.int32), ALPHA, 1e-12, P.FP64, out64=True)
    assert D.dtype == np.float64
    assert abs(D[0, 3] - C / (1 + C)) < 1e-12 and abs(D[3, 0] - C / (1 + C)) < 1e-12
    assert abs(D[2, 5] - C * C / (9 * (1 + C))) < 1e-12
    assert abs(Delta[2, 5] - (1 - math.log(2 * C * C / (9 * (1 + C))))) < 1e-11
    assert Delta[0, 4] == 2.0 and np.all(np.diag(Delta) == 0)
    assert cert.max() <= 1e-12


def test_degenerate_views(ctx):
    import paper_2112_14944_gb300 as P
    # one isolated node: DPPR row 0, PDist 0
    G = ctx.upload(1, np.array([0, 0], np.int64), np.zeros(0, np.int32))
    for prec in (P.FP64, P.FP32):
        D, Delta, cert, st = ctx.dppr(G, np.array([0], np.int32), ALPHA, EPS, prec, n_clamp=2)
        assert st == 0 and D[0, 0] == 0 and Delta[0, 0] == 0 and cert[0] == 0
    # single edge: pi(a,a) = 1/(1+c), pi_d(a,b) = c/(1+c); view of one node
    C = 1 - ALPHA
    G = ctx.upload(2, np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32))
    for prec in (P.FP64, P.FP32):
        D, Delta, _, _ = ctx.dppr(G, np.array([1, 0], np.int32), ALPHA, EPS, prec)
        assert abs(D[0, 1] - C / (1 + C)) < 1e-6 and abs(D[0, 0] - 1 / (1 + C)) < 1e-6
        D1, _, _, _ = ctx.dppr(G, np.array([1], np.int32), ALPHA, EPS, prec)
        assert D1.shape == (1, 1) and abs(D1[0, 0] - 1 / (1 + C)) < 1e-6


def test_isolated_nodes_pdist_upper_clamp(ctx):
    import paper_2112_14944_gb300 as P
    # p_out = 0: two disconnected 30-node blocks plus two isolated nodes
    g = synth.sbm([30, 30, 1, 1], 0.3, 0.0, seed=9)
    assert g.row_ptr[60] == g.row_ptr[62]
    G = ctx.upload_graph(g)
    view = np.arange(g.n, dtype=np.int32)
    for prec in (P.FP64, P.FP32):
        D, Delta, _, _ = ctx.dppr(G, view, ALPHA, EPS, prec, n_clamp=1000)
        for iso in (60, 61):
            assert np.all(D[iso] == 0)
            others = [j for j in range(g.n) if j != iso]
            assert np.allclose(Delta[iso, others], 2 * math.log(1000), atol=1e-6, rtol=0)
        # no walk crosses between the two blocks: z = 0, the upper clamp
        assert np.all(D[:30, 30:60] == 0)
        assert np.allclose(Delta[:30, 30:60], 2 * math.log(1000), atol=1e-6, rtol=0)


def test_config_small_chung_lu_1000_fp64(ctx):
    """Chung-Lu n=1,000, mean degree 10, exponent 2.5, seed 0, alpha 0.15, eps 1e-6, FP64."""
    import paper_2112_14944_gb300 as P
    g = synth.chung_lu(1000, 10, 2.5, seed=0)
    G = ctx.upload_graph(g)
    view = np.arange(g.n, dtype=np.int32)
    Dref, _ = _oracle(g, view, direct=True)
    D, Delta, cert, st = ctx.dppr(G, view, ALPHA, EPS, P.FP64, out64=True)
    assert st == 0 and cert.max() <= EPS
    assert np.abs(D - Dref).max() <= EPS  # the FP64 path meets eps absolutely
    check_pdist(Delta, Dref, cert, g.n, slack=1e-6)


def test_fp32_multiple_groups_ragged_tail(ctx):
    """n = 3,000: the FP32 path splits the sources into groups with a ragged last group."""
    import paper_2112_14944_gb300 as P
    g = synth.chung_lu(3000, 10, 2.5, seed=6)
    G = ctx.upload_graph(g)
    view = np.arange(g.n, dtype=np.int32)
    Dref, _ = _oracle(g, view, direct=True)
    D, Delta, cert, st = ctx.dppr(G, view, ALPHA, EPS, P.FP32)
    stats = ctx.stats()
    assert stats["groups"] >= 2 and g.n % stats["source_group"] != 0
    assert st == 0 and cert.max() <= EPS
    _check_dppr(D, Dref)
    check_pdist(Delta, Dref, cert, g.n)


def test_tight_eps_gives_flat_pdist_gate(ctx):
    """With a tight eps the certified PDist bound falls below 1e-5 for every
    entry above the clamp threshold, so the flat 1e-5 gate holds. The FP32
    path refines on the renormalised x_hi + x_lo pair (certifiable to about
    d_max * 1e-13); the FP64 path reaches 1e-12 directly."""
    import paper_2112_14944_gb300 as P
    for g in (synth.sbm([40, 50, 60, 7], 0.1, 0.004, seed=12), synth.chung_lu(500, 10, 2.5, seed=13)):
        G = ctx.upload_graph(g)
        view = np.arange(g.n, dtype=np.int32)
        Dref, _ = _oracle(g, view, direct=True)
        for prec, eps in ((P.FP32, 1e-11), (P.FP64, 1e-12)):
            D, Delta, cert, st = ctx.dppr(G, view, ALPHA, eps, prec)
            assert st == 0 and cert.max() <= eps
            _check_dppr(D, Dref, tol=2e-7)
            _check_pdist_flat(Delta, O.pdist_from_dppr(Dref, g.n), tol=1e-5)


def test_full_size_chung_lu_10k_fp32_sampled(ctx):
    """Chung-Lu n=10,000, mean degree 20: all-pairs FP32 DPPR/PDist as timed by
    the benchmark; sampled rows checked against the oracle's power iteration,
    every certificate checked, and DPPR symmetry (reversibility) at full size."""
    import paper_2112_14944_gb300 as P
    g = synth.chung_lu(10000, 20, 2.5, seed=0)
    G = ctx.upload_graph(g)
    view = np.arange(g.n, dtype=np.int32)
    D, Delta, cert, st = ctx.dppr(G, view, ALPHA, EPS, P.FP32)
    assert st == 0 and cert.max() <= EPS
    sample = np.array([0, 1, 7, 99, 1234, 5000, 9998, 9999])
    Pm = O.transition_matrix(g.n, g.row_ptr, g.col)
    d = O.degrees(g.n, g.row_ptr, g.col)
    rows = O.ppr_rows(Pm, sample, ALPHA)          # pi(s, .)
    cols = O.ppr_cols(Pm, sample, ALPHA)          # pi(., s)
    Drow = d[sample][:, None] * rows              # pi_d(s, .)
    Dcol = (d[:, None] * cols).T                  # pi_d(., s) as rows
    _check_dppr(D[sample], Drow)
    ref = np.where(np.arange(g.n)[None, :] == sample[:, None], 0.0, O.pdist_from_z(Drow + Dcol, g.n))
    cc = cert[sample][:, None] + cert[None, :]
    tol = 1e-5 + cc / np.maximum(Drow + Dcol - cc, math.e / g.n ** 2)
    assert np.all(np.abs(Delta[sample].astype(np.float64) - ref) <= tol)
    asym = np.abs(D - D.T) / np.maximum(1.0, np.abs(D))
    assert asym.max() <= 2e-6


def test_pdist_standalone_matches_oracle(ctx):
    g = synth.chung_lu(300, 8, 2.5, seed=2)
    Dref, _ = _oracle(g, np.arange(g.n), direct=True)
    Dref[5, :] = 0.0
    Dref[:, 5] = 0.0                               # z = 0 entries
    for dt, tol in [(np.float32, 2e-6), (np.float64, 1e-12)]:
        Din = np.ascontiguousarray(Dref, dtype=dt)
        ref = O.pdist_from_dppr(Din.astype(np.float64), 50)
        out = ctx.pdist(Din, 50)
        assert out.dtype == dt
        _check_pdist_flat(out, ref, tol=tol)
        assert out[5, 7] == np.float64(2 * math.log(50)).astype(dt)


def test_full_size_view_of_2m_graph_sampled(ctx):
    """Chung-Lu n=2,000,000, mean degree 10, a view of 8,192 nodes drawn
    uniformly (the differentiable-layout workload): FP32 DPPR/PDist among the
    view with n_clamp = n. Sampled view rows against the oracle's power
    iteration on the whole graph (rows and columns of the sampled sources),
    every certificate, DPPR symmetry, and the stress energy and gradient of a
    layout of the whole view on sampled rows."""
    import paper_2112_14944_gb300 as P
    g = synth.chung_lu(2_000_000, 10, 2.5, seed=0)
    k = 8192
    view = synth.sample_view(g.n, k, seed=0)
    G = ctx.upload_graph(g)
    D, Delta, cert, st = ctx.dppr(G, view, ALPHA, EPS, P.FP32)
    assert st == 0 and cert.shape == (k,) and cert.max() <= EPS
    pos = np.array([0, 1, 2345, k - 1])             # sampled positions in the view
    src = view[pos]
    Pm = O.transition_matrix(g.n, g.row_ptr, g.col)
    d = O.degrees(g.n, g.row_ptr, g.col)
    rows = O.ppr_rows(Pm, src, ALPHA)               # pi(s, .) over the graph
    cols = O.ppr_cols(Pm, src, ALPHA)               # pi(., s)
    Drow = d[src][:, None] * rows[:, view]          # pi_d(s, t), t in the view
    Dcol = (d[view][:, None] * cols[view, :]).T     # pi_d(t, s) as rows
    _check_dppr(D[pos], Drow)
    z = Drow + Dcol
    ref = O.pdist_from_z(z, g.n)
    ref[np.arange(len(pos)), pos] = 0.0
    cc = cert[pos][:, None] + cert[None, :]
    tol = 1e-5 + cc / np.maximum(z - cc, math.e / float(g.n) ** 2)
    assert np.all(np.abs(Delta[pos].astype(np.float64) - ref) <= tol)
    asym = np.abs(D - D.T) / np.maximum(1.0, np.abs(D))
    assert asym.max() <= 2e-6
    # energy and gradient of a layout of the whole view (pair recomputation)
    # on a seeded symmetric target in the PDist range [2, 2 ln n] (an oracle
    # input never comes from the GPU)
    r = synth.uniform(7, 21, np.arange(k * k, dtype=np.uint64)).reshape(k, k)
    Dsyn = (2.0 + (2.0 * math.log(g.n) - 2.0) * (r + r.T) / 2.0).astype(np.float32)
    np.fill_diagonal(Dsyn, 0.0)
    del r
    X = synth.uniform_x0(k, seed=0) * 8.0
    e, gx, _ = ctx.energy(Dsyn, X, grad_scale=1.0, grad_x=True)
    Dd, Xd = Dsyn.astype(np.float64), X.astype(np.float64)
    e_ref = O.stress(Xd, Dd)
    assert abs(e - e_ref) <= 2e-5 * e_ref
    g_ref = O.stress_grad(Xd, Dd)[pos]
    assert np.abs(gx[pos] - g_ref).max() <= 2e-4 * max(1.0, np.abs(g_ref).max())


def test_frontier_profile_matches_oracle_power_iteration(ctx):
    """The frontier diagnostic (Algorithm 2's threshold) against the oracle's
    power iteration: after sweep t the push residue of node v for source s is
    r = d(s) (x_{t+1} - x_t)_v / alpha, active when r > d(v) eps / max_view d.
    The counts are integers decided by FP64 comparisons on both sides, which
    sum in different orders, so entries within rounding of the threshold may
    differ: a 0.5 % + 3 slack."""
    g = synth.chung_lu(600, 8, 2.5, seed=4)
    view = synth.sample_view(g.n, 40, seed=3)
    G = ctx.upload_graph(g)
    T = 60
    act = ctx.frontier_profile(G, view, T, ALPHA, EPS)
    Pm = O.transition_matrix(g.n, g.row_ptr, g.col)
    d = O.degrees(g.n, g.row_ptr, g.col)
    rmax = EPS / d[view].max()
    B = np.zeros((len(view), g.n))
    B[np.arange(len(view)), view] = ALPHA
    PT = Pm.T.tocsr()
    X = B.copy()
    ref = []
    for _ in range(T):
        Xn = B + (1 - ALPHA) * (PT @ X.T).T
        r = d[view][:, None] * np.abs(Xn - X) / ALPHA
        ref.append(int((r > d[None, :] * rmax).sum()))
        X = Xn
    ref = np.array(ref)
    assert np.all(np.abs(act - ref) <= 0.005 * ref + 3), (act[:10], ref[:10])
    assert act[0] < act[5] and act[-1] < act.max()
