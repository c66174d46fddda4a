"""GPU parity on directed graphs (Sec. 2.1's general setting) against the FP64
oracle, through the C ABI.

The walk steps along out-edges, d(v) is the out-degree (out-strength when
weighted) and a dangling node keeps its walk (reading 2). The library gathers
over an in-neighbour CSR it builds at upload; its FP32 path runs power sweeps
(a directed walk's spectrum is complex) with the same FP64 certificate and
refinement. Gates as for undirected graphs: certificate <= eps, DPPR within
1e-6 * max(1, |ref|), PDist under the certified tolerance.
"""
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


def _oracle(g, view):
    Pm = O.transition_matrix(g.n, g.row_ptr, g.col, g.weight)
    d = O.degrees(g.n, g.row_ptr, g.col, g.weight)
    view = np.asarray(view)
    return O.dppr_rows(O.ppr_direct(Pm, ALPHA)[view], d, view)[:, view]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_directed_dppr_pdist_matches_oracle(ctx, precision):
    import paper_2112_14944_gb300 as P
    prec = P.FP64 if precision == "fp64" else P.FP32
    graphs = [synth.directed_from(synth.chung_lu(500, 10, 2.5, seed=5), seed=6),
              synth.directed_from(synth.dense_clustered(240, blocks=4, density=0.15, seed=5), seed=7)]
    for g in graphs:
        G = ctx.upload_graph(g)
        deg, n, nnz, m = G.degrees()
        assert nnz == g.nnz and np.array_equal(deg > 0, np.diff(g.row_ptr) > 0)
        for view in (np.arange(g.n, dtype=np.int32), synth.sample_view(g.n, g.n // 3, seed=2)):
            Dref = _oracle(g, view)
            D, Delta, cert, st = ctx.dppr(G, view, ALPHA, EPS, prec)
            assert st == 0 and cert.max() <= EPS
            check_dppr(D, Dref)
            check_pdist(Delta, Dref, cert, g.n)
        dangling = np.nonzero(np.diff(g.row_ptr) == 0)[0]
        assert len(dangling) > 0
        D, _, _, _ = ctx.dppr(G, np.arange(g.n, dtype=np.int32), ALPHA, EPS, prec)
        assert np.all(D[dangling] == 0.0)


def test_directed_hubs_split_rows_and_level_dppr(ctx):
    """A directed power-law graph large enough for split hub rows (in-degree
    above 4x the mean), FP32 sampled rows against the oracle, and the level-l
    DPPR of SBM-like blocks on a directed SBM."""
    import paper_2112_14944_gb300 as P
    g = synth.directed_from(synth.chung_lu(4000, 20, 2.5, seed=1), p_both=0.5, seed=3)
    G = ctx.upload_graph(g)
    view = np.arange(g.n, dtype=np.int32)
    D, _, cert, st = ctx.dppr(G, view, ALPHA, EPS, P.FP32)
    assert st == 0 and cert.max() <= EPS
    sample = np.array([0, 1, 50, 1999, 3999])
    Pm = O.transition_matrix(g.n, g.row_ptr, g.col)
    d = O.degrees(g.n, g.row_ptr, g.col)
    ref = O.dppr_rows(O.ppr_rows(Pm, sample, ALPHA), d, sample)
    check_dppr(D[sample], ref)
    gs = synth.directed_from(synth.sbm([60, 80, 70], 0.12, 0.01, seed=2), seed=5)
    Gs = ctx.upload_graph(gs)
    sets = [np.arange(0, 60, dtype=np.int32), np.arange(60, 140, dtype=np.int32), np.arange(140, 210, dtype=np.int32)]
    L, Pl, certl, stl = ctx.level_dppr(Gs, sets, ALPHA, EPS)
    assert stl == 0 and certl.max() <= EPS
    Pm = O.transition_matrix(gs.n, gs.row_ptr, gs.col)
    Dfull = O.dppr_rows(O.ppr_direct(Pm, ALPHA), O.degrees(gs.n, gs.row_ptr, gs.col), np.arange(gs.n))
    ref = O.level_dppr(Dfull, sets)
    check_dppr(L, ref)
    check_pdist(Pl, ref, certl, gs.n)


def test_directed_rejections(ctx):
    import paper_2112_14944_gb300 as P
    from paper_2112_14944_gb300 import _binding as B
    g = synth.directed_from(synth.dense_clustered(600, blocks=6, density=0.15, seed=1), seed=1)
    G = ctx.upload_graph(g)
    view = np.arange(g.n, dtype=np.int32)
    for prec in (P.FP32_TC, P.FP32_BF16TC):
        with pytest.raises(P.PPRVizError) as ei:
            ctx.dppr(G, view, ALPHA, EPS, prec)
        assert ei.value.status == B.PPRVIZ_E_INVALID_ARG
    # the automatic choice takes the CSR sweeps on a dense directed graph
    D, _, cert, st = ctx.dppr(G, view, ALPHA, EPS, P.FP32)
    assert st == 0 and cert.max() <= EPS and ctx.stats()["flops_dense"] == 0
    with pytest.raises(P.PPRVizError) as ei:
        ctx.views_batch([G], synth.uniform_x0(g.n, seed=1), ALPHA, EPS, 1)
    assert ei.value.status == B.PPRVIZ_E_INVALID_ARG
    # an asymmetric CSR flagged undirected is still a bad graph
    with pytest.raises(P.PPRVizError) as ei:
        ctx.upload(3, np.array([0, 1, 1, 2], np.int64), np.array([2, 1], np.int32))
    assert ei.value.status == B.PPRVIZ_E_BAD_GRAPH
