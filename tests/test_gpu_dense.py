"""GPU parity of the dense tensor-core propagation (P1d) against the FP64
oracle, through the C ABI.

The tensor-core path changes only how a sweep is computed (one dense product
of the n x n weights with the n x G state per sweep); the certificate is the
same FP64 residual over the CSR as on the sparse path, so the gates are the
sparse path's: every certificate <= eps, DPPR within 1e-6 * max(1, |ref|) of
the oracle (reading of the paper's "max-abs 1e-6" for FP32 outputs), PDist
under the certified per-entry tolerance of Lemma 1's mechanism.

The BF16 mode (PPRVIZ_FP32_BF16TC: BF16 x BF16 -> FP32 kind::f16 sweeps) is
held to the same gates: its sweeps are only BF16-accurate, and the FP64
residual with FP32 refinement restores eps.

Shapes: n = 600 (ragged against the 128-row tile and the 32-wide inner chunk,
128-source tiles), n = 1000 with k = 1000 (256-source tiles), a 300-node view
of a 900-node graph (84 padded source columns), isolated nodes (a zero row of
the weight matrix keeps its walk), and the dense clustered weighted view at
its full size n = 20,000 on sampled rows plus properties that hold at any size.
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


def _oracle_dppr(g, view):
    n = g.n
    P = O.transition_matrix(n, g.row_ptr, g.col, g.weight)
    d = O.degrees(n, g.row_ptr, g.col, g.weight)
    pi = O.ppr_rows(P, view, ALPHA)
    return O.dppr_rows(pi[:, view], d, view)


def _run(ctx, g, view, precision):
    G = ctx.upload_graph(g)
    D, Pd, cert, _ = ctx.dppr(G, view, ALPHA, EPS, precision)
    return D, Pd, cert, ctx.stats()


@pytest.mark.parametrize("n,seed", [(600, 1), (1000, 2)])
def test_tc_weighted_dense_view_matches_oracle(ctx, n, seed):
    import paper_2112_14944_gb300 as P
    g = synth.dense_clustered(n, blocks=10, density=0.15, seed=seed)
    view = np.arange(n, dtype=np.int32)
    D, Pd, cert, st = _run(ctx, g, view, P.FP32_TC)
    assert st["flops_dense"] > 0 and st["bytes_sweep"] == 0
    assert cert.max() <= EPS
    Dref = _oracle_dppr(g, view)
    check_dppr(D, Dref)
    check_pdist(Pd, Dref, cert, n)


def test_tc_unweighted_with_isolated_nodes(ctx):
    import paper_2112_14944_gb300 as P
    g = synth.sbm([400, 199, 1, 1], 0.2, 0.0, seed=3)
    n = g.n
    deg = np.diff(g.row_ptr)
    assert (deg == 0).sum() == 2
    view = np.arange(n, dtype=np.int32)
    D, Pd, cert, st = _run(ctx, g, view, P.FP32_TC)
    assert st["flops_dense"] > 0
    assert cert.max() <= EPS
    Dref = _oracle_dppr(g, view)
    check_dppr(D, Dref)
    iso = np.nonzero(deg == 0)[0]
    assert np.all(D[iso] == 0.0)
    check_pdist(Pd, Dref, cert, n)


def test_tc_view_subset_with_padded_sources(ctx):
    import paper_2112_14944_gb300 as P
    g = synth.dense_clustered(900, blocks=12, density=0.12, seed=4)
    view = synth.sample_view(900, 300, seed=4)
    D, Pd, cert, st = _run(ctx, g, view, P.FP32_TC)
    assert st["source_group"] == 384
    assert cert.max() <= EPS
    Dref = _oracle_dppr(g, view)
    check_dppr(D, Dref)
    check_pdist(Pd, Dref, cert, 900)


@pytest.mark.parametrize("n,seed", [(600, 1), (1000, 2)])
def test_bf16_weighted_dense_view_matches_oracle(ctx, n, seed):
    """BF16 x BF16 -> FP32 tensor-core sweeps (kind::f16): every sweep is only
    BF16-accurate, and the FP64 residual with FP32 refinement passes restores
    eps, so the gates are the FP32 path's: certificate <= eps, DPPR within
    1e-6 * max(1, |ref|), PDist under the certified tolerance. The BF16 solve
    needs more refinement passes than the 3xTF32 one."""
    import paper_2112_14944_gb300 as P
    g = synth.dense_clustered(n, blocks=10, density=0.15, seed=seed)
    view = np.arange(n, dtype=np.int32)
    D, Pd, cert, st = _run(ctx, g, view, P.FP32_BF16TC)
    assert st["flops_dense"] > 0 and st["bytes_sweep"] == 0
    assert cert.max() <= EPS
    assert st["refine_passes"] >= 1
    Dref = _oracle_dppr(g, view)
    check_dppr(D, Dref)
    check_pdist(Pd, Dref, cert, n)
    _, _, _, st32 = _run(ctx, g, view, P.FP32_TC)
    assert st["refine_passes"] >= st32["refine_passes"]


def test_bf16_isolated_nodes_and_padded_sources(ctx):
    import paper_2112_14944_gb300 as P
    g = synth.sbm([400, 199, 1, 1], 0.2, 0.0, seed=3)
    deg = np.diff(g.row_ptr)
    view = np.arange(g.n, dtype=np.int32)
    D, Pd, cert, _ = _run(ctx, g, view, P.FP32_BF16TC)
    assert cert.max() <= EPS
    Dref = _oracle_dppr(g, view)
    check_dppr(D, Dref)
    assert np.all(D[np.nonzero(deg == 0)[0]] == 0.0)
    check_pdist(Pd, Dref, cert, g.n)
    g = synth.dense_clustered(900, blocks=12, density=0.12, seed=4)
    view = synth.sample_view(900, 300, seed=4)
    D, Pd, cert, st = _run(ctx, g, view, P.FP32_BF16TC)
    assert st["source_group"] == 384 and cert.max() <= EPS
    Dref = _oracle_dppr(g, view)
    check_dppr(D, Dref)
    check_pdist(Pd, Dref, cert, 900)


def test_sweep_kernel_selection_and_agreement(ctx):
    """PPRVIZ_FP32 takes the tensor-core sweeps on a dense view and the CSR
    sweeps on a sparse one; forced CSR and forced tensor-core runs of the same
    dense view agree within the sum of their certificates."""
    import paper_2112_14944_gb300 as P
    g = synth.dense_clustered(700, blocks=7, density=0.15, seed=5)
    view = np.arange(700, dtype=np.int32)
    Da, _, ca, sa = _run(ctx, g, view, P.FP32)
    assert sa["flops_dense"] > 0
    Dc, _, cc, sc = _run(ctx, g, view, P.FP32_CSR)
    assert sc["flops_dense"] == 0 and sc["bytes_sweep"] > 0
    tol = ca[:, None] + cc[:, None] + 2e-7 * np.maximum(1.0, np.abs(Dc))
    assert np.all(np.abs(Da.astype(np.float64) - Dc) <= tol)
    gs = synth.chung_lu(1000, 10, 2.5, seed=0)
    _, _, _, ss = _run(ctx, gs, np.arange(1000, dtype=np.int32), P.FP32)
    assert ss["flops_dense"] == 0


def test_tc_full_size_dense_weighted_view_sampled(ctx):
    """The dense clustered weighted view at full size: n = 20,000, 20 blocks,
    15 % density, lognormal(0, 1) weights, all nodes as the view, automatic
    kernel choice (the bench's launch configuration). Sampled rows against the
    oracle; on the whole output: certificates, the symmetry of DPPR
    (pi_d(s, t) = pi_d(t, s) on undirected graphs, Theorem 1's premise) within
    the certificates, and the row sums sum_t pi(s, t) = 1."""
    import paper_2112_14944_gb300 as P
    n = 20000
    g = synth.dense_clustered(n, blocks=20, density=0.15, seed=0)
    view = np.arange(n, dtype=np.int32)
    D, _, cert, st = _run(ctx, g, view, P.FP32)
    assert st["flops_dense"] > 0
    assert cert.max() <= EPS
    d = O.degrees(n, g.row_ptr, g.col, g.weight)
    # symmetry within the two rows' certificates plus FP32 output rounding
    for r0 in range(0, n, 2000):
        blk = D[r0:r0 + 2000].astype(np.float64)
        other = D[:, r0:r0 + 2000].T.astype(np.float64)
        tol = cert[r0:r0 + 2000, None] + cert[None, :] + 2e-7 * np.maximum(1.0, np.abs(blk))
        assert np.all(np.abs(blk - other) <= tol)
    # sum_t pi(s, t) = 1, and the certificate bounds the whole error row:
    # ||x - pi||_1 <= ||res||_1 / alpha = cert / d(s)
    rows = D.sum(axis=1, dtype=np.float64) / d
    assert np.all(np.abs(rows - 1.0) <= cert / d + 1e-6)
    sample = np.array([0, 12345], dtype=np.int64)
    P_ = O.transition_matrix(n, g.row_ptr, g.col, g.weight)
    pi = O.ppr_rows(P_, sample, ALPHA)
    Dref = O.dppr_rows(pi, d, sample)
    check_dppr(D[sample], Dref)
    # the same view on BF16 tensor-core sweeps with refinement
    Db, _, certb, stb = _run(ctx, g, view, P.FP32_BF16TC)
    assert stb["flops_dense"] > 0 and certb.max() <= EPS
    check_dppr(Db[sample], Dref)
    rows = Db.sum(axis=1, dtype=np.float64) / d
    assert np.all(np.abs(rows - 1.0) <= certb / d + 1e-6)
