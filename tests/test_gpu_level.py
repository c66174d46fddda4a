"""GPU parity of the level-l DPPR between supernodes (Sec. 3.2, Definition 2,
Eq. (2)) against the FP64 oracle, through the C ABI (pprviz_level_dppr).

The oracle averages its full DPPR matrix over the leaf sets, the literal
definition; the GPU propagates once per supernode from the group start
alpha d(s) / |F(V_i)| and averages over the target leaf sets. Gates: every
certificate <= eps; level DPPR within 1e-6 * max(1, |ref|) (the DPPR gate);
level PDist under the certified tolerance of Eq. (1). Singleton leaf sets
reduce to pprviz_dppr's DPPR.
"""
import numpy as np
import pytest

import oracle as O
import synth
from _parity import check_dppr, check_pdist, oracle_dppr

pytestmark = pytest.mark.gpu
ALPHA = 0.15
EPS = 1e-6


@pytest.fixture(scope="module")
def ctx():
    import paper_2112_14944_gb300 as P
    c = P.Context(0)
    yield c
    c.close()


def _sbm_blocks(sizes):
    out, a = [], 0
    for s in sizes:
        out.append(np.arange(a, a + s, dtype=np.int32))
        a += s
    return out


def test_level_dppr_sbm_blocks_as_supernodes(ctx):
    """SBM blocks (and two isolated nodes) as the level-l supernodes."""
    sizes = [60, 80, 45, 100, 70, 1, 1]
    g = synth.sbm(sizes, 0.12, 0.01, seed=7)
    sets = _sbm_blocks(sizes)
    G = ctx.upload_graph(g)
    L, Pd, cert, st = ctx.level_dppr(G, sets, ALPHA, EPS)
    assert st == 0 and cert.max() <= EPS
    Dfull = oracle_dppr(g, ALPHA)
    ref = O.level_dppr(Dfull, sets)
    check_dppr(L, ref)
    check_pdist(Pd, ref, cert, g.n)
    # a supernode whose leaves all have d = 0 has a zero row
    deg = np.diff(g.row_ptr)
    for i, s in enumerate(sets):
        if np.all(deg[s] == 0):
            assert np.all(L[i] == 0.0)


def test_level_dppr_partial_cover_and_fp64_outputs(ctx):
    """Supernodes covering only part of the graph (walks still pass through the
    other nodes), uneven leaf-set sizes, FP64 outputs."""
    g = synth.chung_lu(900, 10, 2.5, seed=3)
    rng_sets = synth.sample_view(g.n, 400, seed=5)
    cuts = [0, 1, 3, 40, 100, 101, 250, 400]
    sets = [np.sort(rng_sets[a:b]).astype(np.int32) for a, b in zip(cuts[:-1], cuts[1:])]
    G = ctx.upload_graph(g)
    L, Pd, cert, st = ctx.level_dppr(G, sets, ALPHA, EPS, out64=True)
    assert L.dtype == np.float64 and st == 0 and cert.max() <= EPS
    ref = O.level_dppr(oracle_dppr(g, ALPHA), sets)
    check_dppr(L, ref)
    check_pdist(Pd, ref, cert, g.n)


def test_level_dppr_singletons_reduce_to_node_dppr(ctx):
    import paper_2112_14944_gb300 as P
    g = synth.chung_lu(500, 8, 2.5, seed=9)
    view = synth.sample_view(g.n, 150, seed=2)
    G = ctx.upload_graph(g)
    L, Pl, cert, st = ctx.level_dppr(G, [[int(v)] for v in view], ALPHA, EPS)
    assert st == 0 and cert.max() <= EPS
    D, Pd, cert2, _ = ctx.dppr(G, view, ALPHA, EPS, P.FP32)
    ref = oracle_dppr(g, ALPHA)[np.ix_(view, view)]
    check_dppr(L, ref)
    check_dppr(D, ref)
    assert np.all(np.abs(L.astype(np.float64) - D) <= cert[:, None] + cert2[:, None] + 2e-7 * np.maximum(1, np.abs(ref)))


def test_level_dppr_many_supernodes_ragged_groups(ctx):
    """Chung-Lu n = 8,000 with 1,400 supernodes of 1..8 random leaves (a
    partial cover): the supernodes take several source groups of the
    propagation, the last one ragged."""
    g = synth.chung_lu(8000, 20, 2.5, seed=0)
    perm = synth.sample_view(g.n, g.n, seed=8)
    nsup = 1400
    sizes = 1 + (np.arange(nsup) * 7919) % 8
    off = np.concatenate([[0], np.cumsum(sizes)])
    sets = [np.sort(perm[off[i]:off[i + 1]]).astype(np.int32) for i in range(nsup)]
    G = ctx.upload_graph(g)
    L, Pd, cert, st = ctx.level_dppr(G, sets, ALPHA, EPS)
    assert st == 0 and cert.max() <= EPS
    st_ = ctx.stats()
    assert st_["groups"] >= 2 and nsup % st_["source_group"] != 0
    ref = O.level_dppr(oracle_dppr(g, ALPHA), sets)
    check_dppr(L, ref)
    check_pdist(Pd, ref, cert, g.n)
    # Eq. (11) averaged: sum_j |F_j| pi_d(V_i, V_j) <= the mean degree of V_i's leaves
    dbar = np.array([O.degrees(g.n, g.row_ptr, g.col)[s].mean() for s in sets])
    assert np.all(L.astype(np.float64) @ sizes <= dbar * (1 + 1e-5) + 1e-6)


def test_level_dppr_rejects_bad_leaf_sets(ctx):
    import paper_2112_14944_gb300 as P
    from paper_2112_14944_gb300 import _binding as B
    g = synth.chung_lu(100, 6, 2.5, seed=1)
    G = ctx.upload_graph(g)
    for sets in ([[1, 2], [2, 3]],          # overlapping
                 [[1, 2], []],              # empty
                 [[1, 200]],                # out of range
                 [[-1]]):
        with pytest.raises((P.PPRVizError, ValueError)) as ei:
            ctx.level_dppr(G, sets, ALPHA, EPS)
        if isinstance(ei.value, P.PPRVizError):
            assert ei.value.status == B.PPRVIZ_E_INVALID_ARG
