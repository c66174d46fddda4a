"""GPU parity of the layout quality metrics of Sec. 2 (ND and ULCV) against
the FP64 oracle's definitions, through the C ABI (pprviz_layout_metrics).

Both sides sum in FP64 from the same coordinates (FP32 coordinates are widened
exactly on both sides), in different orders: relative 1e-12.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2112_14944_gb300 as P
    c = P.Context(0)
    yield c
    c.close()


def _edges(g, view=None):
    """Each undirected edge of g once (u < v), as row indices of the layout."""
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    keep = src < g.col
    e = np.stack([src[keep], g.col[keep].astype(np.int64)], axis=1)
    if view is None:
        return e
    pos = np.full(g.n, -1, dtype=np.int64)
    pos[np.asarray(view)] = np.arange(len(view))
    e = pos[e]
    return e[(e >= 0).all(axis=1)]


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_nd_ulcv_whole_graph_layout(ctx, dt):
    g = synth.chung_lu(800, 10, 2.5, seed=2)
    G = ctx.upload_graph(g)
    X = (synth.uniform_x0(g.n, seed=5).astype(np.float64) * 10).astype(dt)
    nd, ul = ctx.layout_metrics(X, G)
    Xd = X.astype(np.float64)
    assert abs(nd - O.node_distribution(Xd)) <= 1e-12 * O.node_distribution(Xd)
    ref = O.ulcv(Xd, _edges(g))
    assert abs(ul - ref) <= 1e-12 * ref


def test_nd_ulcv_of_a_view_and_device_buffers(ctx):
    torch = pytest.importorskip("torch")
    g = synth.chung_lu(3000, 12, 2.5, seed=4)
    G = ctx.upload_graph(g)
    view = synth.sample_view(g.n, 1200, seed=6)
    X = synth.uniform_x0(len(view), seed=7).astype(np.float32) * 3
    nd, ul = ctx.layout_metrics(torch.from_numpy(X).cuda(), G, torch.from_numpy(view).cuda())
    Xd = X.astype(np.float64)
    assert abs(nd - O.node_distribution(Xd)) <= 1e-12 * O.node_distribution(Xd)
    ref = O.ulcv(Xd, _edges(g, view))
    assert abs(ul - ref) <= 1e-12 * ref
    # ND without a graph
    nd2, ul2 = ctx.layout_metrics(X)
    assert ul2 is None and abs(nd2 - nd) <= 1e-12 * nd


def test_metrics_degenerate_cases(ctx):
    g = synth.chung_lu(200, 6, 2.5, seed=1)
    G = ctx.upload_graph(g)
    X = synth.uniform_x0(g.n, seed=2).astype(np.float64)
    X[17] = X[40]                                   # a coincident pair: ND is infinite
    nd, _ = ctx.layout_metrics(X, G)
    assert nd == math.inf
    # a view with no edge inside it: ULCV is NaN
    deg = np.diff(g.row_ptr)
    iso = np.array([v for v in range(g.n) if deg[v] == 0][:2] or [0], dtype=np.int32)
    if len(iso) == 2:
        _, ul = ctx.layout_metrics(np.array([[0.0, 0.0], [1.0, 1.0]]), G, iso)
        assert math.isnan(ul)
    # a realised layout of the unit square: ND = 5, ULCV = 0
    sq = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    G4 = ctx.upload(4, np.array([0, 2, 4, 6, 8], np.int64), np.array([1, 3, 0, 2, 1, 3, 0, 2], np.int32))
    nd, ul = ctx.layout_metrics(sq, G4)
    assert abs(nd - 5.0) < 1e-14 and abs(ul) < 1e-15
