"""Error paths of the C ABI, each forced from the host without any GPU fault.

  PPRVIZ_E_NOT_CONVERGED: an FP32 call asked for an eps below what the FP32
      refinement can certify (the two-float rows reach about d(s) * 1e-13).
      The call stops after its refinement passes, returns the status, and its
      outputs are still valid: each DPPR row is within its stated certificate
      of the oracle's.
  PPRVIZ_E_OOM: a context whose workspace is capped below what a call needs
      fails before allocating; lifting the cap makes the same call succeed.
  PPRVIZ_E_TIMEOUT: a test aid makes one operand copy of the FP32 inverse's
      tensor-core update go missing, so the bounded wait for it expires; the
      kernel stops, drains what it issued and reports the status.
In every case the context stays usable.
"""
import numpy as np
import pytest

import synth
from _parity import check_dppr, oracle_dppr

pytestmark = pytest.mark.gpu
ALPHA = 0.15


@pytest.fixture(scope="module")
def ctx():
    import paper_2112_14944_gb300 as P
    c = P.Context(0)
    yield c
    c.close()


def test_not_converged_below_the_fp32_floor(ctx):
    import paper_2112_14944_gb300 as P
    from paper_2112_14944_gb300 import _binding as B
    g = synth.chung_lu(400, 10, 2.5, seed=11)
    G = ctx.upload_graph(g)
    view = np.arange(g.n, dtype=np.int32)
    eps = 1e-18
    D, _, cert, st = ctx.dppr(G, view, ALPHA, eps, P.FP32)
    assert st == B.PPRVIZ_E_NOT_CONVERGED
    assert np.all(np.isfinite(cert)) and cert.max() > eps
    # the outputs are valid: within the stated certificate of the exact DPPR
    # (plus the rounding of the FP32 output)
    Dref = oracle_dppr(g, ALPHA)
    err = np.abs(D.astype(np.float64) - Dref)
    assert np.all(err <= cert[:, None] + 1e-7 * np.maximum(1.0, np.abs(Dref)))
    # the context keeps working
    D2, _, cert2, st2 = ctx.dppr(G, view, ALPHA, 1e-6, P.FP32)
    assert st2 == B.PPRVIZ_OK and cert2.max() <= 1e-6
    check_dppr(D2, Dref)


def test_workspace_limit_gives_oom_and_the_context_recovers():
    import paper_2112_14944_gb300 as P
    from paper_2112_14944_gb300 import _binding as B
    c = P.Context(0)
    try:
        g = synth.chung_lu(3000, 10, 2.5, seed=6)
        G = c.upload_graph(g)
        view = np.arange(g.n, dtype=np.int32)
        c.set_workspace_limit(1 << 20)  # 1 MiB: below one k x k output
        with pytest.raises(P.PPRVizError) as ei:
            c.dppr(G, view, ALPHA, 1e-6, P.FP32)
        assert ei.value.status == B.PPRVIZ_E_OOM
        assert "workspace limit" in B.pprviz_last_error(c.h)
        x0 = synth.uniform_x0(g.n, seed=0)
        Dl = np.full((g.n, g.n), 3.0, np.float32)
        np.fill_diagonal(Dl, 0.0)
        with pytest.raises(P.PPRVizError) as ei:
            c.layout(Dl, x0, 2, P.FP32)
        assert ei.value.status == B.PPRVIZ_E_OOM
        with pytest.raises(P.PPRVizError):
            c.set_workspace_limit(-1)
        c.set_workspace_limit(0)
        D, _, cert, st = c.dppr(G, view, ALPHA, 1e-6, P.FP32)
        assert st == B.PPRVIZ_OK and cert.max() <= 1e-6
        X, s = c.layout(Dl, x0, 2, P.FP32)
        assert np.all(np.isfinite(X)) and np.isfinite(s)
    finally:
        c.close()


def test_expired_wait_returns_timeout_and_the_context_recovers(ctx):
    """PPRVIZ_E_TIMEOUT: every wait of the tensor-core kernels is bounded by a
    deadline. pprviz_test_expire_wait makes the next FP32 L^w inverse leave
    out one operand copy of one tile, so the wait for it runs out (nothing
    faults); the layout call returns E_TIMEOUT after about the deadline, and
    the next call on the same context is correct."""
    import time

    import oracle as O
    import paper_2112_14944_gb300 as P
    from _parity import oracle_pdist
    from paper_2112_14944_gb300 import _binding as B
    g = synth.chung_lu(300, 8, 2.5, seed=21)      # kp = 384: three pivot blocks
    D32 = oracle_pdist(g, ALPHA).astype(np.float32)
    x0 = synth.uniform_x0(g.n, seed=2)
    B.pprviz_test_expire_wait(ctx.h)
    t0 = time.perf_counter()
    with pytest.raises(P.PPRVizError) as ei:
        ctx.layout(D32, x0, 1, P.FP32)
    dt = time.perf_counter() - t0
    assert ei.value.status == B.PPRVIZ_E_TIMEOUT
    assert "wait expired" in B.pprviz_last_error(ctx.h)
    assert dt < 30.0
    X, _ = ctx.layout(D32, x0, 1, P.FP32)
    ref = O.smacof_step(x0.astype(np.float64), D32.astype(np.float64))
    assert np.abs(X - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())
