"""The allocation-free energy entry point (pprviz_energy_noalloc) against the
regular pprviz_energy, through the C ABI.

pprviz_energy_noalloc serves callers that may not allocate device memory when
they call (their memory belongs to their own pool or to a framework's
allocator, or sits under a hard cap): its scratch is a fixed device array
inside the library. This file is collected last so that, if it fails, a run
that stops at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

# the energy tests' FP32 tolerance (tests/test_gpu_layout.py)
TOL = 2e-5


def _problem(k, seed):
    """A symmetric distance matrix in [2, 2 ln k] with a zero diagonal, and coordinates."""
    r = synth.uniform(seed, 21, np.arange(k * k, dtype=np.uint64)).reshape(k, k)
    D = 2.0 + (2.0 * np.log(k) - 2.0) * (r + r.T) / 2.0
    np.fill_diagonal(D, 0.0)
    X = synth.uniform_x0(k, seed=seed).astype(np.float64) * 4.0
    return D.astype(np.float32), X.astype(np.float32)


def test_noalloc_energy_matches_energy_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    import paper_2112_14944_gb300 as P
    from paper_2112_14944_gb300 import _binding as B

    ctx = P.Context(0, torch_stream=True)
    # the second call is smaller than the first, so anything the first call
    # left in the shared scratch would show up in its results
    for k, seed, scale in [(700, 1, 0.5), (300, 2, 1.0)]:
        D, X = _problem(k, seed)
        Dd = torch.from_numpy(D).cuda()
        Xd = torch.from_numpy(X).cuda()
        torch.cuda.synchronize()
        e_ref, gx_ref, gd_ref = ctx.energy(Dd, Xd, grad_scale=scale, grad_x=True, grad_pdist=True)
        torch.cuda.synchronize()
        gx = torch.full((k, 2), float("nan"), device="cuda")
        gd = torch.full((k, k), float("nan"), device="cuda")
        torch.cuda.synchronize()
        status, e = B.pprviz_energy_noalloc(Dd, k, Xd, scale, gx, gd)
        torch.cuda.synchronize()
        assert status == B.PPRVIZ_OK
        assert abs(e - e_ref) <= TOL * abs(e_ref)
        gx_ref, gd_ref = gx_ref.cpu().numpy(), gd_ref.cpu().numpy()
        gx, gd = gx.cpu().numpy(), gd.cpu().numpy()
        assert np.isfinite(gx).all() and np.isfinite(gd).all()
        assert np.abs(gx - gx_ref).max() <= TOL * max(1.0, np.abs(gx_ref).max())
        assert np.abs(gd - gd_ref).max() <= TOL * max(1.0, np.abs(gd_ref).max())
        # energy alone (no gradient outputs) gives the same value
        status, e2 = B.pprviz_energy_noalloc(Dd, k, Xd)
        assert status == B.PPRVIZ_OK and abs(e2 - e_ref) <= TOL * abs(e_ref)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    torch = pytest.importorskip("torch")
    from paper_2112_14944_gb300 import _binding as B

    small = torch.zeros(16, device="cuda")
    # the size is checked before any device work is enqueued
    for k in (0, -3, 65537, 1 << 20):
        status, _ = B.pprviz_energy_noalloc(small, k, small)
        assert status == B.PPRVIZ_E_INVALID_ARG
    bad = torch.tensor([[0.0, -1.0], [-1.0, 0.0]], device="cuda")
    xs = torch.zeros((2, 2), device="cuda")
    torch.cuda.synchronize()
    status, _ = B.pprviz_energy_noalloc(bad, 2, xs)
    assert status == B.PPRVIZ_E_INVALID_ARG
