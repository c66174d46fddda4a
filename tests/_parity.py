"""Parity gates shared by the GPU tests (derived from the paper's definitions).

PDist tolerance. The DPPR contract is absolute: the certificate c_s bounds
|pi_d_hat(s, t) - pi_d(s, t)| for every t. Through Eq. (1) the error of
z_ij = pi_d(i,j) + pi_d(j,i) is at most c_i + c_j, and on the unclamped branch
|dDelta| = |d ln z| <= |dz| / min(z, z_hat) (the mechanism of Lemma 1); both
clamps are 1-Lipschitz and below z_min = e / n_clamp^2 the upper clamp holds.
So every entry must satisfy
    |Delta_hat - Delta| <= slack + (c_i + c_j) / max(z - c_i - c_j, z_min),
with `slack` covering FP32 output rounding (~1e-7). For entries well above
z_min this is the flat 1e-5 gate; near the upper clamp an absolute DPPR bound
cannot fix Delta more tightly than this (a tighter eps does: see the tests).
"""
import math

import numpy as np

import oracle as O


def pdist_tolerance(Dref, cert, n_clamp, slack=1e-5):
    c = np.asarray(cert, dtype=np.float64)
    cc = c[:, None] + c[None, :]
    z = Dref + Dref.T
    zmin = math.e / float(n_clamp) ** 2
    tol = slack + cc / np.maximum(z - cc, zmin)
    np.fill_diagonal(tol, slack)
    return tol


def check_pdist(got, Dref, cert, n_clamp, slack=1e-5):
    """Compare a GPU PDist with the oracle's PDist of the oracle DPPR under the
    certified per-entry tolerance; returns the max absolute error."""
    ref = O.pdist_from_dppr(Dref, n_clamp)
    err = np.abs(np.asarray(got, dtype=np.float64) - ref)
    tol = pdist_tolerance(Dref, cert, n_clamp, slack)
    bad = err > tol
    assert not bad.any(), (f"{bad.sum()} PDist entries outside the certified tolerance; "
                           f"worst excess {(err - tol).max():.3e}, max error {err.max():.3e}")
    return float(err.max())


def check_dppr(got, ref, tol=1e-6):
    """|got - ref| <= tol * max(1, |ref|) for every entry; returns the max scaled error."""
    err = np.abs(np.asarray(got, dtype=np.float64) - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() <= tol, f"max rel-abs DPPR error {err.max():.3e}"
    return float(err.max())


def oracle_dppr(g, alpha=0.15):
    """All-pairs DPPR of a graph by the oracle's direct solve (Sec. 3.1,
    Definition 1): Pi = alpha (I - (1 - alpha) P)^-1, rows scaled by d(s)."""
    P = O.transition_matrix(g.n, g.row_ptr, g.col, g.weight)
    d = O.degrees(g.n, g.row_ptr, g.col, g.weight)
    return O.dppr_rows(O.ppr_direct(P, alpha), d, np.arange(g.n))


def oracle_pdist(g, alpha=0.15, n_clamp=None):
    """The oracle's all-pairs PDist of a graph (Eq. (1)), FP64: the input of
    the layout parity tests, so that no oracle input comes from the GPU."""
    return O.pdist_from_dppr(oracle_dppr(g, alpha), g.n if n_clamp is None else n_clamp)
