"""Pins of the oracle's adjoint (mobility VJP) against central finite differences in FP64.

Loss L = sum_k |U_k|^2 (+ a torque-weighted term on Omega to exercise dL/dOmega).  Central
differences with h = 1e-6 and GMRES at 1e-14: truncation O(h^2) and solve error / h stay far
below the 1e-6 relative tolerance.  A slip anywhere in the chain (the seed -(S_L^+)^T K_N, the
transposed pair sum, the projector in A^T, mu = lambda_0 + (I - L) S_L^+ gamma, the sign of the
source-side gradient) shows as an O(1) mismatch on some coordinate.
"""

import numpy as np
import pytest

from tests.test_oracle_invariants import _cluster
from oracle import Problem


def _loss(pr, wl, centres, F, T, wU, wW):
    wl2 = type(wl)(**{**wl.__dict__, "centres": centres})
    U, W, _ = Problem(wl2).solve_mobility(F, T, tol=1e-14, max_iter=300)
    return float(np.sum(wU * U * U) + np.sum(wW * W * W)), U, W


@pytest.mark.parametrize("shapes", ["spheres", "mixed"])
def test_centre_gradient_matches_finite_differences(shapes):
    wl = _cluster("stokes", P=3, m=160, n=80, seed=5, shapes=shapes)
    pr = Problem(wl)
    F, T = wl.F[0], wl.T[0]
    rng = np.random.default_rng(7)
    wU, wW = 1.0, 0.3
    L0, U, W = _loss(pr, wl, wl.centres, F, T, wU, wW)
    g, gF, gT = pr.mobility_vjp(F, T, 2 * wU * U, 2 * wW * W)
    h = 1e-6
    for _ in range(5):
        k, a = rng.integers(0, 3), rng.integers(0, 3)
        cp, cm = wl.centres.copy(), wl.centres.copy()
        cp[k, a] += h
        cm[k, a] -= h
        fd = (_loss(pr, wl, cp, F, T, wU, wW)[0] - _loss(pr, wl, cm, F, T, wU, wW)[0]) / (2 * h)
        assert abs(fd - g[k, a]) <= 1e-6 * np.abs(g).max(), (k, a, fd, g[k, a])
    # a random direction
    d = rng.standard_normal(wl.centres.shape)
    fd = (_loss(pr, wl, wl.centres + h * d, F, T, wU, wW)[0] - _loss(pr, wl, wl.centres - h * d, F, T, wU, wW)[0]) / (2 * h)
    assert abs(fd - np.sum(g * d)) <= 1e-6 * np.abs(g).sum()
    # forces and torques: a random direction in (F, T)
    dF, dT = rng.standard_normal(F.shape), rng.standard_normal(T.shape)
    lp = float(np.sum(wU * pr.solve_mobility(F + h * dF, T + h * dT, tol=1e-14)[0] ** 2)
               + np.sum(wW * pr.solve_mobility(F + h * dF, T + h * dT, tol=1e-14)[1] ** 2))
    lm = float(np.sum(wU * pr.solve_mobility(F - h * dF, T - h * dT, tol=1e-14)[0] ** 2)
               + np.sum(wW * pr.solve_mobility(F - h * dF, T - h * dT, tol=1e-14)[1] ** 2))
    assert abs((lp - lm) / (2 * h) - np.sum(gF * dF) - np.sum(gT * dT)) <= 1e-6 * (np.abs(gF).sum() + np.abs(gT).sum())


def test_translation_invariance_of_gradient():
    """Moving every body together changes nothing: the centre gradient sums to zero."""
    wl = _cluster("stokes", P=3, m=120, n=60, seed=6, shapes="mixed")
    pr = Problem(wl)
    F, T = wl.F[0], wl.T[0]
    U, W, _ = pr.solve_mobility(F, T, tol=1e-14)
    g, _, _ = pr.mobility_vjp(F, T, 2 * U, 0 * W)
    np.testing.assert_allclose(g.sum(axis=0), 0.0, atol=1e-10 * np.abs(g).max())


def test_transposed_matvec_is_the_transpose_of_the_assembled_matrix():
    """A^T w by the oracle's transposed pair sums and transposed one-body apply equals the transpose of
    Eq. 2esysprec assembled from explicit kernel matrices and rotation blocks (rotated mixed shapes)."""
    wl = _cluster("stokes", P=3, m=50, n=25)
    pr = Problem(wl)
    bodies = list(range(3))
    A = pr.assemble_dense(bodies)
    w = np.random.default_rng(4).standard_normal(A.shape[0])
    ref = A.T @ w
    np.testing.assert_allclose(pr.matvec_T(bodies, w), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
