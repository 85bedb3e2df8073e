"""Pins of the triaxial ellipsoid discretisation (Sec. 4.2) through the oracle: a single Type T
ellipsoid (semi-axes 0.4, 0.6, 1) translating along each axis feels the classical ellipsoid drag,
and as a conductor has the classical capacitance:

    F_i = 16 pi mu / (chi + a_i^2 alpha_i),   C = 8 pi / chi,
    chi = int_0^inf dl / Delta(l),  alpha_i = int_0^inf dl / ((a_i^2 + l) Delta(l)),
    Delta(l) = sqrt((a^2 + l)(b^2 + l)(c^2 + l)).

The formula itself is checked against the prolate-spheroid closed forms (an independent textbook
result) before it is used.  A wrong grid (rings, normals of the proxy shift) or a wrong rotation of
a triaxial body misses these by far more than the MFS error.
"""

import numpy as np
import pytest

from mfs_inputs.workloads import ellipsoid_shape
from oracle import Problem
from oracle.mfs_oracle import quat_to_rotation
from test_oracle_closed_forms import _single, _spheroid_closed_forms

scipy_integrate = pytest.importorskip("scipy.integrate")


def _ellipsoid_coefficients(a, b, c, mu=1.0):
    delta = lambda l: np.sqrt((a * a + l) * (b * b + l) * (c * c + l))  # noqa: E731
    chi = scipy_integrate.quad(lambda l: 1.0 / delta(l), 0, np.inf, epsabs=0, epsrel=1e-13, limit=400)[0]
    drag = []
    for ai in (a, b, c):
        alpha = scipy_integrate.quad(lambda l: 1.0 / ((ai * ai + l) * delta(l)), 0, np.inf, epsabs=0,
                                     epsrel=1e-13, limit=400)[0]
        drag.append(16 * np.pi * mu / (chi + ai * ai * alpha))
    return np.array(drag), 8 * np.pi / chi


def test_ellipsoid_formula_matches_spheroid_closed_forms():
    drag, cap = _ellipsoid_coefficients(1.0, 1.0, 1.5)
    fa, ft, c = _spheroid_closed_forms(1.0, 1.5)
    np.testing.assert_allclose(drag, [ft, ft, fa], rtol=1e-10)
    assert abs(cap / c - 1) < 1e-10


def test_grid_counts_follow_the_paper():
    for n_v in (20, 34, 40):
        sh = ellipsoid_shape(n_v, 0.4, 0.6, 1.0, 0.125)
        target = 17 + 3.9 * n_v + 0.44 * n_v * n_v
        assert abs(sh.n_proxy - target) <= 0.02 * target
        assert 1.2 < sh.n_colloc / sh.n_proxy < 1.4  # M ~ 1.3 N
        # proxies lie inside the body, collocation points on it
        x = sh.colloc / np.array([0.4, 0.6, 1.0])
        np.testing.assert_allclose(np.sum(x * x, axis=1), 1.0, atol=1e-12)
        y = sh.proxy / np.array([0.4, 0.6, 1.0])
        assert np.all(np.sum(y * y, axis=1) < 1.0)


def test_type_t_ellipsoid_drag_and_capacitance():
    drag, cap = _ellipsoid_coefficients(0.4, 0.6, 1.0)
    q = np.array([0.9, -0.2, 0.3, 0.25])
    q /= np.linalg.norm(q)
    R = quat_to_rotation(q)
    shape = ellipsoid_shape(24, 0.4, 0.6, 1.0, 0.125)
    pr = Problem(_single(shape, "stokes", quat=q))
    # measured at N_v = 24: 0.8-1.2e-4 for drag and mobility, 6e-6 for the capacitance; at N_v = 34
    # (the large runs) 2-6e-6 and 1.5e-7: the grid converges
    for i in range(3):  # along each body axis, rotated into the world frame
        v = R[:, i]
        F, _, _ = pr.solve_resistance(v[None], np.zeros((1, 3)))
        assert np.linalg.norm(F[0] - drag[i] * v) < 2e-4 * drag[i], (i, F[0] @ v, drag[i])
        U, _, _ = pr.solve_mobility(v[None], np.zeros((1, 3)))  # the recompleted formulation too
        assert np.linalg.norm(U[0] - v / drag[i]) < 2e-4 / drag[i]
    pl = Problem(_single(shape, "laplace", quat=q))
    qn, _ = pl.solve_capacitance(np.array([1.0]))
    assert abs(qn[0] / cap - 1) < 2e-5
