"""Pins of the FP64 oracle against results fixed by the physics, not by the oracle.

Each test would fail on a plausible slip in the oracle: a dropped r r^T/r^2
term or a wrong 8 pi mu (Stokes drag), a wrong torque sign or cross-product
convention (rotation rate), a wrong 4 pi (sphere potential), a wrong pair
coupling (two-sphere potential, Rotne-Prager far field), a wrong rotation of
congruent bodies (rotated spheroid drag).
"""

import numpy as np
import pytest

from mfs_inputs.workloads import Workload, sphere_shape, spheroid_shape, make_workload
from oracle import Problem


def _single(shape, kind, quat=None, mu=1.0):
    return Workload(
        "single", kind, [shape], np.zeros((1, 3)), None if quat is None else np.asarray(quat)[None],
        np.zeros(1, np.int32), np.array([0, 1], np.int32), mu=mu)


# ---------------------------------------------------------------------------
# Isolated sphere: V = Q/(4 pi a), U = F/(6 pi mu a), Omega = T/(8 pi mu a^3)
# ---------------------------------------------------------------------------

def test_isolated_sphere_potential():
    pr = Problem(_single(sphere_shape(600, 300), "laplace"))
    for q in (1.0, -2.5):
        phi, info = pr.solve_elastance(np.array([q]))
        assert abs(phi[0] - q / (4 * np.pi)) <= 1e-7 * abs(q / (4 * np.pi))
        assert info[0].iters <= 2  # P = 1: the preconditioned matrix is the identity


@pytest.mark.parametrize("mu", [1.0, 2.5])
def test_isolated_sphere_mobility(mu):
    pr = Problem(_single(sphere_shape(600, 300), "stokes", mu=mu))
    F = np.array([[0.3, -0.2, 1.0]])
    T = np.array([[0.5, 0.1, -0.7]])
    U, W, _ = pr.solve_mobility(F, T)
    np.testing.assert_allclose(U[0], F[0] / (6 * np.pi * mu), rtol=0, atol=1e-6 * np.abs(F[0]).max() / (6 * np.pi * mu))
    np.testing.assert_allclose(W[0], T[0] / (8 * np.pi * mu), rtol=0, atol=1e-6 * np.abs(T[0]).max() / (8 * np.pi * mu))


# ---------------------------------------------------------------------------
# Two conducting unit spheres, centres 2.5 apart, charges (+1, -1)
# ---------------------------------------------------------------------------

def _two_sphere_potential_bispherical(a, d, terms=200):
    """V_1 = 1 / (c_s - c_m), c_s - c_m = 4 pi a sinh(beta) sum_{m>=1} 1/sinh(m beta), cosh(beta) = d/(2a)."""
    beta = np.arccosh(d / (2 * a))
    m = np.arange(1, terms + 1)
    return 1.0 / (4 * np.pi * a * np.sinh(beta) * np.sum(1.0 / np.sinh(m * beta)))


def _two_sphere_potential_images(a, d, terms=400):
    """Kelvin images for +1 on sphere 1 and -1 on sphere 2 held at V and -V: the image
    charges inside sphere 1 obey rho_{n+1} = rho_n a / (d - x_n), x_{n+1} = a^2 / (d - x_n)
    (positions measured from the own centre), and V = 1 / (4 pi a sum rho_n)."""
    rho, x, total = 1.0, 0.0, 0.0
    for _ in range(terms):
        total += rho
        rho, x = rho * a / (d - x), a * a / (d - x)
    return 1.0 / (4 * np.pi * a * total)


def test_series_agree():
    v1 = _two_sphere_potential_bispherical(1.0, 2.5)
    v2 = _two_sphere_potential_images(1.0, 2.5)
    assert abs(v1 - v2) < 1e-14
    assert abs(v1 - 0.0447467620348398) < 1e-14


def test_two_sphere_potential():
    wl = make_workload("two_sphere_elastance")
    pr = Problem(wl)
    phi, info = pr.solve_elastance(wl.Q)
    v = _two_sphere_potential_bispherical(1.0, 2.5)
    assert abs(phi[0] - v) < 1e-7 * v
    assert abs(phi[1] + v) < 1e-7 * v
    assert info[0].converged


# ---------------------------------------------------------------------------
# Prolate spheroid (a, a, c): drag along and across the axis, capacitance
# ---------------------------------------------------------------------------

def _spheroid_closed_forms(a, c, mu=1.0):
    e = np.sqrt(1 - (a / c) ** 2)
    lg = np.log((1 + e) / (1 - e))
    f_axial = 16 * np.pi * mu * c * e**3 / ((1 + e * e) * lg - 2 * e)
    f_trans = 32 * np.pi * mu * c * e**3 / (2 * e + (3 * e * e - 1) * lg)
    cap = 8 * np.pi * c * e / lg
    return f_axial, f_trans, cap


def test_spheroid_closed_forms_sphere_limit():
    fa, ft, cap = _spheroid_closed_forms(1.0, 1.0 + 1e-5)
    assert abs(fa / (6 * np.pi) - 1) < 1e-4 and abs(ft / (6 * np.pi) - 1) < 1e-4
    assert abs(cap / (4 * np.pi) - 1) < 1e-4


@pytest.mark.parametrize("m,n,c,dsep,tol", [(600, 300, 1.5, 0.3, 2e-5), (800, 400, 2.0, 0.25, 5e-5)])
def test_spheroid_drag_and_capacitance(m, n, c, dsep, tol):
    shape = spheroid_shape(m, n, 1.0, c, dsep)
    fa, ft, cap = _spheroid_closed_forms(1.0, c)
    pr = Problem(_single(shape, "stokes"))
    U, _, _ = pr.solve_mobility(np.array([[1.0, 0.0, 0.0]]), np.zeros((1, 3)))
    assert abs(U[0, 0] * ft - 1) < tol
    U, _, _ = pr.solve_mobility(np.array([[0.0, 0.0, 1.0]]), np.zeros((1, 3)))
    assert abs(U[0, 2] * fa - 1) < tol
    pl = Problem(_single(shape, "laplace"))
    phi, _ = pl.solve_elastance(np.array([1.0]))
    assert abs(1 / phi[0] / cap - 1) < tol


def test_rotated_spheroid_drag():
    """A rotated spheroid moves as R diag(1/F_t, 1/F_t, 1/F_a) R^T f (Remark congruent, Eq. Krot)."""
    from oracle.mfs_oracle import quat_to_rotation

    shape = spheroid_shape(600, 300, 1.0, 1.5, 0.3)
    fa, ft, _ = _spheroid_closed_forms(1.0, 1.5)
    q = np.array([0.8, 0.2, -0.5, 0.3])
    q /= np.linalg.norm(q)
    R = quat_to_rotation(q)
    pr = Problem(_single(shape, "stokes", quat=q))
    f = np.array([0.4, -1.0, 0.7])
    U, _, _ = pr.solve_mobility(f[None], np.zeros((1, 3)))
    expect = R @ (np.diag([1 / ft, 1 / ft, 1 / fa]) @ (R.T @ f))
    assert np.linalg.norm(U[0] - expect) < 2e-5 * np.linalg.norm(expect)


# ---------------------------------------------------------------------------
# Far field: two spheres 20 radii apart follow the Rotne-Prager tensor
# ---------------------------------------------------------------------------

def test_rotne_prager_far_field():
    dist = 20.0
    wl = Workload("rp", "stokes", [sphere_shape(600, 300)], np.array([[0, 0, 0], [dist * 0.6, dist * 0.8, 0]]),
                  None, np.zeros(2, np.int32), np.array([0, 2], np.int32))
    pr = Problem(wl)
    F = np.array([[0.0, 0.0, 0.0], [0.3, -1.0, 0.5]])
    U, W, _ = pr.solve_mobility(F, np.zeros((2, 3)))
    r = wl.centres[0] - wl.centres[1]
    d = np.linalg.norm(r)
    dh = r / d
    M12 = ((1 + 2 / (3 * d * d)) * np.eye(3) + (1 - 2 / (d * d)) * np.outer(dh, dh)) / (8 * np.pi * d)
    # translation-translation coupling: Rotne-Prager is exact to O(d^-7)
    assert np.linalg.norm(U[0] - M12 @ F[1]) < 2e-6 * np.linalg.norm(M12 @ F[1])
    # sphere 1 rotates with half the vorticity of the Stokeslet at its centre
    om = np.cross(F[1], r) / (8 * np.pi * d**3)
    assert np.linalg.norm(W[0] - om) < 1e-5 * np.linalg.norm(om)
    # self mobility is corrected only at O(d^-4)
    assert np.linalg.norm(U[1] - F[1] / (6 * np.pi)) < 5e-5 * np.linalg.norm(F[1] / (6 * np.pi))


# ---------------------------------------------------------------------------
# One body: the saddle-point (Schur complement) mobility M = (K_N^T S^+ K_M)^-1 (Sec. 3.2)
# ---------------------------------------------------------------------------
def _stokeslet_block(X, Y, mu=1.0):
    d = X[:, None, :] - Y[None, :, :]
    r = np.linalg.norm(d, axis=2)
    S = np.eye(3)[None, None] / r[..., None, None] + d[..., :, None] * d[..., None, :] / r[..., None, None] ** 3
    return (S / (8 * np.pi * mu)).transpose(0, 2, 1, 3).reshape(3 * X.shape[0], 3 * Y.shape[0])


def _rigid_motion_matrix(P):
    """Block rows [I, A_i] with A_i omega = omega x p_i (the body centre at the origin)."""
    K = np.zeros((3 * P.shape[0], 6))
    for i, p in enumerate(P):
        K[3 * i:3 * i + 3, :3] = np.eye(3)
        K[3 * i:3 * i + 3, 3:] = np.array([[0, p[2], -p[1]], [-p[2], 0, p[0]], [p[1], -p[0], 0]])
    return K


def test_single_body_mobility_matches_saddle_point_form():
    """A rotated (1,1,1.5) spheroid: the recompleted solver's 6x6 mobility matrix (completion, projectors,
    GMRES, recovery) against the saddle-point form built from the plain pseudo-inverse of the self block;
    the two discretisations agree to an error that falls spectrally with N (measured 2.0e-5 at N=150,
    2.0e-7 at N=300, 3.4e-10 at N=600)."""
    from oracle.mfs_oracle import quat_to_rotation

    q = np.array([0.3, -0.6, 0.2, 0.7])
    q /= np.linalg.norm(q)
    R = quat_to_rotation(q)
    errs = []
    for m, n in ((300, 150), (600, 300)):
        shape = spheroid_shape(m, n, 1.0, 1.5, 0.3)
        pr = Problem(_single(shape, "stokes", quat=q))
        X, Y = shape.colloc @ R.T, shape.proxy @ R.T
        resistance = _rigid_motion_matrix(Y).T @ np.linalg.pinv(_stokeslet_block(X, Y)) @ _rigid_motion_matrix(X)
        M_sp = np.linalg.inv(resistance)
        cols = []
        for e in np.eye(6):
            U, W, _ = pr.solve_mobility(e[None, :3], e[None, 3:], tol=1e-13)
            cols.append(np.concatenate([U[0], W[0]]))
        M_rec = np.column_stack(cols)
        errs.append(np.linalg.norm(M_rec - M_sp) / np.linalg.norm(M_sp))
    assert errs[1] < 2e-6, errs
    assert errs[1] < errs[0] / 20, errs
