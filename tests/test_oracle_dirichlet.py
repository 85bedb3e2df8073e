"""Pins of the oracle's Dirichlet problems: capacitance (Sec. 2.1) and resistance (Sec. 2.2), one-body
preconditioned with the pseudo-inverse of the bare self block (Sec. 2.3, Eq. 2sysprec, Algorithm 1).

Pinned against what physics fixes independently of the oracle:
* isolated sphere: q = 4 pi a phi, f = 6 pi mu a v, t = 8 pi mu a^3 omega (a dropped 4 pi, 6 pi,
  a wrong torque sign or cross-product convention in K_M, K_N fails);
* two conductors 2.5 apart held at (+1, -1): q = +-(c_s - c_m) from the bispherical series (a wrong
  pair coupling or a sign slip in the preconditioned system fails);
* prolate spheroid drag along and across its axis (closed forms), rotated (Remark congruent);
* the capacitance and resistance matrices are the inverses of the elastance and mobility matrices
  the recompleted solver computes (an independent formulation, Sec. 3) and symmetric positive
  definite; the paper's 2-way error (Eq. 2way) with distinct proxy offsets is small.
"""

import numpy as np
import pytest

from mfs_inputs.workloads import Workload, make_workload, sphere_shape, spheroid_shape
from oracle import Problem
from oracle.mfs_oracle import quat_to_rotation
from test_oracle_closed_forms import _single, _spheroid_closed_forms, _two_sphere_potential_bispherical


def _cluster(kind, P, shape, seed=7, spacing=2.6, quats=False):
    rng = np.random.default_rng(seed)
    side = int(np.ceil(P ** (1 / 3)))
    grid = np.array([(i, j, k) for i in range(side) for j in range(side) for k in range(side)], float)[:P]
    centres = spacing * grid + 0.05 * rng.standard_normal((P, 3))
    q = None
    if quats:
        q = rng.standard_normal((P, 4))
        q /= np.linalg.norm(q, axis=1, keepdims=True)
    return Workload("cluster", kind, [shape], centres, q, np.zeros(P, np.int32), np.array([0, P], np.int32))


def test_isolated_sphere_capacitance():
    pr = Problem(_single(sphere_shape(600, 300), "laplace"))
    for phi in (1.0, -0.3):
        q, info = pr.solve_capacitance(np.array([phi]))
        assert abs(q[0] - 4 * np.pi * phi) <= 1e-7 * abs(4 * np.pi * phi)
        assert info[0].iters <= 2  # P = 1: the preconditioned matrix is the identity


@pytest.mark.parametrize("mu", [1.0, 2.5])
def test_isolated_sphere_resistance(mu):
    pr = Problem(_single(sphere_shape(600, 300), "stokes", mu=mu))
    U = np.array([[0.3, -0.2, 1.0]])
    W = np.array([[0.5, 0.1, -0.7]])
    F, T, _ = pr.solve_resistance(U, W)
    np.testing.assert_allclose(F[0], 6 * np.pi * mu * U[0], rtol=0, atol=1e-6 * 6 * np.pi * mu)
    np.testing.assert_allclose(T[0], 8 * np.pi * mu * W[0], rtol=0, atol=1e-6 * 8 * np.pi * mu)


def test_two_sphere_capacitance():
    wl = make_workload("two_sphere_elastance")
    pr = Problem(wl)
    q, info = pr.solve_capacitance(np.array([1.0, -1.0]))
    c = 1.0 / _two_sphere_potential_bispherical(1.0, 2.5)  # c_s - c_m
    assert abs(q[0] - c) < 1e-7 * c
    assert abs(q[1] + c) < 1e-7 * c
    assert info[0].converged


def test_rotated_spheroid_resistance():
    """A rotated (1,1,1.5) spheroid: f = R diag(F_t, F_t, F_a) R^T v (closed forms, Remark congruent)."""
    shape = spheroid_shape(600, 300, 1.0, 1.5, 0.3)
    fa, ft, _ = _spheroid_closed_forms(1.0, 1.5)
    q = np.array([0.3, -0.6, 0.2, 0.7])
    q /= np.linalg.norm(q)
    R = quat_to_rotation(q)
    pr = Problem(_single(shape, "stokes", quat=q))
    v = np.array([0.4, -1.0, 0.7])
    F, _, _ = pr.solve_resistance(v[None], np.zeros((1, 3)))
    expect = R @ (np.diag([ft, ft, fa]) @ (R.T @ v))
    assert np.linalg.norm(F[0] - expect) < 2e-5 * np.linalg.norm(expect)


def test_capacitance_inverts_elastance():
    """C E = I for a 4-conductor cluster: two formulations (Sec. 2.1 and Sec. 3.1), one physics."""
    wl = _cluster("laplace", 4, sphere_shape(300, 150))
    pr = Problem(wl)
    C = np.column_stack([pr.solve_capacitance(e)[0] for e in np.eye(4)])
    E = np.column_stack([pr.solve_elastance(e)[0] for e in np.eye(4)])
    np.testing.assert_allclose(C, C.T, atol=1e-6 * np.abs(C).max())
    assert np.all(np.linalg.eigvalsh(0.5 * (C + C.T)) > 0)
    np.testing.assert_allclose(C @ E, np.eye(4), atol=1e-5)


def test_resistance_inverts_mobility():
    """R M = I for three rotated spheroids (6P = 18 columns each way), R symmetric positive definite."""
    # discretisation-level properties: at M=300, N=150 the asymmetry is 1.7e-4 and R M - I 4.7e-5,
    # at M=600, N=300 5.2e-6 and 4.9e-7 (converging with N, as the method should)
    wl = _cluster("stokes", 3, spheroid_shape(600, 300, 1.0, 1.5, 0.3), quats=True, spacing=3.4)
    pr = Problem(wl)
    P = 3
    cols_R, cols_M = [], []
    for e in np.eye(6 * P):
        V = e.reshape(P, 6)
        F, T, _ = pr.solve_resistance(V[:, :3], V[:, 3:])
        cols_R.append(np.concatenate([F, T], axis=1).reshape(-1))
        U, W, _ = pr.solve_mobility(V[:, :3], V[:, 3:])
        cols_M.append(np.concatenate([U, W], axis=1).reshape(-1))
    Rm, Mm = np.column_stack(cols_R), np.column_stack(cols_M)
    np.testing.assert_allclose(Rm, Rm.T, atol=2e-5 * np.abs(Rm).max())
    assert np.all(np.linalg.eigvalsh(0.5 * (Rm + Rm.T)) > 0)
    assert np.abs(Rm @ Mm - np.eye(6 * P)).max() < 5e-6


def test_two_way_error():
    """Eq. 2way: resistance with R_p = 0.7, then mobility with the proxy offset 1.05 times larger."""
    res = _cluster("stokes", 5, sphere_shape(600, 300, rp=0.7), spacing=2.5)
    mob = _cluster("stokes", 5, sphere_shape(600, 300, rp=1 - 1.05 * 0.3), spacing=2.5)
    rng = np.random.default_rng(11)
    U_ref, W_ref = rng.standard_normal((5, 3)), rng.standard_normal((5, 3))
    F, T, _ = Problem(res).solve_resistance(U_ref, W_ref)
    U, W, _ = Problem(mob).solve_mobility(F, T)
    ref = np.concatenate([U_ref, W_ref], axis=1)
    err = np.abs(np.concatenate([U, W], axis=1) - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err  # measured 9.5e-6
    # the same discretisation both ways is an inverse crime: far smaller than the discretisation error
    U2, W2, _ = Problem(res).solve_mobility(F, T)
    crime = np.abs(np.concatenate([U2, W2], axis=1) - ref).max() / np.abs(ref).max()
    assert crime < err
