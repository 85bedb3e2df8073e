"""Pins of the oracle's off-surface evaluation (Eq. rep, Eq. repS, Eq. multirep, Eq. erepK) and of the
surface residual (Eq. residual) against exact exterior solutions.

* a sphere translating with velocity v drives Stokes' flow
  u = (3a/4)(v + (v.e)e)/r + (a^3/4)(v - 3(v.e)e)/r^3,  e = x/r;
* a sphere rotating with omega drives u = (a/r)^3 omega x x;
* a conductor with net charge Q has the potential Q/(4 pi r).
A wrong strength formula (projector, completion, sign) or a wrong kernel in the evaluation breaks one of
them at O(1).  The MFS error itself grows towards the surface (at r = 1.07 it is 2e-6 of the largest
value for mobility and 3e-5 for resistance, the bare-self-block formulation); the probes lie in
1.2 <= r <= 6 and are held to 1e-5, and the surface itself is covered by the residual test.
"""

import numpy as np

from mfs_inputs.workloads import sphere_shape, spheroid_shape
from oracle import Problem
from test_oracle_closed_forms import _single
from test_oracle_dirichlet import _cluster


def _probe_points(rng, n, rmin, rmax):
    e = rng.standard_normal((n, 3))
    e /= np.linalg.norm(e, axis=1, keepdims=True)
    return e * rng.uniform(rmin, rmax, (n, 1))


def _stokes_translating(x, v, a=1.0):
    r = np.linalg.norm(x, axis=1, keepdims=True)
    e = x / r
    ve = np.sum(e * v, axis=1, keepdims=True)
    return 0.75 * a * (v + ve * e) / r + 0.25 * a**3 * (v - 3 * ve * e) / r**3


def _stokes_rotating(x, w, a=1.0):
    r = np.linalg.norm(x, axis=1, keepdims=True)
    return (a / r) ** 3 * np.cross(w, x)


def test_mobility_field_of_a_sphere():
    pr = Problem(_single(sphere_shape(600, 300), "stokes"))
    rng = np.random.default_rng(1)
    x = _probe_points(rng, 40, 1.2, 6.0)
    F, T = np.array([[0.3, -0.2, 1.0]]), np.array([[0.5, 0.1, -0.7]])
    U, W, info = pr.solve_mobility(F, T)
    strengths = pr.total_strengths_mobility([0], info[0].x, F, T)
    u = pr.evaluate([0], strengths, x)
    exact = _stokes_translating(x, U[0]) + _stokes_rotating(x, W[0])
    assert np.abs(u - exact).max() < 1e-5 * np.abs(exact).max()


def test_resistance_field_of_a_sphere():
    pr = Problem(_single(sphere_shape(600, 300), "stokes"))
    rng = np.random.default_rng(2)
    x = _probe_points(rng, 40, 1.2, 6.0)
    v, w = np.array([[0.2, 0.9, -0.4]]), np.array([[-0.3, 0.6, 0.2]])
    _, _, info = pr.solve_resistance(v, w)
    u = pr.evaluate([0], pr.strengths_dirichlet([0], info[0].x), x)
    exact = _stokes_translating(x, v[0]) + _stokes_rotating(x, w[0])
    assert np.abs(u - exact).max() < 1e-5 * np.abs(exact).max()


def test_potential_of_a_charged_sphere():
    pr = Problem(_single(sphere_shape(600, 300), "laplace"))
    rng = np.random.default_rng(3)
    x = _probe_points(rng, 40, 1.2, 6.0)
    Q = np.array([1.7])
    phi, info = pr.solve_elastance(Q)
    u = pr.evaluate([0], pr.total_strengths_elastance([0], info[0].x, Q), x)
    exact = Q[0] / (4 * np.pi * np.linalg.norm(x, axis=1))
    assert np.abs(u - exact).max() < 1e-5 * np.abs(exact).max()
    # capacitance: the same field from the conductor held at its potential
    q, info = pr.solve_capacitance(phi)
    u2 = pr.evaluate([0], pr.strengths_dirichlet([0], info[0].x), x)
    assert np.abs(u2 - exact).max() < 1e-5 * np.abs(exact).max()


def _residual(m, n):
    """max and RMS of Eq. residual on a 2000-point lattice of each of three rotated (1,1,1.5) spheroids."""
    shape = spheroid_shape(m, n, 1.0, 1.5, 0.3)
    wl = _cluster("stokes", 3, shape, quats=True, spacing=3.4)
    pr = Problem(wl)
    rng = np.random.default_rng(4)
    F, T = rng.standard_normal((3, 3)), rng.standard_normal((3, 3))
    U, W, info = pr.solve_mobility(F, T)
    mu = pr.total_strengths_mobility(list(range(3)), info[0].x, F, T)
    fine = spheroid_shape(2000, 300, 1.0, 1.5, 0.3).colloc
    mx, rms = 0.0, 0.0
    for k in range(3):
        x_loc = fine @ pr.R[k].T
        u = pr.evaluate(list(range(3)), mu, wl.centres[k] + x_loc)
        g = U[k] + np.cross(W[k], x_loc)
        e = np.linalg.norm(u - g, axis=1)
        mx = max(mx, np.max(e / np.linalg.norm(g, axis=1)))
        rms = max(rms, np.sqrt(np.mean(e**2) / np.mean(np.sum(g**2, axis=1))))
    return mx, rms


def test_surface_residual_converges():
    """Eq. residual of the mobility solution (flow minus the rigid motion of the computed U, Omega) falls
    with the discretisation: measured max 5.4e-2 -> 5.9e-3 and RMS 8.7e-3 -> 9.1e-4 from M=300 to
    M=600 (and 3.5e-4 / 3.8e-5 at M=1200).  A wrong strength (projector, completion) or evaluation
    would leave an O(1) residual that does not fall."""
    mx1, rms1 = _residual(300, 150)
    mx2, rms2 = _residual(600, 300)
    assert mx2 < 1e-2 and rms2 < 2e-3
    assert mx1 > 5 * mx2 and rms1 > 5 * rms2


def test_stress_of_translating_and_rotating_sphere():
    """Classical results on a unit sphere in Stokes flow (mu = 1.7): translating with v, the surface
    traction is uniform, T = -3 mu v / (2a), and the pressure is p = (3 mu a / 2) (v . x) / r^3;
    rotating with omega, T = -3 mu (omega x x) / a and p = 0.  Summing the traction over an
    equal-area lattice gives the force of the fluid on the body, -6 pi mu a v (Eq. forces), minus the
    force [f; t] = K_N^T lambda the resistance solve reports (the force the body exerts).  The traction (a derivative of
    the field, on the surface) converges more slowly than the velocity: measured max relative error
    13 %, 1.1 %, 3.6e-4 at M = 300, 600, 1200 (R_p = 0.7)."""
    mu = 1.7
    v, w = np.array([[0.2, -0.5, 0.9]]), np.array([[0.4, 0.3, -0.6]])
    on = sphere_shape(2000, 300).colloc  # surface points, outward normals = positions
    errs = []
    for m, n in ((600, 300), (1200, 600)):
        pr = Problem(_single(sphere_shape(m, n), "stokes", mu=mu))
        worst = 0.0
        for vel, omg in ((v, np.zeros((1, 3))), (np.zeros((1, 3)), w)):
            _, _, info = pr.solve_resistance(vel, omg)
            p, T = pr.evaluate_stress([0], pr.strengths_dirichlet([0], info[0].x), on, on)
            exact = -3 * mu * vel[0] / 2 - 3 * mu * np.cross(omg[0], on)
            scale = np.abs(exact).max()
            worst = max(worst, np.abs(T - exact).max() / scale, np.abs(p - 1.5 * mu * (on @ vel[0])).max() / scale)
        errs.append(worst)
    assert errs[1] < 1e-3 and errs[0] > 10 * errs[1], errs
    _, _, info = pr.solve_resistance(v, np.zeros((1, 3)))
    _, T = pr.evaluate_stress([0], pr.strengths_dirichlet([0], info[0].x), on, on)
    np.testing.assert_allclose(T.sum(axis=0) * 4 * np.pi / on.shape[0], -6 * np.pi * mu * v[0], rtol=1e-3)
