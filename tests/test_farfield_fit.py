"""The equivalent-source representation behind the far-field treecode, checked in plain NumPy (CPU).

A node's sources (random points filling a sphere of radius 0.83 r_e, random strengths) are replaced
by 196 point sources on a Fibonacci sphere of radius r_e whose strengths are the least-squares fit
(pseudo-inverse truncated at 1e-12 of the largest singular value) of the sources' field at 392 check
points on a sphere of radius 2.5 r_e.  Outside, the two fields must agree: this pins the parameters
the treecode uses (separation 3 r_e by default) against the accuracy it claims, 1e-6 relative at the
default separation and better further out, for the Laplace and the Stokeslet kernel, and shows that
the fitted strengths are not amplified (their size is that of the sources).
"""

import numpy as np
import pytest

NE, NC, CHECK, RATIO = 196, 392, 2.5, 0.83


def fibonacci(n):
    """Unit vectors z_i = 1 - (2i + 1)/n, phi_i = 2 pi i / Phi^2 (the lattice of the point sets)."""
    i = np.arange(n)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = 2.0 * np.pi * i / ((1.0 + np.sqrt(5.0)) / 2.0) ** 2
    rho = np.sqrt(1.0 - z * z)
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def kernel_matrix(x, y, d):
    """Field at x of unit sources at y: 1/r (d = 1) or the Stokeslet (I + r r^T / r^2) / r (d = 3),
    as a (len(x) d) x (len(y) d) matrix."""
    r = x[:, None, :] - y[None, :, :]
    dist = np.linalg.norm(r, axis=2)
    if d == 1:
        return 1.0 / dist
    G = np.eye(3)[None, None] / dist[..., None, None] + r[..., :, None] * r[..., None, :] / dist[..., None, None] ** 3
    return G.transpose(0, 2, 1, 3).reshape(len(x) * 3, len(y) * 3)


def fit_error(d, separation, seed=0, re=1.7):
    rng = np.random.default_rng(seed)
    # sources filling the ball of radius 0.83 r_e (node of radius re around the origin)
    ns = 600
    u = rng.standard_normal((ns, 3))
    src = u / np.linalg.norm(u, axis=1, keepdims=True) * (RATIO * re) * rng.random(ns)[:, None] ** (1 / 3)
    lam = rng.standard_normal(ns * d)
    eq = re * fibonacci(NE)
    chk = CHECK * re * fibonacci(NC)
    A = kernel_matrix(chk, eq, d)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    keep = s > 1e-12 * s[0]
    pinv = (Vt[keep].T / s[keep]) @ U[:, keep].T
    mu = pinv @ (kernel_matrix(chk, src, d) @ lam)
    # targets on a sphere at the separation, rotated off the lattices
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    tgt = separation * re * fibonacci(500) @ q.T
    exact = kernel_matrix(tgt, src, d) @ lam
    approx = kernel_matrix(tgt, eq, d) @ mu
    return float(np.linalg.norm(approx - exact) / np.linalg.norm(exact)), float(np.abs(mu).max() / np.abs(lam).max())


@pytest.mark.parametrize("d", [1, 3])
def test_equivalent_sources_reproduce_the_far_field(d):
    errs = {sep: fit_error(d, sep)[0] for sep in (3.0, 4.0, 6.0)}
    assert errs[3.0] < 1e-6, errs      # the default separation
    assert errs[4.0] < errs[3.0] and errs[6.0] < errs[4.0], errs  # decays with distance
    assert errs[6.0] < 1e-8, errs


@pytest.mark.parametrize("d", [1, 3])
def test_fitted_strengths_are_not_amplified(d):
    # the pseudo-inverse is ill-conditioned, but the data lie in its well-resolved range
    _, growth = fit_error(d, 3.0, seed=1)
    assert growth < 10.0, growth


def test_fit_is_exact_for_sources_on_the_equivalent_sphere():
    # sources at the equivalent points themselves: the fit recovers their field everywhere outside
    d, re = 3, 1.0
    eq = re * fibonacci(NE)
    chk = CHECK * re * fibonacci(NC)
    A = kernel_matrix(chk, eq, d)
    lam = np.random.default_rng(2).standard_normal(NE * d)
    mu = np.linalg.lstsq(A, A @ lam, rcond=1e-12)[0]
    tgt = 3.0 * re * fibonacci(300)
    assert np.linalg.norm(kernel_matrix(tgt, eq, d) @ (mu - lam)) < 1e-9 * np.linalg.norm(kernel_matrix(tgt, eq, d) @ lam)


def _pressure_matrix(x, y):
    """Pressure at x of unit Stokeslets at y: (r . lambda) / r^3 (times 1/(4 pi)), len(x) x 3 len(y)."""
    r = x[:, None, :] - y[None, :, :]
    dist = np.linalg.norm(r, axis=2)
    return (r / dist[..., None] ** 3).reshape(len(x), 3 * len(y))


def test_equivalent_sources_pressure_accuracy():
    """The pressure (a derivative of the velocity field) of the fitted equivalent Stokeslets: an order
    less accurate than the velocity at the default separation (1.2e-6 against 1.2e-7 at 3 r_e),
    tightening with distance (1.1e-7 at 4 r_e) -- what the treecode's mfs_evaluate_stress inherits
    from each node."""
    rng = np.random.default_rng(3)
    re, ns = 1.7, 600
    u = rng.standard_normal((ns, 3))
    src = u / np.linalg.norm(u, axis=1, keepdims=True) * (RATIO * re) * rng.random(ns)[:, None] ** (1 / 3)
    lam = rng.standard_normal(ns * 3)
    eq, chk = re * fibonacci(NE), CHECK * re * fibonacci(NC)
    A = kernel_matrix(chk, eq, 3)
    mu = np.linalg.lstsq(A, kernel_matrix(chk, src, 3) @ lam, rcond=1e-12)[0]
    errs = {}
    for sep in (3.0, 4.0):
        tgt = sep * re * fibonacci(400)
        exact = _pressure_matrix(tgt, src) @ lam
        errs[sep] = float(np.linalg.norm(_pressure_matrix(tgt, eq) @ mu - exact) / np.linalg.norm(exact))
    assert errs[3.0] < 5e-6 and errs[4.0] < 5e-7, errs
