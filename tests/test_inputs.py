"""The seeded input generators: geometry is what the docstrings promise and seeds reproduce."""

import numpy as np

from mfs_inputs import fibonacci_sphere, grow_cluster, make_workload, rsa_in_cube, spheroid_lattice, spheroid_proxy


def test_fibonacci_sphere_on_radius():
    p = fibonacci_sphere(500, 0.7)
    np.testing.assert_allclose(np.linalg.norm(p, axis=1), 0.7, atol=1e-14)
    np.testing.assert_allclose(p.mean(axis=0), 0.0, atol=5e-3)


def test_spheroid_lattice_reduces_to_sphere_and_lies_on_surface():
    np.testing.assert_allclose(spheroid_lattice(300, 1.0, 1.0), fibonacci_sphere(300, 1.0), atol=1e-12)
    p = spheroid_lattice(800, 1.0, 2.0)
    np.testing.assert_allclose(p[:, 0] ** 2 + p[:, 1] ** 2 + p[:, 2] ** 2 / 4.0, 1.0, atol=1e-12)
    # area-uniform: the share of points above z = 0 is one half
    assert abs((p[:, 2] > 0).mean() - 0.5) < 2e-3


def test_spheroid_proxy_inside_at_offset():
    a, c, ds = 1.0, 2.0, 0.25
    y = spheroid_proxy(400, a, c, ds)
    x = spheroid_lattice(400, a, c)
    np.testing.assert_allclose(np.linalg.norm(x - y, axis=1), ds, atol=1e-12)
    assert np.all(y[:, 0] ** 2 + y[:, 1] ** 2 + y[:, 2] ** 2 / c**2 < 1.0)


def test_rsa_gaps():
    rng = np.random.default_rng(0)
    c = rsa_in_cube(rng, np.ones(60), 14.0, 0.1)
    d = np.linalg.norm(c[:, None] - c[None], axis=2) + 10 * np.eye(60)
    assert d.min() >= 2.1 - 1e-12
    assert c.min() >= 1.0 and c.max() <= 13.0


def test_grow_cluster_gaps():
    rng = np.random.default_rng(1)
    c = grow_cluster(rng, 80, 2.0, 0.05, 0.5)
    d = np.linalg.norm(c[:, None] - c[None], axis=2) + 100 * np.eye(80)
    assert d.min() >= 4.05 - 1e-9
    # every grown body touches (at its own gap <= 0.5) at least one earlier body
    for b in range(1, 80):
        assert d[b, :b].min() <= 4.5 + 1e-9


def test_workloads_are_seeded():
    a = make_workload("sphere100_mobility", count=20, m=60, n=30)
    b = make_workload("sphere100_mobility", count=20, m=60, n=30)
    np.testing.assert_array_equal(a.centres, b.centres)
    np.testing.assert_array_equal(a.F, b.F)
    w = make_workload("batched256_mobility", num_suspensions=6, m=60, n=30)
    assert w.num_suspensions == 6 and w.F.shape == (4, w.num_bodies, 3)
    assert np.all(np.diff(w.body_offsets) >= 2) and np.all(np.diff(w.body_offsets) <= 64)
    c = make_workload("two_sphere_elastance")
    assert c.off_diagonal_pairs() == 2 * 600 * 300


def test_ellipsoid_gap_closed_forms_and_brute_force():
    from mfs_inputs.geometry import (ellipsoid_gap, ellipsoid_shape_matrices, quaternion_rotations,
                                     random_quaternions)

    # spheres: |d| - r_A - r_B
    f, _ = ellipsoid_gap(np.array([[3.0, 1.0, 0.0]]), np.eye(3)[None], 0.25 * np.eye(3)[None])
    assert abs(f[0] - (np.sqrt(10.0) - 1.5)) < 1e-13
    # (1,1,2) spheroids with parallel axes: tip to tip and side by side
    Q = np.diag([1.0, 1.0, 4.0])[None]
    assert abs(ellipsoid_gap(np.array([[0.0, 0.0, 4.3]]), Q, Q)[0][0] - 0.3) < 1e-13
    assert abs(ellipsoid_gap(np.array([[2.2, 0.0, 0.0]]), Q, Q)[0][0] - 0.2) < 1e-13
    # rotated: at least the closest pair of densely sampled surface points, and within their spacing
    rng = np.random.default_rng(0)
    q = random_quaternions(rng, 2)
    QQ = ellipsoid_shape_matrices(q, (1.0, 1.0, 2.0))
    d = np.array([[2.5, 1.0, 0.7]])
    f, n = ellipsoid_gap(d, QQ[0][None], QQ[1][None])
    R = quaternion_rotations(q)
    u = rng.standard_normal((100000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    ax = np.array([1.0, 1.0, 2.0])
    pa, pb = (u * ax) @ R[0].T, d[0] + (u * ax) @ R[1].T
    # the supporting planes with normal n: the gap is the slab between them (sampled surfaces reach
    # the planes up to the sampling error)
    slab = float((pb @ n[0]).min() - (pa @ n[0]).max())
    assert f[0] - 1e-12 <= slab < f[0] + 1e-4
    best = min(np.linalg.norm(pb - p, axis=1).min() for p in pa[::50])
    assert f[0] <= best + 1e-12 and best - f[0] < 0.02


def test_spheroid_cluster_true_surface_gaps():
    """The 1000-spheroid cluster (first 150 bodies): every body after the first has an earlier
    neighbour at surface gap in [0.05, 0.5], and no two bodies are closer than 0.05."""
    from mfs_inputs.geometry import ellipsoid_gap, ellipsoid_shape_matrices

    wl = make_workload("spheroid1000_mobility", count=150, m=60, n=30)
    Q = ellipsoid_shape_matrices(wl.quats, wl.shapes[0].semi_axes)
    i, j = np.triu_indices(wl.num_bodies, 1)
    near = np.linalg.norm(wl.centres[j] - wl.centres[i], axis=1) < 4.0 + 0.5
    gaps, _ = ellipsoid_gap(wl.centres[j[near]] - wl.centres[i[near]], Q[i[near]], Q[j[near]])
    assert gaps.min() > 0.05 - 1e-9
    for b in range(1, wl.num_bodies):
        mine = gaps[j[near] == b]
        assert mine.size and 0.05 - 1e-9 <= mine.min() <= 0.5 + 1e-9
