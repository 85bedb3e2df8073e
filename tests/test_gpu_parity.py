"""GPU parity: libmfs (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (relative 2-norm unless said otherwise): matvec <= 1e-6 and solved velocities /
potentials <= 1e-5 (the accuracy targets of the FP32 path); bare pair sums <= 1e-6; the FP64
reference path (precision = 1) <= 1e-11.  Sizes are ragged on purpose: N not a multiple of
4, M not a multiple of 32, tiles that straddle bodies, several suspensions, up to 4 rhs.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from mfs_inputs.workloads import Workload, make_workload, sphere_shape, spheroid_shape  # noqa: E402
from oracle import Problem  # noqa: E402
from oracle.mfs_oracle import split_workload  # noqa: E402


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module", autouse=True)
def _built():
    _need_gpu()
    import __graft_entry__

    __graft_entry__.build()


def _mixed(kind, P=7, m=150, n=75, seed=21, nsusp=1):
    rng = np.random.default_rng(seed)
    shapes = [sphere_shape(m, n), spheroid_shape(m + 10, n + 5, 1.0, 1.5, 0.3)]
    sid = (rng.random(P) < 0.5).astype(np.int32)
    quats = rng.standard_normal((P, 4))
    quats /= np.linalg.norm(quats, axis=1, keepdims=True)
    # bodies on a jittered lattice, 3.6 apart (gaps >= 0.3 for the 1.5 spheroids)
    side = int(np.ceil(P ** (1 / 3)))
    grid = np.array([(i, j, k) for i in range(side) for j in range(side) for k in range(side)], float)[:P]
    centres = 3.6 * grid + 0.05 * rng.standard_normal((P, 3))
    offs = np.linspace(0, P, nsusp + 1).round().astype(np.int32)
    wl = Workload("mixed", kind, shapes, centres, quats, sid, offs)
    wl.F = rng.standard_normal((4, P, 3))
    wl.T = rng.standard_normal((4, P, 3))
    wl.Q = rng.standard_normal(P)
    return wl


def _ctx(wl, **kw):
    from paper_2409_04215_gb300 import MFS

    return MFS.from_workload(wl, **kw)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _oracle_pair(pr, wl, strengths, include_self):
    out = []
    for s in range(wl.num_suspensions):
        bodies = list(pr.suspension_bodies(s))
        parts = pr.split(bodies, strengths[_seg(pr, bodies, "proxy")], on="proxy")
        out.append(np.concatenate(pr.pair_sum(bodies, parts, include_self)))
    return np.concatenate(out)


def _seg(pr, bodies, on):
    d = pr.d
    sizes = [(pr.X[k] if on == "colloc" else pr.Y[k]).shape[0] * d for k in range(pr.P)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    return slice(off[bodies[0]], off[bodies[-1] + 1])


@pytest.mark.parametrize("kind", ["stokes", "laplace"])
@pytest.mark.parametrize("include_self", [False, True])
@pytest.mark.parametrize("nrhs", [1, 2, 4])
def test_pair_sum(kind, include_self, nrhs):
    wl = _mixed(kind, nsusp=2)
    ctx = _ctx(wl)
    pr = Problem(wl)
    rng = np.random.default_rng(nrhs)
    d = pr.d
    s = rng.standard_normal((nrhs, ctx.sum_N, d))
    u = ctx.pair_sum(torch.tensor(s, device="cuda"), include_self=include_self).cpu().numpy()
    for h in range(nrhs):
        ref = _oracle_pair(pr, wl, s[h].reshape(-1), include_self)
        assert _rel(u[h].reshape(-1), ref) < 1e-6


@pytest.mark.parametrize("tensor_cores", [0, 1])
@pytest.mark.parametrize("kind", ["stokes", "laplace"])
@pytest.mark.parametrize("smooth", [True, False])
def test_precond_apply_backward(kind, smooth, tensor_cores):
    """S_L^(k) (lambda_gpu - lambda_oracle) is small: the FP32 two-step apply is backward stable (Eq. pseudo).

    smooth: gamma is the field that the other bodies induce on each body (what GMRES feeds the
    preconditioner); the backward error is then the FP32 accuracy of t = U^T g (eps_32 sqrt(dM),
    about 2e-6 here).  Otherwise gamma is white noise, the worst case, where the FP32 second
    step's rounding of the large high-frequency coefficients shows at the 1e-5 level.  Neither
    reaches the matvec at this size: the self block is replaced by the identity there
    (Eq. 2esysprec), and test_matvec holds the matvec to 1e-6.
    """
    wl = _mixed(kind)
    ctx = _ctx(wl, tensor_cores=tensor_cores)
    pr = Problem(wl)
    rng = np.random.default_rng(3)
    bodies = list(range(pr.P))
    if smooth:
        lam_rand = [rng.standard_normal(pr.Y[k].shape[0] * pr.d) for k in bodies]
        gam = np.concatenate(pr.pair_sum(bodies, lam_rand, include_self=False))
        tol = 1e-5
    else:
        gam = rng.standard_normal(ctx.sum_M * pr.d)
        tol = 1e-4
    lam = ctx.precond_apply(gam.reshape(-1, pr.d), project=False).cpu().numpy().reshape(-1)
    got = pr.split(bodies, lam, on="proxy")
    g = pr.split(bodies, gam)
    for k in bodies:
        ref = pr.pinv_apply(k, g[k], project=False)
        f = pr.shape_of(k)
        # S_L^(k) = R_M S_L^(0) R_N^T
        diff = pr.rotate_points(k, f.SL @ pr.rotate_points(k, got[k] - ref, True), False)
        assert np.linalg.norm(diff) < tol * np.linalg.norm(g[k])
    # projected apply: zero net charge / force and torque on every body (Sec. 3.3 item 2)
    lamp = ctx.precond_apply(gam.reshape(-1, pr.d), project=True).cpu().numpy().reshape(-1)
    for k, lk in zip(bodies, pr.split(bodies, lamp, on="proxy")):
        if kind == "stokes":
            assert np.abs(pr.K_N(k).T @ lk).max() < 1e-5 * np.abs(lk).sum()
        else:
            assert abs(lk.sum()) < 1e-5 * np.abs(lk).sum()


@pytest.mark.parametrize("tensor_cores", [0, 1])
@pytest.mark.parametrize("kind", ["stokes", "laplace"])
@pytest.mark.parametrize("nrhs", [1, 4])
def test_matvec(kind, nrhs, tensor_cores):
    wl = _mixed(kind, nsusp=2)
    ctx = _ctx(wl, tensor_cores=tensor_cores)
    pr = Problem(wl)
    rng = np.random.default_rng(5)
    gam = rng.standard_normal((nrhs, ctx.sum_M, pr.d))
    y = ctx.matvec(torch.tensor(gam, device="cuda")).cpu().numpy()
    for h in range(nrhs):
        ref = np.concatenate([pr.matvec(list(pr.suspension_bodies(s)),
                                        gam[h].reshape(-1)[_seg(pr, list(pr.suspension_bodies(s)), "colloc")])
                              for s in range(wl.num_suspensions)])
        assert _rel(y[h].reshape(-1), ref) < 1e-6


def test_matvec_host_buffers_match_device():
    wl = _mixed("stokes")
    ctx = _ctx(wl)
    gam = np.random.default_rng(6).standard_normal((1, ctx.sum_M, 3))
    y_host = ctx.matvec(gam).numpy()
    y_dev = ctx.matvec(torch.tensor(gam, device="cuda")).cpu().numpy()
    np.testing.assert_array_equal(y_host, y_dev)


def test_matvec_full_size_sampled():
    """100 spheres, M=1200, N=600 (the benchmark geometry): sampled target bodies against the oracle."""
    wl = make_workload("sphere100_mobility")
    ctx = _ctx(wl)
    pr = Problem(wl)
    bodies = list(range(pr.P))
    lam0 = [pr.lambda0(k, wl.F[0, k], wl.T[0, k]) for k in bodies]
    gam = -np.concatenate(pr.pair_sum(bodies, lam0, include_self=True))  # the first Krylov direction
    y = ctx.matvec(torch.tensor(gam.reshape(1, -1, 3), device="cuda")).cpu().numpy().reshape(-1)
    g = pr.split(bodies, gam)
    lam_hat = [pr.pinv_apply(k, gk, project=True) for k, gk in zip(bodies, g)]
    sample = [0, 37, 99]
    ref = pr.pair_sum(bodies, lam_hat, include_self=False, target_bodies=sample)
    got = pr.split(bodies, y)
    num = sum(np.sum((got[k] - g[k] - r) ** 2) for k, r in zip(sample, ref))
    den = sum(np.sum((g[k] + r) ** 2) for k, r in zip(sample, ref))
    assert np.sqrt(num / den) < 1e-6


def test_solve_mobility_small():
    wl = _mixed("stokes")
    ctx = _ctx(wl)
    pr = Problem(wl)
    U, W, info = ctx.solve_mobility(torch.tensor(wl.F[:1], device="cuda"), torch.tensor(wl.T[:1], device="cuda"))
    Ur, Wr, _ = pr.solve_mobility(wl.F[0], wl.T[0], tol=1e-12)
    got = np.concatenate([U.cpu().numpy()[0], W.cpu().numpy()[0]], axis=1)
    assert _rel(got, np.concatenate([Ur, Wr], axis=1)) < 1e-5
    assert info.converged and info.iters > 1
    # the autotuned pair-kernel policy is reported by name
    assert ctx.pair_variant(1).startswith(("PackedStokes", "Scalar<3,1,"))


def test_solve_mobility_host_buffers():
    wl = _mixed("stokes", seed=4)
    ctx = _ctx(wl)
    pr = Problem(wl)
    U, W, info = ctx.solve_mobility(wl.F[:1], wl.T[:1])  # NumPy in, CPU tensors out
    Ur, Wr, _ = pr.solve_mobility(wl.F[0], wl.T[0], tol=1e-12)
    assert U.device.type == "cpu"
    assert _rel(np.concatenate([U.numpy()[0], W.numpy()[0]], 1), np.concatenate([Ur, Wr], 1)) < 1e-5


def test_solve_elastance_two_spheres():
    from tests.test_oracle_closed_forms import _two_sphere_potential_bispherical

    wl = make_workload("two_sphere_elastance")
    ctx = _ctx(wl)
    V, info = ctx.solve_elastance(torch.tensor(wl.Q[None], device="cuda"))
    V = V.cpu().numpy()[0]
    phi, _ = Problem(wl).solve_elastance(wl.Q)
    assert _rel(V, phi) < 1e-5
    v = _two_sphere_potential_bispherical(1.0, 2.5)
    assert abs(V[0] - v) < 1e-6 * v and abs(V[1] + v) < 1e-6 * v


def test_solve_elastance_cluster():
    wl = _mixed("laplace")
    ctx = _ctx(wl)
    V, _ = ctx.solve_elastance(wl.Q[None])
    phi, _ = Problem(wl).solve_elastance(wl.Q, tol=1e-12)
    assert _rel(V.numpy()[0], phi) < 1e-5


def test_batched_suspensions_four_rhs():
    """Independent suspensions (one of a single body) with 4 rhs each iterate as separate GMRES lanes."""
    wl = make_workload("batched256_mobility", num_suspensions=5, p_lo=1, p_hi=6, m=120, n=60, seed=9)
    ctx = _ctx(wl)
    U, W, info = ctx.solve_mobility(torch.tensor(wl.F, device="cuda"), torch.tensor(wl.T, device="cuda"))
    U, W = U.cpu().numpy(), W.cpu().numpy()
    assert info.lanes == 4 * wl.num_suspensions
    for s in range(wl.num_suspensions):
        sub = split_workload(wl, s)
        pr = Problem(sub)
        b0, b1 = wl.body_offsets[s], wl.body_offsets[s + 1]
        for h in range(4):
            Ur, Wr, _ = pr.solve_mobility(sub.F[h], sub.T[h], tol=1e-12)
            got = np.concatenate([U[h, b0:b1], W[h, b0:b1]], 1)
            assert _rel(got, np.concatenate([Ur, Wr], 1)) < 1e-5


def test_single_body_and_zero_rhs():
    wl = Workload("one", "stokes", [sphere_shape(200, 100)], np.zeros((1, 3)), None, np.zeros(1, np.int32),
                  np.array([0, 1], np.int32))
    ctx = _ctx(wl)
    g = np.random.default_rng(1).standard_normal((1, ctx.sum_M, 3))
    y = ctx.matvec(g).numpy()
    np.testing.assert_array_equal(y, g)  # no off-diagonal pairs: the identity
    U, W, info = ctx.solve_mobility(np.zeros((1, 1, 3)), np.zeros((1, 1, 3)))
    assert np.all(U.numpy() == 0) and np.all(W.numpy() == 0) and info.converged
    F, T = np.array([[0.0, 0.0, 1.0]]), np.array([[0.0, 0.5, 0.0]])
    U, W, _ = ctx.solve_mobility(F[None], T[None])
    Ur, Wr, _ = Problem(wl).solve_mobility(F, T, tol=1e-12)
    # FP32 rounding of u_0 passes through the recovery S_L^+ (about 1e-6 here): the solution tolerance
    assert _rel(np.concatenate([U.numpy()[0], W.numpy()[0]]), np.concatenate([Ur, Wr])) < 1e-5
    # the closed forms hold to the discretisation error of M=200, N=100 (about 4e-5)
    assert abs(U.numpy()[0, 0, 2] * 6 * np.pi - 1) < 1e-4
    assert abs(W.numpy()[0, 0, 1] * 8 * np.pi / 0.5 - 1) < 1e-4


def test_fp64_reference_path():
    wl = _mixed("stokes", nsusp=2)
    ctx = _ctx(wl, precision=1)
    pr = Problem(wl)
    gam = np.random.default_rng(8).standard_normal((1, ctx.sum_M, 3))
    y = ctx.matvec(gam).numpy().reshape(-1)
    ref = np.concatenate([pr.matvec(list(pr.suspension_bodies(s)),
                                    gam.reshape(-1)[_seg(pr, list(pr.suspension_bodies(s)), "colloc")])
                          for s in range(wl.num_suspensions)])
    assert _rel(y, ref) < 1e-11


def test_invalid_arguments_are_reported():
    from paper_2409_04215_gb300 import MFS, MFSError

    wl = _mixed("stokes")
    ctx = _ctx(wl)
    with pytest.raises(MFSError) as e:
        ctx.solve_elastance(np.ones((1, wl.num_bodies)))
    assert e.value.status == 1
    with pytest.raises(MFSError):
        MFS("stokes", np.array([[0.0, 0, 0]]), [(np.zeros((4, 3)), np.zeros((2, 3)))])  # M < N
    with pytest.raises(MFSError):
        MFS("stokes", np.array([[np.nan, 0, 0]]), [(wl.shapes[0].proxy, wl.shapes[0].colloc)])


def test_not_converged_is_reported():
    wl = _mixed("stokes")
    ctx = _ctx(wl, max_iter=2, restart=2, gmres_tol=1e-14)
    U, W, info = ctx.solve_mobility(wl.F[:1], wl.T[:1], allow_not_converged=True)
    assert info.status == 4 and not info.converged and info.iters == 2
    assert np.all(np.isfinite(U.numpy()))


@pytest.mark.parametrize("kind", ["stokes", "laplace"])
def test_update_centers_matches_fresh_context(kind):
    """mfs_update_centers moves the bodies and keeps the one-body factors (Remark congruent): a context
    moved to new centres (the bodies shuffled over the lattice and shifted) solves exactly as a context
    set up there (same pair-kernel policy, bit for bit), twice in a row, and within the bar of the
    oracle's solve at the new positions."""
    import copy

    wl = _mixed(kind, P=8, nsusp=1, seed=44)
    ctx = _ctx(wl, autotune=0)
    rng = np.random.default_rng(45)
    for step in range(2):
        moved = copy.copy(wl)
        moved.centres = wl.centres[rng.permutation(wl.num_bodies)] + rng.standard_normal(3)
        ctx.update_centers(moved.centres)
        fresh = _ctx(moved, autotune=0)
        if kind == "stokes":
            F, T = torch.tensor(wl.F[:1], device="cuda"), torch.tensor(wl.T[:1], device="cuda")
            a = torch.cat(ctx.solve_mobility(F, T)[:2], -1).cpu().numpy()
            b = torch.cat(fresh.solve_mobility(F, T)[:2], -1).cpu().numpy()
            Ur, Wr, _ = Problem(moved).solve_mobility(wl.F[0], wl.T[0], tol=1e-12)
            ref = np.concatenate([Ur, Wr], axis=1)
        else:
            Q = torch.tensor(wl.Q[None], device="cuda")
            a = ctx.solve_elastance(Q)[0].cpu().numpy()
            b = fresh.solve_elastance(Q)[0].cpu().numpy()
            ref = Problem(moved).solve_elastance(wl.Q, tol=1e-12)[0]
        assert np.array_equal(a, b), step
        assert _rel(a.reshape(ref.shape), ref) < 1e-5, step
        fresh.close()
    ctx.close()
