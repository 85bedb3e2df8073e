"""GPU parity of the Dirichlet problems (capacitance Sec. 2.1, resistance Sec. 2.2) against the oracle.

Same bars as the recompleted path: the one-body apply with the bare self block is backward stable to
1e-5 on a smooth field (Eq. pseudo), the matvec of Eq. 2sysprec is within 1e-6 and solved charges,
forces and torques within 1e-5 of the FP64 oracle (relative 2-norms); closed forms where physics fixes
the answer.  Both one-body applies (tensor cores and CUDA cores) and the FP64 path are covered.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from mfs_inputs.workloads import make_workload, sphere_shape  # noqa: E402
from oracle import Problem  # noqa: E402

from test_gpu_parity import _ctx, _mixed, _rel, _seg  # noqa: E402
from test_oracle_dirichlet import _cluster  # noqa: E402
from test_oracle_closed_forms import _single, _two_sphere_potential_bispherical  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


@pytest.mark.parametrize("tensor_cores", [0, 1])
@pytest.mark.parametrize("kind", ["stokes", "laplace"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_dirichlet_apply_backward_stable(kind, nrhs, tensor_cores):
    wl = _mixed(kind, seed=41)
    ctx = _ctx(wl, tensor_cores=tensor_cores)
    pr = Problem(wl)
    rng = np.random.default_rng(9)
    bodies = list(range(pr.P))
    gams = []
    for _ in range(nrhs):  # smooth fields: what the other bodies induce on each body
        a = [rng.standard_normal(pr.Y[k].shape[0] * pr.d) for k in bodies]
        gams.append(np.concatenate(pr.pair_sum(bodies, a, include_self=False)))
    gam = np.stack(gams).reshape(nrhs, -1, pr.d)
    alpha = ctx.dirichlet_apply(torch.tensor(gam, device="cuda")).cpu().numpy().reshape(nrhs, -1)
    for h in range(nrhs):
        got = pr.split(bodies, alpha[h], on="proxy")
        g = pr.split(bodies, gam[h].reshape(-1))
        for k in bodies:
            ref = pr.pinv_apply_dirichlet(k, g[k])
            S0 = pr.shape_of(k).S0
            diff = pr.rotate_points(k, S0 @ pr.rotate_points(k, got[k] - ref, True), False)
            assert np.linalg.norm(diff) < 1e-5 * np.linalg.norm(g[k])
    ctx.close()


@pytest.mark.parametrize("tensor_cores", [0, 1])
@pytest.mark.parametrize("kind", ["stokes", "laplace"])
@pytest.mark.parametrize("nrhs", [1, 4])
def test_dirichlet_matvec(kind, nrhs, tensor_cores):
    wl = _mixed(kind, nsusp=2)
    ctx = _ctx(wl, tensor_cores=tensor_cores)
    pr = Problem(wl)
    gam = np.random.default_rng(5).standard_normal((nrhs, ctx.sum_M, pr.d))
    y = ctx.dirichlet_matvec(torch.tensor(gam, device="cuda")).cpu().numpy()
    for h in range(nrhs):
        ref = np.concatenate([pr.matvec_dirichlet(list(pr.suspension_bodies(s)),
                                                  gam[h].reshape(-1)[_seg(pr, list(pr.suspension_bodies(s)), "colloc")])
                              for s in range(wl.num_suspensions)])
        assert _rel(y[h].reshape(-1), ref) < 1e-6
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-9)])
def test_solve_resistance_small(precision, tol):
    wl = _mixed("stokes", nsusp=2)
    ctx = _ctx(wl, precision=precision, gmres_tol=1e-7 if precision == 0 else 1e-12)
    pr = Problem(wl)
    rng = np.random.default_rng(12)
    U, W = rng.standard_normal((2, wl.num_bodies, 3)), rng.standard_normal((2, wl.num_bodies, 3))
    F, T, info = ctx.solve_resistance(torch.tensor(U, device="cuda"), torch.tensor(W, device="cuda"))
    assert info.converged
    for h in range(2):
        Fr, Tr, _ = pr.solve_resistance(U[h], W[h])
        got = np.concatenate([F.cpu().numpy()[h], T.cpu().numpy()[h]], axis=1)
        assert _rel(got, np.concatenate([Fr, Tr], axis=1)) < tol
    ctx.close()


def test_solve_capacitance_small():
    wl = _mixed("laplace", nsusp=2)
    ctx = _ctx(wl)
    pr = Problem(wl)
    phi = np.random.default_rng(13).standard_normal((3, wl.num_bodies))
    q, info = ctx.solve_capacitance(torch.tensor(phi, device="cuda"))
    assert info.converged
    for h in range(3):
        assert _rel(q.cpu().numpy()[h], pr.solve_capacitance(phi[h])[0]) < 1e-5
    ctx.close()


def test_closed_forms_on_gpu():
    """Isolated sphere q = 4 pi phi, f = 6 pi v, t = 8 pi omega; two spheres q = +-(c_s - c_m)."""
    ctx = _ctx(_single(sphere_shape(600, 300), "laplace"))
    q, _ = ctx.solve_capacitance(np.array([[1.0]]))
    assert abs(q.numpy()[0, 0] / (4 * np.pi) - 1) < 1e-6
    ctx.close()
    ctx = _ctx(_single(sphere_shape(600, 300), "stokes"))
    F, T, _ = ctx.solve_resistance(np.array([[[0.3, -0.2, 1.0]]]), np.array([[[0.5, 0.1, -0.7]]]))
    # relative 2e-6 of the largest component: FP32 pairs and TF32-piece apply
    np.testing.assert_allclose(F.numpy()[0, 0], 6 * np.pi * np.array([0.3, -0.2, 1.0]), rtol=0,
                               atol=2e-6 * 6 * np.pi)
    np.testing.assert_allclose(T.numpy()[0, 0], 8 * np.pi * np.array([0.5, 0.1, -0.7]), rtol=0,
                               atol=2e-6 * 8 * np.pi)
    ctx.close()
    ctx = _ctx(make_workload("two_sphere_elastance"))
    q, _ = ctx.solve_capacitance(np.array([[1.0, -1.0]]))
    c = 1.0 / _two_sphere_potential_bispherical(1.0, 2.5)
    assert abs(q.numpy()[0, 0] / c - 1) < 1e-6 and abs(q.numpy()[0, 1] / c + 1) < 1e-6
    ctx.close()


def test_two_way_error_gpu():
    """Eq. 2way on the GPU: resistance (R_p = 0.7) then mobility (proxy offset x 1.05) of 5 spheres, both
    solves compared with the oracle's, and the 2-way error itself with the oracle's."""
    res = _cluster("stokes", 5, sphere_shape(600, 300, rp=0.7), spacing=2.5)
    mob = _cluster("stokes", 5, sphere_shape(600, 300, rp=1 - 1.05 * 0.3), spacing=2.5)
    rng = np.random.default_rng(11)
    U_ref, W_ref = rng.standard_normal((5, 3)), rng.standard_normal((5, 3))
    cr, cm = _ctx(res), _ctx(mob)
    F, T, _ = cr.solve_resistance(U_ref[None], W_ref[None])
    U, W, _ = cm.solve_mobility(F, T)
    Fo, To, _ = Problem(res).solve_resistance(U_ref, W_ref)
    assert _rel(np.concatenate([F.numpy()[0], T.numpy()[0]], 1), np.concatenate([Fo, To], 1)) < 1e-5
    Uo, Wo, _ = Problem(mob).solve_mobility(Fo, To)
    # the round trip's velocities against the oracle's: the solve bar
    got = np.concatenate([U.numpy()[0], W.numpy()[0]], 1)
    assert _rel(got, np.concatenate([Uo, Wo], 1)) < 1e-5
    # Eq. 2way: the oracle's error here is 9.5e-6, a discretisation error only 5-10x above the FP32
    # path's own solution error (about 1e-6 per solve), so the FP32 path's value is held to twice the
    # oracle's bound (1e-5) and above the same-discretisation round trip; the compensated path
    # (precision = 3, below) reproduces the oracle's value itself
    ref = np.concatenate([U_ref, W_ref], axis=1)
    e_gpu = np.abs(got - ref).max() / np.abs(ref).max()
    assert e_gpu < 2e-5, e_gpu
    U2, W2, _ = cr.solve_mobility(F, T)  # the same discretisation both ways (inverse crime)
    crime = np.abs(np.concatenate([U2.numpy()[0], W2.numpy()[0]], 1) - ref).max() / np.abs(ref).max()
    assert crime < e_gpu, (crime, e_gpu)
    cr.close()
    cm.close()


def test_two_way_error_gpu_compensated():
    """Eq. 2way with compensated double-FP32 pair sums and the FP64 one-body apply (precision = 3):
    the GPU's 2-way error equals the oracle's to 1 % of its value."""
    res = _cluster("stokes", 5, sphere_shape(600, 300, rp=0.7), spacing=2.5)
    mob = _cluster("stokes", 5, sphere_shape(600, 300, rp=1 - 1.05 * 0.3), spacing=2.5)
    rng = np.random.default_rng(11)
    U_ref, W_ref = rng.standard_normal((5, 3)), rng.standard_normal((5, 3))
    cr, cm = _ctx(res, precision=3, gmres_tol=1e-11), _ctx(mob, precision=3, gmres_tol=1e-11)
    F, T, _ = cr.solve_resistance(U_ref[None], W_ref[None])
    U, W, _ = cm.solve_mobility(F, T)
    Fo, To, _ = Problem(res).solve_resistance(U_ref, W_ref)
    Uo, Wo, _ = Problem(mob).solve_mobility(Fo, To)
    ref = np.concatenate([U_ref, W_ref], axis=1)
    e_gpu = np.abs(np.concatenate([U.numpy()[0], W.numpy()[0]], 1) - ref).max() / np.abs(ref).max()
    e_orc = np.abs(np.concatenate([Uo, Wo], 1) - ref).max() / np.abs(ref).max()
    assert abs(e_gpu - e_orc) < 0.01 * e_orc, (e_gpu, e_orc)
    cr.close()
    cm.close()


def test_resistance_full_size_matches_oracle():
    """100 spheres, M = 1200 (the benchmark geometry): forces and torques of the resistance problem
    within 1e-5 of the stored FP64 oracle solution (tests/golden, GMRES tolerance 1e-12)."""
    import json
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sphere100_resistance_oracle.json")
    g = json.load(open(path))
    wl = make_workload("sphere100_mobility")
    ctx = _ctx(wl)
    rng = np.random.default_rng(14)
    U_ref, W_ref = rng.standard_normal((1, 100, 3)), rng.standard_normal((1, 100, 3))
    F, T, info = ctx.solve_resistance(torch.tensor(U_ref, device="cuda"), torch.tensor(W_ref, device="cuda"))
    assert info.converged
    ref = np.concatenate([np.array(g["F"]), np.array(g["T"])], axis=1)
    got = np.concatenate([F.cpu().numpy()[0], T.cpu().numpy()[0]], axis=1)
    assert _rel(got, ref) < 1e-5, _rel(got, ref)
    ctx.close()
