"""Tensor-core one-body apply (tcgen05 TF32 GEMMs on operand pieces) against the FP64 oracle.

tensor_cores = 1 (three TF32 pieces, six products: FP32-level products) meets the bars of the
CUDA-core path: the apply is backward stable to 1e-5 on a smooth field (Eq. pseudo), the matvec
is within 1e-6 and solved velocities within 1e-5 (relative 2-norms).  tensor_cores = 2 (two
pieces, three products: 3xTF32, products to ~2^-21) is held to 3e-5 and 3e-6 on the first two
and to the same 1e-5 on solutions.
Sizes are ragged for the GEMM tiles: K = dM not a multiple of 32 (zero-padded K), factor rows
dN not a multiple of 128, column counts (bodies x rhs) not a multiple of 16 and above 256 (two
column tiles, the second ragged).
"""

import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import Problem  # noqa: E402

from test_gpu_parity import _ctx, _mixed, _rel, _seg  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sphere100_mobility_oracle.json")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _backward_err(pr, bodies, lam, gam):
    """max over bodies of |S_L^(k) (lambda_k - lambda_k,oracle)| / |gamma_k| (Eq. pseudo)."""
    got = pr.split(bodies, lam, on="proxy")
    g = pr.split(bodies, gam)
    worst = 0.0
    for k in bodies:
        ref = pr.pinv_apply(k, g[k], project=False)
        f = pr.shape_of(k)
        diff = pr.rotate_points(k, f.SL @ pr.rotate_points(k, got[k] - ref, True), False)
        worst = max(worst, np.linalg.norm(diff) / np.linalg.norm(g[k]))
    return worst


BACKWARD_TOL = {1: 1e-5, 2: 3e-5}
MATVEC_TOL = {1: 1e-6, 2: 3e-6}


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("kind", ["stokes", "laplace"])
@pytest.mark.parametrize("P,m,n,nrhs", [(7, 150, 75, 1), (7, 150, 75, 3), (150, 64, 30, 4)])
def test_tc_apply_backward_stable(kind, P, m, n, nrhs, mode):
    wl = _mixed(kind, P=P, m=m, n=n, seed=31)
    ctx = _ctx(wl, tensor_cores=mode)
    pr = Problem(wl)
    rng = np.random.default_rng(7)
    bodies = list(range(pr.P))
    gams = []
    for _ in range(nrhs):  # smooth fields: what the other bodies induce on each body
        lam_rand = [rng.standard_normal(pr.Y[k].shape[0] * pr.d) for k in bodies]
        gams.append(np.concatenate(pr.pair_sum(bodies, lam_rand, include_self=False)))
    gam = np.stack(gams).reshape(nrhs, -1, pr.d)
    lam = ctx.precond_apply(torch.tensor(gam, device="cuda"), project=False).cpu().numpy().reshape(nrhs, -1)
    for h in range(nrhs):
        assert _backward_err(pr, bodies, lam[h], gam[h].reshape(-1)) < BACKWARD_TOL[mode]
    # projected apply: zero net charge / force and torque on every body (Sec. 3.3)
    lamp = ctx.precond_apply(torch.tensor(gam, device="cuda"), project=True).cpu().numpy().reshape(nrhs, -1)
    for h in range(nrhs):
        for k, lk in zip(bodies, pr.split(bodies, lamp[h], on="proxy")):
            if kind == "stokes":
                assert np.abs(pr.K_N(k).T @ lk).max() < 1e-5 * np.abs(lk).sum()
            else:
                assert abs(lk.sum()) < 1e-5 * np.abs(lk).sum()
    ctx.close()


def test_tc_apply_agrees_with_cuda_core_apply():
    """Both FP32 applies approximate the same FP64 apply: on white noise they agree to the FP32 level."""
    wl = _mixed("stokes", P=9, m=150, n=75, seed=32)
    a, b = _ctx(wl, tensor_cores=1), _ctx(wl, tensor_cores=0)
    gam = torch.tensor(np.random.default_rng(8).standard_normal((2, a.sum_M, 3)), device="cuda")
    for project in (True, False):
        la = a.precond_apply(gam, project=project).cpu().numpy()
        lb = b.precond_apply(gam, project=project).cpu().numpy()
        assert np.isfinite(la).all()
        # forward differences follow the one-body condition number; bounded well away from O(1)
        assert _rel(la, lb) < 1e-2
    a.close()
    b.close()


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("kind", ["stokes", "laplace"])
@pytest.mark.parametrize("nrhs", [1, 4])
def test_tc_matvec(kind, nrhs, mode):
    wl = _mixed(kind, nsusp=2)
    ctx = _ctx(wl, tensor_cores=mode)
    pr = Problem(wl)
    gam = np.random.default_rng(5).standard_normal((nrhs, ctx.sum_M, pr.d))
    y = ctx.matvec(torch.tensor(gam, device="cuda")).cpu().numpy()
    for h in range(nrhs):
        ref = np.concatenate([pr.matvec(list(pr.suspension_bodies(s)),
                                        gam[h].reshape(-1)[_seg(pr, list(pr.suspension_bodies(s)), "colloc")])
                              for s in range(wl.num_suspensions)])
        assert _rel(y[h].reshape(-1), ref) < MATVEC_TOL[mode]
    ctx.close()


def test_tc_solve_mobility_small():
    wl = _mixed("stokes")
    ctx = _ctx(wl, tensor_cores=1)
    pr = Problem(wl)
    U, W, info = ctx.solve_mobility(torch.tensor(wl.F[:1], device="cuda"), torch.tensor(wl.T[:1], device="cuda"))
    Ur, Wr, _ = pr.solve_mobility(wl.F[0], wl.T[0], tol=1e-12)
    got = np.concatenate([U.cpu().numpy()[0], W.cpu().numpy()[0]], axis=1)
    assert _rel(got, np.concatenate([Ur, Wr], axis=1)) < 1e-5
    assert info.converged
    ctx.close()


def test_tc_solve_elastance_small():
    wl = _mixed("laplace")
    ctx = _ctx(wl, tensor_cores=1)
    pr = Problem(wl)
    V, info = ctx.solve_elastance(torch.tensor(wl.Q[None], device="cuda"))
    phi, _ = pr.solve_elastance(wl.Q, tol=1e-12)
    assert _rel(V.cpu().numpy()[0], phi) < 1e-5
    assert info.converged
    ctx.close()


@pytest.mark.parametrize("mode", [1, 2])
def test_tc_sphere100_mobility_matches_oracle(mode):
    """The benchmark geometry (100 spheres, M = 1200, N = 600) against the stored FP64 oracle solve."""
    from mfs_inputs import make_workload
    from paper_2409_04215_gb300 import MFS

    g = json.load(open(GOLDEN))
    ref = np.concatenate([np.array(g["U"]), np.array(g["Omega"])], axis=1)
    wl = make_workload("sphere100_mobility")
    ctx = MFS.from_workload(wl, tensor_cores=mode)
    U, W, info = ctx.solve_mobility(torch.tensor(wl.F, device="cuda"), torch.tensor(wl.T, device="cuda"))
    got = np.concatenate([U.cpu().numpy()[0], W.cpu().numpy()[0]], axis=1)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert info.converged
    assert err < 1e-5, f"relative error {err:.3e}"
    ctx.close()
