"""GPU adjoint (mfs_mobility_vjp) against the FP64 oracle adjoint and against finite differences.

Gradients of L = sum_k |U_k|^2 + 0.3 sum_k |Omega_k|^2 with respect to the body centres, forces
and torques: within 1e-4 (relative, max-norm) of the oracle's adjoint, and within 1e-4 of central
finite differences (h = 1e-6) of the GPU's FP64 reference solve (precision = 1, GMRES 1e-13), on
rotated mixed shapes, two suspensions and 1 or 2 right-hand sides (gradients summed over them).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from tests.test_gpu_parity import _mixed  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _loss_grads(U, W):
    return 2.0 * U, 0.6 * W


@pytest.mark.parametrize("tensor_cores", [1, 0])  # the transposed one-body apply on tcgen05 or CUDA cores
@pytest.mark.parametrize("nrhs", [1, 2])
def test_vjp_matches_oracle_adjoint(nrhs, tensor_cores):
    from oracle import Problem
    from paper_2409_04215_gb300 import MFS

    wl = _mixed("stokes", P=6, m=160, n=80, seed=31, nsusp=2)
    ctx = MFS.from_workload(wl, gmres_tol=1e-10, tensor_cores=tensor_cores)
    F = torch.tensor(wl.F[:nrhs], device="cuda")
    T = torch.tensor(wl.T[:nrhs], device="cuda")
    U, W, _ = ctx.solve_mobility(F, T)
    gU, gW = _loss_grads(U, W)
    dc, dF, dT = ctx.mobility_vjp(gU, gW, want_force_grads=True)
    pr = Problem(wl)
    ref_c = np.zeros((wl.num_bodies, 3))
    for h in range(nrhs):
        Ur, Wr, _ = pr.solve_mobility(wl.F[h], wl.T[h], tol=1e-13)
        gc, gF, gT = pr.mobility_vjp(wl.F[h], wl.T[h], 2.0 * Ur, 0.6 * Wr)
        ref_c += gc
        np.testing.assert_allclose(dF.cpu().numpy()[h], gF, rtol=0, atol=1e-4 * np.abs(gF).max())
        np.testing.assert_allclose(dT.cpu().numpy()[h], gT, rtol=0, atol=1e-4 * np.abs(gT).max())
    got = dc.cpu().numpy()
    assert np.abs(got - ref_c).max() <= 1e-4 * np.abs(ref_c).max()
    # translation invariance per suspension
    for s in range(wl.num_suspensions):
        b0, b1 = wl.body_offsets[s], wl.body_offsets[s + 1]
        assert np.abs(got[b0:b1].sum(axis=0)).max() <= 1e-4 * np.abs(ref_c).max()


def test_vjp_matches_finite_differences_of_fp64_gpu_solve():
    from paper_2409_04215_gb300 import MFS

    wl = _mixed("stokes", P=5, m=160, n=80, seed=32)
    F = torch.tensor(wl.F[:1], device="cuda")
    T = torch.tensor(wl.T[:1], device="cuda")
    ctx = MFS.from_workload(wl)
    U, W, _ = ctx.solve_mobility(F, T)
    dc = ctx.mobility_vjp(*_loss_grads(U, W))[0].cpu().numpy()
    ref = MFS.from_workload(wl, precision=1, gmres_tol=1e-13, autotune=0)

    def loss(c):
        ref.update_centers(c)
        u, w, _ = ref.solve_mobility(F, T)
        return float((u * u).sum() + 0.3 * (w * w).sum())

    rng = np.random.default_rng(3)
    h = 1e-6
    for _ in range(4):
        k, a = rng.integers(0, wl.num_bodies), rng.integers(0, 3)
        cp, cm = wl.centres.copy(), wl.centres.copy()
        cp[k, a] += h
        cm[k, a] -= h
        fd = (loss(cp) - loss(cm)) / (2 * h)
        assert abs(fd - dc[k, a]) <= 1e-4 * np.abs(dc).max(), (k, a, fd, dc[k, a])


def test_autograd_function():
    from paper_2409_04215_gb300 import MFS, mobility

    wl = _mixed("stokes", P=4, m=120, n=60, seed=33)
    ctx = MFS.from_workload(wl, gmres_tol=1e-10)
    c = torch.tensor(wl.centres, device="cuda", requires_grad=True)
    F = torch.tensor(wl.F[:1], device="cuda", requires_grad=True)
    T = torch.tensor(wl.T[:1], device="cuda", requires_grad=True)
    U, W = mobility(ctx, c, F, T)
    loss = (U * U).sum() + 0.3 * (W * W).sum()
    loss.backward()
    dc, dF, dT = ctx.mobility_vjp(2.0 * U.detach(), 0.6 * W.detach(), want_force_grads=True)
    np.testing.assert_allclose(c.grad.cpu().numpy(), dc.cpu().numpy(), rtol=1e-12, atol=0)
    np.testing.assert_allclose(F.grad.cpu().numpy(), dF.cpu().numpy(), rtol=1e-12, atol=0)
    assert T.grad is not None


@pytest.mark.parametrize("nrhs", [1, 2])
def test_vjp_fp64_path_matches_oracle_adjoint(nrhs):
    """precision = 1 runs the whole adjoint in FP64 (transposed sums, transposed one-body apply and
    the centre gradient as plain FP64 loops): gradients within 1e-8 of the oracle's adjoint, four
    orders below the FP32 path's bar."""
    from oracle import Problem
    from paper_2409_04215_gb300 import MFS

    wl = _mixed("stokes", P=6, m=160, n=80, seed=31, nsusp=2)
    ctx = MFS.from_workload(wl, precision=1, autotune=0, gmres_tol=1e-13)
    F = torch.tensor(wl.F[:nrhs], device="cuda")
    T = torch.tensor(wl.T[:nrhs], device="cuda")
    U, W, _ = ctx.solve_mobility(F, T)
    dc, dF, dT = ctx.mobility_vjp(*_loss_grads(U, W), want_force_grads=True)
    pr = Problem(wl)
    ref_c = np.zeros((wl.num_bodies, 3))
    for h in range(nrhs):
        Ur, Wr, _ = pr.solve_mobility(wl.F[h], wl.T[h], tol=1e-13)
        gc, gF, gT = pr.mobility_vjp(wl.F[h], wl.T[h], 2.0 * Ur, 0.6 * Wr)
        ref_c += gc
        np.testing.assert_allclose(dF.cpu().numpy()[h], gF, rtol=0, atol=1e-8 * np.abs(gF).max())
        np.testing.assert_allclose(dT.cpu().numpy()[h], gT, rtol=0, atol=1e-8 * np.abs(gT).max())
    assert np.abs(dc.cpu().numpy() - ref_c).max() <= 1e-8 * np.abs(ref_c).max()
    ctx.close()
