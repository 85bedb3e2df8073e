"""Accuracy of the matvec of Eq. 2esysprec on the vectors GMRES applies it to and on rough vectors.

The FP32 pair kernel evaluates each pair term to about eps_32 of its size, so the error of the
off-diagonal sum is about eps_32 |lambda_hat| (lambda_hat = (I - L) S_L^+ gamma, Eq. pseudo), not
eps_32 |y|.  On the first Krylov direction of a solve (the completion right-hand side -u_0 of Eq.
stou0) |lambda_hat| is of the order of |y| and the FP32 matvec meets the 1e-6 bar by an order.  Rough
gamma excites the smallest singular values of S_L: |lambda_hat| / |y| is about 19 for white noise on
the six-sphere smoke geometry, and FP32 pair sums then lose 1.6e-6; later Krylov vectors, stripped of
their smooth part by the orthogonalisation, come close to that.  The compensated double-FP32 kernels
(precision = 3) carry every pair term as hi + lo and hold the matvec to 1e-7 on any of these (about
1e-8 measured on white noise).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from mfs_inputs import make_workload  # noqa: E402
from oracle import Problem  # noqa: E402

from test_gpu_parity import _ctx, _mixed, _rel, _seg  # noqa: E402

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _smoke_geometry():
    return make_workload("sphere100_mobility", count=6, m=240, n=120, seed=3)


def _oracle_matvec(pr, wl, gam):
    return np.concatenate([pr.matvec(list(pr.suspension_bodies(s)),
                                     gam[_seg(pr, list(pr.suspension_bodies(s)), "colloc")])
                           for s in range(wl.num_suspensions)])


def _krylov_basis(pr, b, k):
    """Orthonormal Arnoldi basis v_0..v_{k-1} of the oracle's operator from b (Algorithm 1 SOLVE)."""
    bodies = list(range(pr.P))
    V = [b / np.linalg.norm(b)]
    for _ in range(k - 1):
        w = pr.matvec(bodies, V[-1])
        for _ in range(2):  # CGS2
            w = w - sum(np.dot(v, w) * v for v in V)
        V.append(w / np.linalg.norm(w))
    return V


def test_matvec_on_krylov_vectors():
    """The twelve Krylov vectors of a mobility solve.  The first, -u_0 / |u_0|, is smooth and the FP32
    path holds it to 1e-6 (8.6e-8 measured); orthogonalisation strips the smooth part from the later
    ones, whose FP32 error grows to about 1.3e-6 by the seventh, always within the per-pair rounding
    bound 4 eps_32 |lambda_hat| / |y|.  The compensated path (precision = 3) holds all of them to 1e-7."""
    wl = _smoke_geometry()
    pr = Problem(wl)
    ctx = _ctx(wl)
    ctx3 = _ctx(wl, precision=3)
    bodies = list(range(pr.P))
    lam0 = [pr.lambda0(k, wl.F[0, k], wl.T[0, k]) for k in bodies]
    b = -np.concatenate(pr.pair_sum(bodies, lam0, include_self=True))
    for j, v in enumerate(_krylov_basis(pr, b, 12)):
        ref = pr.matvec(bodies, v)
        vt = torch.tensor(v.reshape(1, -1, 3), device="cuda")
        err = _rel(ctx.matvec(vt).cpu().numpy().reshape(-1), ref)
        err3 = _rel(ctx3.matvec(vt).cpu().numpy().reshape(-1), ref)
        lam_hat = np.concatenate([pr.pinv_apply(k, g, project=True) for k, g in zip(bodies, pr.split(bodies, v))])
        bound = 4.0 * EPS32 * np.linalg.norm(lam_hat) / np.linalg.norm(ref)
        assert err < bound, f"Krylov vector {j}: FP32 {err:.3e} above {bound:.3e}"
        if j == 0:
            assert err < 1e-6, f"first Krylov vector: FP32 {err:.3e}"
        assert err3 < 1e-7, f"Krylov vector {j}: compensated {err3:.3e}"
    ctx.close()
    ctx3.close()


def test_fp32_white_noise_error_follows_strength_size():
    """On white noise the FP32 error stays within a small multiple of eps_32 |lambda_hat| / |y| (the
    per-pair rounding of terms as large as the strengths), measured 1.5x."""
    wl = _smoke_geometry()
    pr = Problem(wl)
    ctx = _ctx(wl)
    bodies = list(range(pr.P))
    gam = np.random.default_rng(0).standard_normal(ctx.sum_M * 3)
    y = ctx.matvec(torch.tensor(gam.reshape(1, -1, 3), device="cuda")).cpu().numpy().reshape(-1)
    ref = pr.matvec(bodies, gam)
    lam_hat = np.concatenate([pr.pinv_apply(k, g, project=True) for k, g in zip(bodies, pr.split(bodies, gam))])
    bound = EPS32 * np.linalg.norm(lam_hat) / np.linalg.norm(ref)
    assert _rel(y, ref) < 4.0 * bound
    ctx.close()


@pytest.mark.parametrize("geom", ["smoke", "mixed_stokes", "mixed_laplace"])
@pytest.mark.parametrize("nrhs", [1, 4])
def test_compensated_matvec_white_noise(geom, nrhs):
    if geom == "smoke":
        wl = _smoke_geometry()
    else:
        wl = _mixed(geom.split("_")[1], nsusp=2)
    pr = Problem(wl)
    ctx = _ctx(wl, precision=3)
    d = pr.d
    gam = np.random.default_rng(7).standard_normal((nrhs, ctx.sum_M, d))
    y = ctx.matvec(torch.tensor(gam, device="cuda")).cpu().numpy()
    assert ctx.pair_variant(nrhs).startswith("Comp")
    for h in range(nrhs):
        err = _rel(y[h].reshape(-1), _oracle_matvec(pr, wl, gam[h].reshape(-1)))
        assert err < 1e-7, f"rhs {h}: {err:.3e}"
    ctx.close()


def test_compensated_pair_sum_right_hand_side():
    """u_0 over all pairs, self blocks included (Eq. stou0), with the compensated kernel."""
    wl = _mixed("stokes", nsusp=2)
    pr = Problem(wl)
    ctx = _ctx(wl, precision=3)
    s = np.random.default_rng(8).standard_normal((1, ctx.sum_N, 3))
    u = ctx.pair_sum(torch.tensor(s, device="cuda"), include_self=True).cpu().numpy()[0].reshape(-1)
    ref = []
    for sp in range(wl.num_suspensions):
        bs = list(pr.suspension_bodies(sp))
        ref.append(np.concatenate(pr.pair_sum(bs, pr.split(bs, s[0].reshape(-1)[_seg(pr, bs, "proxy")], on="proxy"),
                                              include_self=True)))
    assert _rel(u, np.concatenate(ref)) < 2e-8
    ctx.close()


def test_compensated_solve_mobility():
    """precision = 3 (compensated pairs, FP64 one-body apply, FP64 GMRES at 1e-11): the velocities
    agree with the oracle's to 1e-8, three orders below the FP32 path's 1e-5 bar."""
    wl = _mixed("stokes")
    pr = Problem(wl)
    ctx = _ctx(wl, precision=3, gmres_tol=1e-11)
    U, W, info = ctx.solve_mobility(wl.F[:1], wl.T[:1])
    Ur, Wr, _ = pr.solve_mobility(wl.F[0], wl.T[0], tol=1e-13)
    got = np.concatenate([U.numpy()[0], W.numpy()[0]], 1)
    assert info.converged
    assert _rel(got, np.concatenate([Ur, Wr], 1)) < 1e-8
    ctx.close()
