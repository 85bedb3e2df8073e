"""GPU parity on triaxial (Type T) ellipsoids (Sec. 4.2): a small cluster against oracle solves, and the
5000-body cluster's matvec on sampled target bodies against the oracle's direct sums."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from mfs_inputs.workloads import ellipsoid_cluster, make_workload  # noqa: E402
from oracle import Problem  # noqa: E402

from test_gpu_parity import _ctx, _rel  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def test_type_t_cluster_mobility_and_resistance():
    wl = ellipsoid_cluster(count=6, n_v=16, seed=3, name="typeT6")
    ctx = _ctx(wl)
    pr = Problem(wl)
    U, W, info = ctx.solve_mobility(wl.F, wl.T)
    Ur, Wr, _ = pr.solve_mobility(wl.F[0], wl.T[0], tol=1e-12)
    assert info.converged
    assert _rel(np.concatenate([U.numpy()[0], W.numpy()[0]], 1), np.concatenate([Ur, Wr], 1)) < 1e-5
    V = np.random.default_rng(5).standard_normal((2, 6, 3))
    F, T, info = ctx.solve_resistance(V[:1], V[1:])
    Fr, Tr, _ = pr.solve_resistance(V[0], V[1], tol=1e-12)
    assert info.converged
    assert _rel(np.concatenate([F.numpy()[0], T.numpy()[0]], 1), np.concatenate([Fr, Tr], 1)) < 1e-5
    ctx.close()


def test_type_t_5000_matvec_sampled():
    """5000 Type T ellipsoids, N_v = 34 (M = 839, N = 660): the matvec of Eq. 2esysprec on the first
    Krylov direction, three sampled target bodies against the oracle's sums over all 4999 sources."""
    wl = make_workload("ellipsoidT5000_mobility")
    ctx = _ctx(wl, max_iter=60, restart=60)
    pr = Problem(wl)
    rng = np.random.default_rng(8)
    bodies = list(range(pr.P))
    # a smooth surface field: rigid motions of every body (the data of a resistance problem)
    V = rng.standard_normal((pr.P, 6))
    gam = np.concatenate([pr.K_M(k) @ V[k] for k in bodies])
    y = ctx.matvec(torch.tensor(gam.reshape(1, -1, 3), device="cuda")).cpu().numpy().reshape(-1)
    g = pr.split(bodies, gam)
    sample = [0, 2500, 4999]
    lam_hat = [pr.pinv_apply(k, gk, project=True) for k, gk in zip(bodies, g)]
    ref = pr.pair_sum(bodies, lam_hat, include_self=False, target_bodies=sample)
    got = pr.split(bodies, y)
    num = sum(np.sum((got[k] - g[k] - r) ** 2) for k, r in zip(sample, ref))
    den = sum(np.sum((g[k] + r) ** 2) for k, r in zip(sample, ref))
    assert np.sqrt(num / den) < 1e-6
    ctx.close()
