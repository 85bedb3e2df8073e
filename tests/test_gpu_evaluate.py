"""GPU parity of mfs_evaluate (the field of the last solve at arbitrary points: Eq. rep, Eq. repS with the
strengths of Eq. multirep, Eq. erepK or Eq. reconbal) against the oracle's direct FP64 evaluation.

Bar: relative 2-norm 2e-6 over the points for the FP32 path (the GPU solve's 1e-7 GMRES tolerance and
its FP32 sums both enter), 1e-10 for the FP64 path.  The points are random exterior points and points
on the body surfaces, with owners given explicitly or chosen as the nearest body.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from mfs_inputs.workloads import make_workload, sphere_shape  # noqa: E402
from oracle import Problem  # noqa: E402

from test_gpu_parity import _ctx, _mixed, _rel  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _points(wl, pr, rng, n_ext=300):
    """Exterior points around the bodies and a subset of each body's surface nodes, with owner bodies."""
    pts, own = [], []
    lo, hi = wl.centres.min(0) - 2.0, wl.centres.max(0) + 2.0
    while len(pts) < n_ext:
        x = rng.uniform(lo, hi)
        d = np.linalg.norm(wl.centres - x, axis=1)
        if d.min() > 1.8:  # outside every body (semi-axes <= 1.5 here)
            pts.append(x)
            own.append(int(np.argmin(d)))
    for k in range(wl.num_bodies):
        X = pr.X[k][::7]  # a subset of the surface nodes
        pts.extend(list(X))
        own.extend([k] * X.shape[0])
    return np.array(pts), np.array(own, np.int32)


def _oracle_field(pr, wl, strengths_of, pts, own):
    out = np.zeros((pts.shape[0], pr.d))
    for s in range(wl.num_suspensions):
        bodies = list(pr.suspension_bodies(s))
        sel = np.isin(own, bodies)
        if sel.any():
            out[sel] = pr.evaluate(bodies, strengths_of(s, bodies), pts[sel]).reshape(-1, pr.d)
    return out


@pytest.mark.parametrize("precision,tol", [(0, 2e-6), (1, 1e-10)])
def test_evaluate_after_mobility(precision, tol):
    wl = _mixed("stokes", nsusp=2)
    ctx = _ctx(wl, precision=precision, gmres_tol=1e-7 if precision == 0 else 1e-13)
    pr = Problem(wl)
    F, T = torch.tensor(wl.F[:2], device="cuda"), torch.tensor(wl.T[:2], device="cuda")
    U, W, _ = ctx.solve_mobility(F, T)
    pts, own = _points(wl, pr, np.random.default_rng(1))
    u = ctx.evaluate(torch.tensor(pts, device="cuda"), own, nrhs=2).cpu().numpy()
    for h in range(2):
        _, _, info = pr.solve_mobility(wl.F[h], wl.T[h], tol=1e-13)  # one GMRES result per suspension
        ref = _oracle_field(pr, wl, lambda s, b: pr.total_strengths_mobility(b, info[s].x, wl.F[h], wl.T[h]),
                            pts, own)
        assert _rel(u[h], ref) < tol
    ctx.close()


def test_evaluate_after_elastance_with_nearest_owner():
    wl = _mixed("laplace")
    ctx = _ctx(wl)
    pr = Problem(wl)
    ctx.solve_elastance(torch.tensor(wl.Q[None], device="cuda"))
    pts, _ = _points(wl, pr, np.random.default_rng(2))
    u = ctx.evaluate(pts).numpy()[0]  # owners: nearest body
    _, info = pr.solve_elastance(wl.Q, tol=1e-13)
    bodies = list(range(wl.num_bodies))
    ref = pr.evaluate(bodies, pr.total_strengths_elastance(bodies, info[0].x, wl.Q), pts)
    assert _rel(u[:, 0], ref) < 2e-6
    ctx.close()


@pytest.mark.parametrize("kind", ["stokes", "laplace"])
def test_evaluate_after_dirichlet_solves(kind):
    wl = _mixed(kind)
    ctx = _ctx(wl)
    pr = Problem(wl)
    rng = np.random.default_rng(3)
    bodies = list(range(wl.num_bodies))
    pts, own = _points(wl, pr, rng)
    if kind == "stokes":
        V, Om = rng.standard_normal((wl.num_bodies, 3)), rng.standard_normal((wl.num_bodies, 3))
        ctx.solve_resistance(V[None], Om[None])
        _, _, info = pr.solve_resistance(V, Om, tol=1e-13)
    else:
        phi = rng.standard_normal(wl.num_bodies)
        ctx.solve_capacitance(phi[None])
        _, info = pr.solve_capacitance(phi, tol=1e-13)
    u = ctx.evaluate(pts, own).numpy()[0]
    ref = pr.evaluate(bodies, pr.strengths_dirichlet(bodies, info[0].x), pts).reshape(-1, pr.d)
    assert _rel(u, ref) < 2e-6
    ctx.close()


def test_evaluate_errors():
    from paper_2409_04215_gb300 import MFSError

    wl = _mixed("stokes", nsusp=2)
    ctx = _ctx(wl)
    pts = np.array([[10.0, 0.0, 0.0]])
    with pytest.raises(MFSError):  # no solve yet
        ctx.evaluate(pts, [0])
    ctx.solve_mobility(wl.F[:1], wl.T[:1])
    with pytest.raises(MFSError):  # several suspensions need owners
        ctx.evaluate(pts)
    with pytest.raises(MFSError):  # owner out of range
        ctx.evaluate(pts, [wl.num_bodies])
    with pytest.raises(MFSError):  # nrhs differs from the solve's
        ctx.evaluate(pts, [0], nrhs=2)
    ctx.close()


def test_surface_residual_full_size():
    """The benchmark geometry (100 spheres, M = 1200): Eq. residual of the GPU solution on a 4800-point
    lattice of 5 of the spheres is at the discretisation level (parity of the evaluation itself is held
    by the small cases above)."""
    wl = make_workload("sphere100_mobility")
    ctx = _ctx(wl)
    U, W, _ = ctx.solve_mobility(torch.tensor(wl.F, device="cuda"), torch.tensor(wl.T, device="cuda"))
    fine = sphere_shape(4800, 600).colloc
    sample = [0, 33, 66, 99, 50]
    pts = np.concatenate([wl.centres[k] + fine for k in sample])
    own = np.repeat(np.array(sample, np.int32), fine.shape[0])
    u = ctx.evaluate(torch.tensor(pts, device="cuda"), own).cpu().numpy()[0]
    Uh, Wh = U.cpu().numpy()[0], W.cpu().numpy()[0]
    g = np.concatenate([Uh[k] + np.cross(Wh[k], fine) for k in sample])
    eps = np.linalg.norm(u - g, axis=1) / np.linalg.norm(g, axis=1)
    # M = 1200 spheres at gaps >= 0.1: a discretisation-level residual, far below O(1)
    assert eps.max() < 1e-2 and np.sqrt(np.mean(eps**2)) < 1e-3
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(0, 2e-6), (1, 1e-10)])
def test_stress_after_resistance_and_mobility(precision, tol):
    """Pressure and traction (Eq. traction) at surface and exterior points against the oracle's sums."""
    wl = _mixed("stokes", nsusp=2)
    ctx = _ctx(wl, precision=precision, gmres_tol=1e-7 if precision == 0 else 1e-13)
    pr = Problem(wl)
    pts, own = _points(wl, pr, np.random.default_rng(6), n_ext=100)
    nrm = np.random.default_rng(7).standard_normal(pts.shape)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    rng = np.random.default_rng(8)
    V, Om = rng.standard_normal((1, wl.num_bodies, 3)), rng.standard_normal((1, wl.num_bodies, 3))
    ctx.solve_resistance(V, Om)
    p, T = ctx.evaluate_stress(pts, nrm, own)
    _, _, info = pr.solve_resistance(V[0], Om[0], tol=1e-13)
    pref, Tref = np.zeros(len(pts)), np.zeros((len(pts), 3))
    for s in range(wl.num_suspensions):
        b = list(pr.suspension_bodies(s))
        sel = np.isin(own, b)
        pref[sel], Tref[sel] = pr.evaluate_stress(b, pr.strengths_dirichlet(b, info[s].x), pts[sel], nrm[sel])
    assert _rel(p.numpy()[0], pref) < tol and _rel(T.numpy()[0], Tref) < tol
    # after a mobility solve: pressure only
    ctx.solve_mobility(wl.F[:1], wl.T[:1])
    p, T = ctx.evaluate_stress(pts, owner=own, traction=False)
    assert T is None
    _, _, info = pr.solve_mobility(wl.F[0], wl.T[0], tol=1e-13)
    for s in range(wl.num_suspensions):
        b = list(pr.suspension_bodies(s))
        sel = np.isin(own, b)
        pref[sel], _ = pr.evaluate_stress(b, pr.total_strengths_mobility(b, info[s].x, wl.F[0], wl.T[0]),
                                         pts[sel], nrm[sel])
    assert _rel(p.numpy()[0], pref) < tol
    ctx.close()
