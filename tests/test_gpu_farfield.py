"""The far-field accelerator of the pair sums (mfs_options.farfield = 1): an equivalent-source treecode,
the GPU counterpart of the FMM the paper uses for its large runs (Sec. 4).

Its sums are an approximation of the direct sums, so the oracle here is the direct sum itself: the
treecode's matvec of Eq. 2esysprec and its all-pairs right-hand side (Eq. stou0) are held to the
oracle's FP64 direct sums (relative 2-norm 1e-6, the matvec bar) on a 400-body cluster of Type T
ellipsoids, on sampled targets of the 10 000-body cluster of Sec. 4.2, against the GPU's own direct
sums on several suspensions and on the Laplace kernel, and its mobility solve to the stored 100-sphere
oracle solution (1e-5).
"""

import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from mfs_inputs import make_workload  # noqa: E402
from oracle import Problem  # noqa: E402

from test_gpu_parity import _ctx, _rel  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _rigid_field(pr, wl, seed):
    """A rigid motion of every body at its collocation points, v + omega x (x - c) (Eq. Kdef)."""
    V = np.random.default_rng(seed).standard_normal((pr.P, 6))
    return np.concatenate([(V[k, :3] + np.cross(V[k, 3:], pr.X[k] - wl.centres[k])).reshape(-1)
                           for k in range(pr.P)])


def test_farfield_matvec_and_rhs_type_t_cluster():
    wl = make_workload("ellipsoidT5000_mobility", count=400, n_v=16)
    pr = Problem(wl)
    ctx = _ctx(wl, farfield=1)
    bodies = list(range(pr.P))
    gam = _rigid_field(pr, wl, 1)
    y = ctx.matvec(torch.tensor(gam.reshape(1, -1, 3), device="cuda")).cpu().numpy().reshape(-1)
    assert _rel(y, pr.matvec(bodies, gam)) < 1e-6
    s = np.random.default_rng(2).standard_normal((1, ctx.sum_N, 3))
    u = ctx.pair_sum(torch.tensor(s, device="cuda"), include_self=True).cpu().numpy().reshape(-1)
    ref = np.concatenate(pr.pair_sum(bodies, pr.split(bodies, s.reshape(-1), on="proxy"), include_self=True))
    assert _rel(u, ref) < 1e-6
    ctx.close()


def test_farfield_matches_direct_on_suspensions_and_rhs():
    """Several suspensions (one of a single body: an empty interaction list), 4 right-hand sides:
    treecode against the direct GPU sums, white-noise strengths."""
    wl = make_workload("batched256_mobility", num_suspensions=6, p_lo=1, p_hi=40, m=120, n=60, seed=9)
    direct, tree = _ctx(wl), _ctx(wl, farfield=1)
    s = torch.tensor(np.random.default_rng(3).standard_normal((4, direct.sum_N, 3)), device="cuda")
    for include_self in (False, True):
        a = direct.pair_sum(s, include_self=include_self).cpu().numpy()
        b = tree.pair_sum(s, include_self=include_self).cpu().numpy()
        for h in range(4):
            assert _rel(b[h].reshape(-1), a[h].reshape(-1)) < 1e-6, (include_self, h)
    direct.close()
    tree.close()


def test_farfield_laplace_elastance():
    wl = make_workload("sphere100_elastance", m=300, n=150)
    direct, tree = _ctx(wl), _ctx(wl, farfield=1)
    s = torch.tensor(np.random.default_rng(4).standard_normal((1, direct.sum_N, 1)), device="cuda")
    a = direct.pair_sum(s, include_self=True).cpu().numpy().reshape(-1)
    b = tree.pair_sum(s, include_self=True).cpu().numpy().reshape(-1)
    assert _rel(b, a) < 1e-6
    Q = torch.tensor(wl.Q[None], device="cuda")
    Va, _ = direct.solve_elastance(Q)
    Vb, info = tree.solve_elastance(Q)
    assert info.converged and _rel(Vb.cpu().numpy(), Va.cpu().numpy()) < 1e-5
    direct.close()
    tree.close()


def test_farfield_sphere100_solve_against_golden():
    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                    "sphere100_mobility_oracle.json")))
    wl = make_workload("sphere100_mobility")
    ctx = _ctx(wl, farfield=1)
    U, W, info = ctx.solve_mobility(torch.tensor(wl.F, device="cuda"), torch.tensor(wl.T, device="cuda"))
    assert info.converged
    got = np.concatenate([U.cpu().numpy()[0], W.cpu().numpy()[0]], 1)
    assert _rel(got, np.concatenate([np.array(g["U"]), np.array(g["Omega"])], 1)) < 1e-5
    assert info.pairs_evaluated < info.pairs  # the treecode evaluated fewer pairs than the direct sums hold
    ctx.close()


def test_farfield_type_t_10000_sampled():
    """Sec. 4.2's 10 000-ellipsoid cluster at its full discretisation (N_v = 34): the treecode matvec on
    three sampled target bodies against the oracle's sums over all 9 999 other bodies, at the default
    separation (3 equivalent radii) and at the smallest allowed (2.5, the check sphere); the direct
    GPU sum on the same targets shows what FP32 alone contributes."""
    wl = make_workload("ellipsoidT10000_mobility")
    pr = Problem(wl)
    bodies = list(range(pr.P))
    gam = _rigid_field(pr, wl, 5)
    g = pr.split(bodies, gam)
    sample = [0, 4321, 9999]
    lam_hat = [pr.pinv_apply(k, g[k], project=True) for k in bodies]
    ref = pr.pair_sum(bodies, lam_hat, include_self=False, target_bodies=sample)

    def err(ctx):
        y = ctx.matvec(torch.tensor(gam.reshape(1, -1, 3), device="cuda")).cpu().numpy().reshape(-1)
        got = pr.split(bodies, y)
        num = sum(np.sum((got[k] - g[k] - r) ** 2) for k, r in zip(sample, ref))
        den = sum(np.sum((g[k] + r) ** 2) for k, r in zip(sample, ref))
        ctx.close()
        return float(np.sqrt(num / den))

    e3 = err(_ctx(wl, farfield=1, max_iter=60, restart=60))
    e25 = err(_ctx(wl, farfield=1, farfield_separation=2.5, max_iter=60, restart=60))
    ed = err(_ctx(wl, max_iter=60, restart=60))
    print(f"10 000 ellipsoids, sampled matvec error: separation 3: {e3:.2e}, 2.5: {e25:.2e}, direct: {ed:.2e}")
    assert e3 < 1e-6 and e25 < 1e-6 and ed < 1e-6


def test_farfield_follows_moved_bodies():
    """mfs_update_centers with the treecode: the tree, node geometry and interaction lists are rebuilt,
    so the matvec at the new positions matches a direct context moved the same way (and one set up
    there), twice in a row, and a solve after the move matches the oracle's."""
    wl = make_workload("sphere100_mobility", count=40, m=300, n=150, seed=21)
    tree, direct = _ctx(wl, farfield=1), _ctx(wl)
    s = torch.tensor(np.random.default_rng(22).standard_normal((1, tree.sum_N, 3)), device="cuda")
    rng = np.random.default_rng(23)
    centres = wl.centres.copy()
    for step in range(2):
        # a rigid shift of the whole cluster plus a shuffle of which body sits where (a new tree)
        centres = centres[rng.permutation(len(centres))] + rng.standard_normal(3)
        tree.update_centers(centres)
        direct.update_centers(centres)
        moved = make_workload("sphere100_mobility", count=40, m=300, n=150, seed=21)
        moved.centres = centres
        pr = Problem(moved)
        # pair sums of white-noise strengths, and the matvec of a rigid motion (smooth: no amplification
        # of FP32 rounding through the one-body pseudo-inverse)
        a = direct.pair_sum(s, include_self=False).cpu().numpy().reshape(-1)
        b = tree.pair_sum(s, include_self=False).cpu().numpy().reshape(-1)
        assert _rel(b, a) < 1e-6, step
        gam = torch.tensor(_rigid_field(pr, moved, 30 + step).reshape(1, -1, 3), device="cuda")
        a = direct.matvec(gam).cpu().numpy().reshape(-1)
        b = tree.matvec(gam).cpu().numpy().reshape(-1)
        assert _rel(b, a) < 1e-6, step
    U, W, info = tree.solve_mobility(torch.tensor(wl.F[:1], device="cuda"), torch.tensor(wl.T[:1], device="cuda"))
    Ur, Wr, _ = pr.solve_mobility(wl.F[0], wl.T[0], tol=1e-12)
    assert info.converged
    got = np.concatenate([U.cpu().numpy()[0], W.cpu().numpy()[0]], 1)
    assert _rel(got, np.concatenate([Ur, Wr], 1)) < 1e-5
    tree.close()
    direct.close()


def test_farfield_dirichlet_and_adjoint():
    """The other solves on the treecode's forward sums: resistance (Sec. 2.2) and the mobility adjoint
    (its forward solve and right-hand side use the treecode; the transposed sums stay direct) against
    the same solves with direct sums, and capacitance (Sec. 2.1) on the Laplace kernel."""
    wl = make_workload("sphere100_mobility", count=40, m=300, n=150, seed=24)
    direct, tree = _ctx(wl, gmres_tol=1e-9), _ctx(wl, farfield=1, gmres_tol=1e-9)
    rng = np.random.default_rng(25)
    Uin, Win = rng.standard_normal((1, wl.num_bodies, 3)), rng.standard_normal((1, wl.num_bodies, 3))
    Fa, Ta, ia = direct.solve_resistance(Uin, Win)
    Fb, Tb, ib = tree.solve_resistance(Uin, Win)
    assert ia.converged and ib.converged
    assert _rel(np.concatenate([Fb.numpy(), Tb.numpy()], 2), np.concatenate([Fa.numpy(), Ta.numpy()], 2)) < 1e-5
    for nrhs in (1, 2):  # the centre gradient runs on both trees (target and source sides)
        F, T = torch.tensor(wl.F[:nrhs], device="cuda"), torch.tensor(wl.T[:nrhs], device="cuda")
        grads = []
        for ctx in (direct, tree):
            U, W, _ = ctx.solve_mobility(F, T)
            dc, dF, dT = ctx.mobility_vjp(2.0 * U, 0.6 * W, want_force_grads=True)
            grads.append((dc.cpu().numpy(), np.concatenate([dF.cpu().numpy().reshape(-1),
                                                            dT.cpu().numpy().reshape(-1)])))
        (dca, fa), (dcb, fb) = grads
        assert _rel(dcb, dca) < 1e-4, nrhs
        assert _rel(fb, fa) < 1e-4, nrhs
        assert np.abs(dcb.sum(axis=0)).max() <= 1e-4 * np.abs(dca).max()  # translation invariance
    direct.close()
    tree.close()
    lw = make_workload("sphere100_elastance", count=40, m=300, n=150)
    direct, tree = _ctx(lw, gmres_tol=1e-9), _ctx(lw, farfield=1, gmres_tol=1e-9)
    phi = np.random.default_rng(26).standard_normal((2, lw.num_bodies))
    qa, _ = direct.solve_capacitance(phi)
    qb, info = tree.solve_capacitance(phi)
    assert info.converged and _rel(qb.numpy(), qa.numpy()) < 1e-5
    direct.close()
    tree.close()


def test_farfield_transposed_sums():
    """The adjoint's transposed pair sums through their own treecode (collocation points as sources,
    proxy points as targets), before and after a move.  A^T applies (S_L^+)^T after the pair sum, which
    amplifies FP32-level errors of the sum on this coarse grid (the direct FP32 path lands about 5e-5
    from the FP64 GPU path on a rigid-motion w), so the bar is relative: the treecode's A^T w is held
    to the FP64 GPU path within 1.5x the direct FP32 path's own error (plus 1e-6)."""
    wl = make_workload("sphere100_mobility", count=40, m=300, n=150, seed=27)
    tree, direct = _ctx(wl, farfield=1), _ctx(wl)
    ref = _ctx(wl, precision=1, autotune=0)
    pr = Problem(wl)
    for step in range(2):
        if step:
            centres = wl.centres[np.random.default_rng(28).permutation(wl.num_bodies)] + 0.5
            for ctx in (tree, direct, ref):
                ctx.update_centers(centres)
            moved = make_workload("sphere100_mobility", count=40, m=300, n=150, seed=27)
            moved.centres = centres
            pr = Problem(moved)
            wl = moved
        rigid = _rigid_field(pr, wl, 40 + step)
        noise = np.random.default_rng(50 + step).standard_normal(rigid.size)
        for v in (rigid, noise):
            w = torch.tensor(v.reshape(1, -1, 3), device="cuda")
            r = ref.matvec_transposed(w).cpu().numpy().reshape(-1)
            e_dir = _rel(direct.matvec_transposed(w).cpu().numpy().reshape(-1), r)
            e_tree = _rel(tree.matvec_transposed(w).cpu().numpy().reshape(-1), r)
            assert e_tree <= 1.5 * e_dir + 1e-6, (step, e_tree, e_dir)
    for ctx in (tree, direct, ref):
        ctx.close()


def test_farfield_evaluate_points():
    """mfs_evaluate through the treecode (the points reordered into the tree's body order, one-off
    interaction lists with each owner's farthest point as its radius) against the direct evaluation:
    points near the bodies' surfaces and points between them, owners given or found, mobility with two
    right-hand sides and elastance."""
    rng = np.random.default_rng(32)
    for name in ("sphere100_mobility", "sphere100_elastance"):
        wl = make_workload(name, count=40, m=300, n=150, seed=31) if name.endswith("mobility") else \
            make_workload(name, count=40, m=300, n=150)
        tree, direct = _ctx(wl, farfield=1), _ctx(wl)
        nrhs = 2 if name.endswith("mobility") else 1
        FT = rng.standard_normal((2, nrhs, wl.num_bodies, 3))
        for ctx in (tree, direct):
            if name.endswith("mobility"):
                ctx.solve_mobility(torch.tensor(FT[0], device="cuda"), torch.tensor(FT[1], device="cuda"))
            else:
                ctx.solve_elastance(torch.tensor(wl.Q[None], device="cuda"))
        k = rng.integers(0, wl.num_bodies, 3000)
        d = rng.standard_normal((3000, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        near = wl.centres[k] + rng.uniform(1.02, 1.5, 3000)[:, None] * d
        box = rng.uniform(wl.centres.min(0), wl.centres.max(0), (4000, 3))
        dist = np.linalg.norm(box[:, None, :] - wl.centres[None], axis=2)
        box = box[dist.min(1) > 1.05][:800]
        pts = np.concatenate([near, box])
        owner = np.linalg.norm(pts[:, None, :] - wl.centres[None], axis=2).argmin(1).astype(np.int32)
        for own in (owner, None):
            a = direct.evaluate(pts, owner=own, nrhs=nrhs).numpy()
            b = tree.evaluate(pts, owner=own, nrhs=nrhs).numpy()
            assert _rel(b, a) < 1e-6, (name, own is None)
        tree.close()
        direct.close()


def test_farfield_pressure_and_traction():
    """mfs_evaluate_stress through the treecode (per-owner interaction lists of bodies and tree nodes,
    the pressure and traction of the equivalent Stokeslets in the far field) against the direct sums,
    after a mobility solve with two right-hand sides and after a resistance solve."""
    rng = np.random.default_rng(33)
    wl = make_workload("sphere100_mobility", count=40, m=300, n=150, seed=34)
    tree, direct = _ctx(wl, farfield=1), _ctx(wl)
    k = rng.integers(0, wl.num_bodies, 3000)
    d = rng.standard_normal((3000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts = wl.centres[k] + rng.uniform(1.0, 1.4, 3000)[:, None] * d
    nrm = rng.standard_normal((3000, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    for solve in ("mobility", "resistance"):
        FT = rng.standard_normal((2, 2, wl.num_bodies, 3))
        for ctx in (tree, direct):
            if solve == "mobility":
                ctx.solve_mobility(torch.tensor(FT[0], device="cuda"), torch.tensor(FT[1], device="cuda"))
            else:
                ctx.solve_resistance(FT[0], FT[1])
        for own in (k.astype(np.int32), None):
            pa, ta = direct.evaluate_stress(pts, normals=nrm, owner=own, nrhs=2)
            pb, tb = tree.evaluate_stress(pts, normals=nrm, owner=own, nrhs=2)
            assert _rel(pb.numpy(), pa.numpy()) < 1e-6, (solve, "pressure")
            assert _rel(tb.numpy(), ta.numpy()) < 1e-6, (solve, "traction")
    tree.close()
    direct.close()


@pytest.mark.parametrize("kind", ["stokes", "laplace"])
def test_farfield_small_and_many_rhs(kind):
    """Degenerate trees and every right-hand-side count: one body (no pairs at all off the body), two
    bodies, and several suspensions of uneven size, 1-4 right-hand sides, both kernels, against the
    direct GPU sums."""
    name = "batched256_mobility"
    for count, kw in ((1, dict(num_suspensions=1, p_lo=1, p_hi=1)), (2, dict(num_suspensions=1, p_lo=2, p_hi=2)),
                      (None, dict(num_suspensions=5, p_lo=1, p_hi=30))):
        wl = make_workload(name, m=120, n=60, seed=41, **kw)
        if kind == "laplace":
            wl.kind = "laplace"
        direct, tree = _ctx(wl), _ctx(wl, farfield=1)
        d = 3 if kind == "stokes" else 1
        for nrhs in (1, 2, 3, 4):
            s = torch.tensor(np.random.default_rng(nrhs).standard_normal((nrhs, direct.sum_N, d)), device="cuda")
            for include_self in (False, True):
                a = direct.pair_sum(s, include_self=include_self).cpu().numpy()
                b = tree.pair_sum(s, include_self=include_self).cpu().numpy()
                if not np.any(a):  # one body, self pairs left out: nothing to sum
                    assert not np.any(b)
                    continue
                assert _rel(b.reshape(-1), a.reshape(-1)) < 1e-6, (count, nrhs, include_self)
        direct.close()
        tree.close()
