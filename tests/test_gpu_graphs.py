"""The CUDA-graph GMRES loop (mfs_options.graphs = 1, the default without profiling) runs the same
kernels as the host loop on the same data: every solve kind gives bit-identical results and the
same iteration counts either way (the graph adds one copy kernel per iteration)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from mfs_inputs.workloads import make_workload  # noqa: E402

from test_gpu_parity import _ctx, _mixed  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _both(wl, run, **kw):
    out = []
    for graphs in (0, 1):
        ctx = _ctx(wl, graphs=graphs, **kw)
        res = run(ctx)
        out.append(res)
        ctx.close()
    return out


def _same(a, b):
    for x, y in zip(a[:-1], b[:-1]):
        np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())
    ia, ib = a[-1], b[-1]
    assert (ia.iters, ia.matvecs, ia.pair_launches) == (ib.iters, ib.matvecs, ib.pair_launches)
    # the graph iterations (all but the first) add one kernel each: v_j copied to the matvec input
    assert ib.launches == ia.launches + (ib.matvecs - 1)
    assert ia.converged and ib.converged and ia.iters > 2


@pytest.mark.parametrize("precision", [0, 1])
def test_mobility_and_vjp(precision):
    wl = _mixed("stokes", nsusp=2)
    F, T = torch.tensor(wl.F[:2], device="cuda"), torch.tensor(wl.T[:2], device="cuda")

    def run(ctx):
        U, W, info = ctx.solve_mobility(F, T)
        dc, _, _ = ctx.mobility_vjp(U, W)  # the transposed solve runs as a graph too
        return U, W, dc, info

    _same(*_both(wl, run, precision=precision))


def test_elastance_resistance_capacitance():
    wl = _mixed("laplace")
    _same(*_both(wl, lambda c: c.solve_elastance(torch.tensor(wl.Q[None], device="cuda"))))
    _same(*_both(wl, lambda c: c.solve_capacitance(torch.tensor(wl.Q[None], device="cuda"))))
    ws = _mixed("stokes")
    V = torch.tensor(np.random.default_rng(3).standard_normal((2, 1, ws.num_bodies, 3)), device="cuda")
    _same(*_both(ws, lambda c: c.solve_resistance(V[0], V[1])))


def test_batched_lanes():
    wl = make_workload("batched256_mobility", num_suspensions=9, p_lo=1, p_hi=8, m=120, n=60, seed=4)
    F, T = torch.tensor(wl.F, device="cuda"), torch.tensor(wl.T, device="cuda")
    _same(*_both(wl, lambda c: c.solve_mobility(F, T)))


def test_repeated_solves_reuse_the_graph():
    wl = _mixed("stokes")
    ctx = _ctx(wl)
    F, T = torch.tensor(wl.F[:1], device="cuda"), torch.tensor(wl.T[:1], device="cuda")
    U1, W1, i1 = ctx.solve_mobility(F, T)
    U2, W2, i2 = ctx.solve_mobility(2.0 * F, 2.0 * T)  # linear: twice the velocities
    np.testing.assert_allclose(U2.cpu().numpy(), 2.0 * U1.cpu().numpy(), rtol=0, atol=1e-12 * np.abs(U1.cpu().numpy()).max())
    ctx.close()
