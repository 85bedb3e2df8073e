"""mfs_matvec_transposed (y = A^T w, the adjoint's operator) against the oracle's transposed matvec,
and the GPU's A and A^T against each other through <A x, y> = <x, A^T y>.  Both one-body applies
(tcgen05 pieces, CUDA-core split-K); rotated mixed shapes, two suspensions, 1 or 2 rhs.  Bar: the
forward matvec's 1e-6 (relative 2-norm)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import Problem  # noqa: E402

from test_gpu_parity import _ctx, _mixed, _rel, _seg  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


@pytest.mark.parametrize("tensor_cores", [1, 0])
@pytest.mark.parametrize("nrhs", [1, 2])
def test_transposed_matvec_matches_oracle(nrhs, tensor_cores):
    wl = _mixed("stokes", nsusp=2)
    ctx = _ctx(wl, tensor_cores=tensor_cores)
    pr = Problem(wl)
    w = np.random.default_rng(21).standard_normal((nrhs, ctx.sum_M, 3))
    y = ctx.matvec_transposed(torch.tensor(w, device="cuda")).cpu().numpy()
    for h in range(nrhs):
        ref = np.concatenate([pr.matvec_T(list(pr.suspension_bodies(s)),
                                          w[h].reshape(-1)[_seg(pr, list(pr.suspension_bodies(s)), "colloc")])
                              for s in range(wl.num_suspensions)])
        assert _rel(y[h].reshape(-1), ref) < 1e-6
    ctx.close()


def test_adjoint_identity_on_gpu():
    wl = _mixed("stokes", nsusp=2, seed=23)
    ctx = _ctx(wl)
    rng = np.random.default_rng(22)
    x = torch.tensor(rng.standard_normal((1, ctx.sum_M, 3)), device="cuda")
    yv = torch.tensor(rng.standard_normal((1, ctx.sum_M, 3)), device="cuda")
    lhs = float((ctx.matvec(x) * yv).sum())
    rhs = float((x * ctx.matvec_transposed(yv)).sum())
    scale = float(torch.linalg.norm(ctx.matvec(x)) * torch.linalg.norm(yv))
    assert abs(lhs - rhs) <= 1e-6 * scale
    ctx.close()


def test_transposed_matvec_rejects_laplace():
    from paper_2409_04215_gb300 import MFSError

    wl = _mixed("laplace")
    ctx = _ctx(wl)
    with pytest.raises(MFSError):
        ctx.matvec_transposed(np.zeros((1, ctx.sum_M, 1)))
    ctx.close()


def test_transposed_matvec_fp64_path():
    """precision = 1: the transposed pair sums in plain FP64 loops and the FP64 transposed one-body
    apply hold A^T w to the oracle's FP64 transposed matvec at the FP64 path's matvec bar (1e-11)."""
    wl = _mixed("stokes", nsusp=2)
    ctx = _ctx(wl, precision=1, autotune=0)
    pr = Problem(wl)
    w = np.random.default_rng(24).standard_normal((2, ctx.sum_M, 3))
    y = ctx.matvec_transposed(torch.tensor(w, device="cuda")).cpu().numpy()
    for h in range(2):
        ref = np.concatenate([pr.matvec_T(list(pr.suspension_bodies(s)),
                                          w[h].reshape(-1)[_seg(pr, list(pr.suspension_bodies(s)), "colloc")])
                              for s in range(wl.num_suspensions)])
        assert _rel(y[h].reshape(-1), ref) < 1e-11
    ctx.close()
