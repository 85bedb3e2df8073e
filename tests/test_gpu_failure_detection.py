"""Failure detection without a GPU fault: the kernels' bounded device waits give up, flag the error and
return, and the host reports MFS_ERR_DEVICE_TIMEOUT with the CUDA context intact (a lost bulk copy or a
tensor-core stage that never lands takes the same path).  The wait that runs out is an mbarrier phase
that nothing completes, bounded to a thousand polls."""

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


def test_bounded_wait_reports_timeout_and_context_survives():
    from paper_2409_04215_gb300.api import selftest_bounded_wait

    assert selftest_bounded_wait(True) == 0  # the phase is completed: the wait succeeds
    assert selftest_bounded_wait(False) == 7  # nothing completes it: MFS_ERR_DEVICE_TIMEOUT
    assert selftest_bounded_wait(False, limit=10) == 7
    torch.cuda.synchronize()
    # the context is intact: a matvec right after still matches the oracle
    wl = _mixed("stokes", nsusp=2)
    ctx = _ctx(wl)
    pr = Problem(wl)
    gam = np.random.default_rng(5).standard_normal((1, ctx.sum_M, 3))
    y = ctx.matvec(torch.tensor(gam, device="cuda")).cpu().numpy()
    ref = np.concatenate([pr.matvec(list(pr.suspension_bodies(s)),
                                    gam[0].reshape(-1)[_seg(pr, list(pr.suspension_bodies(s)), "colloc")])
                          for s in range(wl.num_suspensions)])
    assert _rel(y[0].reshape(-1), ref) < 1e-6
    ctx.close()
