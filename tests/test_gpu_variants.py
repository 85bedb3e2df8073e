"""Every forward entry of the pair-kernel table, forced through mfs_options.pair_variant, against the
oracle's direct sums (the autotuner may pick any of them on some geometry): ragged bodies of two
shapes, two suspensions, with and without self pairs, relative 2-norm 1e-6 as the matvec for the
FP32 kernels and 2e-8 for the compensated double-FP32 kernels (names "Comp...", precision = 3,
whose pair terms are accurate to about 2^-28)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import Problem  # noqa: E402

from test_gpu_parity import _ctx, _mixed, _oracle_pair, _rel  # noqa: E402


def _opts(name):
    return {"precision": 3} if name.startswith("Comp") else {}


def _tol(name):
    return 2e-8 if name.startswith("Comp") else 1e-6


def _table():
    from paper_2409_04215_gb300.api import pair_variants

    try:
        return [t for t in pair_variants() if not t[4]]
    except RuntimeError:  # library not built here (collection without a GPU)
        return []


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


@pytest.mark.parametrize("include_self", [False, True])
def test_every_variant_matches_oracle(include_self):
    table = _table()
    assert table
    problems = {}
    for kind in ("stokes", "laplace"):
        wl = _mixed(kind, nsusp=2, seed=51)
        problems[kind] = (wl, Problem(wl))
    for idx, name, d, nrhs, _ in table:
        kind = "stokes" if d == 3 else "laplace"
        wl, pr = problems[kind]
        ctx = _ctx(wl, pair_variant=idx, **_opts(name))
        rng = np.random.default_rng(idx)
        s = rng.standard_normal((nrhs, ctx.sum_N, d))
        u = ctx.pair_sum(torch.tensor(s, device="cuda"), include_self=include_self).cpu().numpy()
        assert ctx.pair_variant(nrhs) == name
        for h in range(nrhs):
            ref = _oracle_pair(pr, wl, s[h].reshape(-1), include_self)
            assert _rel(u[h].reshape(-1), ref) < _tol(name), (name, h)
        ctx.close()


def test_every_variant_tiny_bodies():
    """Bodies of 12 collocation and 6 proxy points: every target tile spans the maximum of 32 bodies,
    so the per-tile table of centre offsets (96 entries) is larger than a 64-thread CTA."""
    table = _table()
    assert table
    problems = {}
    for kind in ("stokes", "laplace"):
        wl = _mixed(kind, P=80, m=12, n=6, nsusp=2, seed=52)
        problems[kind] = (wl, Problem(wl))
    for idx, name, d, nrhs, _ in table:
        kind = "stokes" if d == 3 else "laplace"
        wl, pr = problems[kind]
        ctx = _ctx(wl, pair_variant=idx, **_opts(name))
        s = np.random.default_rng(idx + 100).standard_normal((nrhs, ctx.sum_N, d))
        u = ctx.pair_sum(torch.tensor(s, device="cuda"), include_self=False).cpu().numpy()
        for h in range(nrhs):
            ref = _oracle_pair(pr, wl, s[h].reshape(-1), False)
            assert _rel(u[h].reshape(-1), ref) < _tol(name), (name, h)
        ctx.close()
