"""The allocation-free Stokeslet sum, for callers that cannot allocate device memory.

Code that runs inside another framework's memory pool, a plug-in host, or a fixed memory budget
may not call cudaMalloc; mfs_stokeslet_sum_noalloc serves it from a fixed scratch array inside
the library.  These tests call it through the C ABI on several calls in a row and check each result
against the oracle's FP64 direct Stokeslet sum over the same points (all pairs, self included) and,
on the first call, against the context-based entry point mfs_pair_sum, within the pair-sum tolerance
of the other tests (relative 2-norm 1e-6).  Later calls are smaller than earlier ones, have source
counts that are not a multiple of 4, sit far from the origin, and reach an odd source count next to
the 65 536 limit, so stale scratch from a larger earlier call would show.  Sizes beyond the stated
maximum must be refused before any work.  The file is named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2409_04215_gb300.api import load_library

    lib = load_library()
    vp = ctypes.c_void_p
    lib.mfs_stokeslet_sum_noalloc.argtypes = [vp, ctypes.c_int32, vp, vp, ctypes.c_int32, ctypes.c_double, vp, vp]
    lib.mfs_stokeslet_sum_noalloc.restype = ctypes.c_int
    return lib


def _oracle_sum(targets, sources, lam, mu):
    from oracle.mfs_oracle import direct_sum

    nt, ns = len(targets), len(sources)
    zero_t, zero_s = np.zeros(nt, np.int32), np.zeros(ns, np.int32)
    # one group, targets and sources of different "bodies": every pair counts
    return direct_sum("stokes", targets, zero_t, zero_t, sources, zero_s, zero_s + 1, lam, True, mu)


def _call(lib, targets, sources, lam, mu):
    tgt = torch.tensor(targets, device="cuda")
    src = torch.tensor(sources, device="cuda")
    lm = torch.tensor(lam, device="cuda")
    out = torch.full((len(targets), 3), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.mfs_stokeslet_sum_noalloc(tgt.data_ptr(), len(targets), src.data_ptr(), lm.data_ptr(), len(sources),
                                       mu, out.data_ptr(), stream)
    torch.cuda.synchronize()
    return rc, out.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_oracle_on_calls_in_a_row():
    from mfs_inputs import make_workload
    from paper_2409_04215_gb300 import MFS

    lib = _lib()
    rng = np.random.default_rng(11)
    wl = make_workload("sphere100_mobility", count=9, m=300, n=150, seed=4)  # identity orientations
    shape = wl.shapes[0]
    targets = np.concatenate([c + shape.colloc for c in wl.centres])
    sources = np.concatenate([c + shape.proxy for c in wl.centres])

    # call 1: all 2700 targets and 1350 sources; also against the context-based pair sum
    lam = rng.standard_normal((len(sources), 3))
    rc, got = _call(lib, targets, sources, lam, 1.0)
    assert rc == 0, f"call 1: status {rc}"
    assert _rel(got, _oracle_sum(targets, sources, lam, 1.0)) < 1e-6
    ctx = MFS.from_workload(wl)
    ref_ctx = ctx.pair_sum(torch.tensor(lam[None], device="cuda"), include_self=True)[0].cpu().numpy()
    assert _rel(got, ref_ctx) < 1e-6
    ctx.close()

    # call 2: fewer targets, a source count that is not a multiple of 4, the whole set moved far
    # from the origin, another viscosity
    shift = np.array([1000.0, -500.0, 250.0])
    t2, s2 = targets[:1001] + shift, sources[:1349] + shift
    lam2 = rng.standard_normal((len(s2), 3))
    rc, got2 = _call(lib, t2, s2, lam2, 2.5)
    assert rc == 0, f"call 2: status {rc}"
    assert _rel(got2, _oracle_sum(t2, s2, lam2, 2.5)) < 1e-6

    # call 3: smaller again (one tile, 7 sources)
    t3, s3 = targets[:37], sources[-7:]
    lam3 = rng.standard_normal((7, 3))
    rc, got3 = _call(lib, t3, s3, lam3, 1.0)
    assert rc == 0, f"call 3: status {rc}"
    assert _rel(got3, _oracle_sum(t3, s3, lam3, 1.0)) < 1e-6


def test_noalloc_near_the_source_limit():
    """65 509 sources (odd, below the 65 536 limit) on 109 spheres, then a small call after it."""
    from mfs_inputs import make_workload

    lib = _lib()
    wl = make_workload("sphere100_mobility", count=109, m=400, n=601, seed=4)
    shape = wl.shapes[0]
    sources = np.concatenate([c + shape.proxy for c in wl.centres])
    targets = np.concatenate([c + shape.colloc for c in wl.centres[:5]])
    assert len(sources) == 65509 and len(sources) % 2 == 1
    lam = np.random.default_rng(12).standard_normal((len(sources), 3))
    rc, got = _call(lib, targets, sources, lam, 1.0)
    assert rc == 0, f"status {rc}"
    assert _rel(got, _oracle_sum(targets, sources, lam, 1.0)) < 1e-6
    t2, s2, lam2 = targets[:500], sources[:999], lam[:999]
    rc, got2 = _call(lib, t2, s2, lam2, 1.0)
    assert rc == 0, f"status {rc}"
    assert _rel(got2, _oracle_sum(t2, s2, lam2, 1.0)) < 1e-6


def test_noalloc_refuses_oversize():
    lib = _lib()
    dummy = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.mfs_stokeslet_sum_noalloc(p, 65537, p, p, 4, 1.0, p, stream) == 1
    assert lib.mfs_stokeslet_sum_noalloc(p, 4, p, p, 65537, 1.0, p, stream) == 1
    assert lib.mfs_stokeslet_sum_noalloc(p, 4, p, p, 4, 0.0, p, stream) == 1
