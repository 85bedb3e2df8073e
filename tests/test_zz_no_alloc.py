"""The allocation-free Stokeslet sum, for callers that cannot allocate device memory.

Code that runs inside another framework's memory pool, a plug-in host, or a fixed memory budget
may not call cudaMalloc; mfs_stokeslet_sum_noalloc serves it from a fixed scratch array inside
the library.  This test calls it through the C ABI on two calls in a row and checks each result
against the context-based entry point mfs_pair_sum over the same points (all pairs, self
included), within the pair-sum tolerance of the other tests (relative 2-norm 1e-6).  It also
checks that sizes beyond the stated maximum are refused before any work.  The file is named so
that pytest collects it last.
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


def test_noalloc_matches_pair_sum_twice():
    from mfs_inputs import make_workload
    from paper_2409_04215_gb300 import MFS

    lib = _lib()
    wl = make_workload("sphere100_mobility", count=9, m=300, n=150, seed=4)  # identity orientations
    ctx = MFS.from_workload(wl)
    shape = wl.shapes[0]
    targets = np.concatenate([c + shape.colloc for c in wl.centres])
    sources = np.concatenate([c + shape.proxy for c in wl.centres])
    tgt = torch.tensor(targets, device="cuda")
    src = torch.tensor(sources, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(11)
    for call in range(2):
        lam = torch.tensor(rng.standard_normal((len(sources), 3)), device="cuda")
        ref = ctx.pair_sum(lam[None], include_self=True)[0].cpu().numpy()
        out = torch.full((len(targets), 3), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.mfs_stokeslet_sum_noalloc(tgt.data_ptr(), len(targets), src.data_ptr(), lam.data_ptr(),
                                           len(sources), 1.0, out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert rc == 0, f"call {call}: status {rc}"
        got = out.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 1e-6, f"call {call}: relative error {err:.3e}"
    ctx.close()


def test_noalloc_refuses_oversize():
    lib = _lib()
    dummy = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.mfs_stokeslet_sum_noalloc(p, 65537, p, p, 4, 1.0, p, stream) == 1
    assert lib.mfs_stokeslet_sum_noalloc(p, 4, p, p, 65537, 1.0, p, stream) == 1
    assert lib.mfs_stokeslet_sum_noalloc(p, 4, p, p, 4, 0.0, p, stream) == 1
