"""Full-size solves against stored FP64 oracle results (tests/golden, written by make_golden.py).

The 100-sphere mobility problem (M = 1200, N = 600, the benchmark geometry): solved velocities
and angular velocities within 1e-5 (relative 2-norm) of the oracle's GMRES solution at 1e-12,
with the default GPU tolerance 1e-7, for the tensor-core (default) and the CUDA-core one-body
apply; the mixed path (FP64 apply) agrees to 1e-6.
"""

import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sphere100_mobility_oracle.json")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from mfs_inputs import make_workload

    g = json.load(open(GOLDEN))
    ref = np.concatenate([np.array(g["U"]), np.array(g["Omega"])], axis=1)
    return make_workload("sphere100_mobility"), ref


@pytest.mark.parametrize("precision,tensor_cores,tol", [(0, 1, 1e-5), (0, 0, 1e-5), (2, 0, 1e-6)])
def test_sphere100_mobility_matches_oracle(setup, precision, tensor_cores, tol):
    from paper_2409_04215_gb300 import MFS

    wl, ref = setup
    ctx = MFS.from_workload(wl, precision=precision, tensor_cores=tensor_cores)
    U, W, info = ctx.solve_mobility(torch.tensor(wl.F, device="cuda"), torch.tensor(wl.T, device="cuda"))
    got = np.concatenate([U.cpu().numpy()[0], W.cpu().numpy()[0]], axis=1)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert info.converged
    assert err < tol, f"relative error {err:.3e}"
    ctx.close()
