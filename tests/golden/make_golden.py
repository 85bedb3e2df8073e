"""Write the stored FP64 oracle results used by the GPU tests and the benchmark.

Calls only the oracle (oracle/) on the seeded inputs (mfs_inputs/):

    python tests/golden/make_golden.py sphere100_mobility

sphere100_mobility_oracle.json: U and Omega [100][3] of the 100-sphere mobility problem
(M = 1200, N = 600, R_p = 0.7, forces and torques N(0,1), seed 2), oracle GMRES tolerance 1e-12.

sphere100_resistance_oracle.json: forces and torques [100][3] of the resistance problem (Sec. 2.2) on
the same geometry for rigid motions U, Omega ~ N(0,1) drawn with numpy default_rng(14) (U first,
each of shape (1, 100, 3)), oracle GMRES tolerance 1e-12.
"""

from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from mfs_inputs import make_workload  # noqa: E402
from oracle import Problem  # noqa: E402


def sphere100_mobility():
    wl = make_workload("sphere100_mobility")
    t0 = time.time()
    pr = Problem(wl)
    U, W, info = pr.solve_mobility(wl.F[0], wl.T[0], tol=1e-12)
    out = {
        "workload": "sphere100_mobility",
        "description": wl.description,
        "oracle_gmres_tol": 1e-12,
        "oracle_iters": info[0].iters,
        "oracle_residual": info[0].residual_estimate,
        "sigma_ratio": float(pr.factors[0].sigma[-1] / pr.factors[0].sigma[0]),
        "seconds": time.time() - t0,
        "U": U.tolist(),
        "Omega": W.tolist(),
    }
    with open(os.path.join(HERE, "sphere100_mobility_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(f"iters {info[0].iters}, {out['seconds']:.0f} s")


def sphere100_resistance():
    import numpy as np

    wl = make_workload("sphere100_mobility")
    rng = np.random.default_rng(14)
    U_ref, W_ref = rng.standard_normal((1, 100, 3)), rng.standard_normal((1, 100, 3))
    t0 = time.time()
    pr = Problem(wl)
    F, T, info = pr.solve_resistance(U_ref[0], W_ref[0], tol=1e-12, max_iter=300)
    out = {
        "workload": "sphere100_mobility geometry, resistance problem",
        "description": wl.description,
        "inputs": "U, Omega = numpy.random.default_rng(14).standard_normal((1, 100, 3)) twice",
        "oracle_gmres_tol": 1e-12,
        "oracle_iters": info[0].iters,
        "oracle_residual": info[0].residual_estimate,
        "seconds": time.time() - t0,
        "F": F.tolist(),
        "T": T.tolist(),
    }
    with open(os.path.join(HERE, "sphere100_resistance_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(f"iters {info[0].iters}, {out['seconds']:.0f} s")


if __name__ == "__main__":
    for name in sys.argv[1:] or ["sphere100_mobility"]:
        globals()[name]()
