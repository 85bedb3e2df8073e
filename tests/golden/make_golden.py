"""Write the stored FP64 oracle results used by the GPU tests and the benchmark.

Calls only the oracle (oracle/) on the seeded inputs (mfs_inputs/):

    python tests/golden/make_golden.py sphere100_mobility

sphere100_mobility_oracle.json: U and Omega [100][3] of the 100-sphere mobility problem
(M = 1200, N = 600, R_p = 0.7, forces and torques N(0,1), seed 2), oracle GMRES tolerance 1e-12.

sphere100_resistance_oracle.json: forces and torques [100][3] of the resistance problem (Sec. 2.2) on
the same geometry for rigid motions U, Omega ~ N(0,1) drawn with numpy default_rng(14) (U first,
each of shape (1, 100, 3)), oracle GMRES tolerance 1e-12.

batched256_mobility_oracle.json: U and Omega [4][P_s][3] of 16 of the 256 suspensions (the largest,
the two with the most spheroids, then sizes spread over the rest; batched256_sample_suspensions), each
solved on its own with all 4 right-hand sides, GMRES tolerance 1e-12.

spheroid1000_sub100_mobility_oracle.json: U and Omega [100][3] of the first 100 bodies of the
1000-spheroid cluster (Sec. 4.2's cluster construction with true surface gaps U[0.05,0.5]; M = 2000,
N = 1000, Delta_sep = 0.25), gravity-like forces (0,0,-1) and zero torques, GMRES tolerance 1e-12.
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


def spheroid1000_sub100_mobility():
    """The first 100 bodies of the 1000-spheroid cluster (semi-axes (1,1,2), true surface gaps
    U[0.05,0.5], M = 2000, N = 1000, Delta_sep = 0.25, F = (0,0,-1), T = 0), oracle GMRES at 1e-12."""
    wl = make_workload("spheroid1000_mobility").first_bodies(100)
    t0 = time.time()
    pr = Problem(wl)
    t_setup = time.time() - t0
    U, W, info = pr.solve_mobility(wl.F[0], wl.T[0], tol=1e-12)
    out = {
        "workload": "spheroid1000_mobility, first 100 bodies",
        "description": wl.description,
        "oracle_gmres_tol": 1e-12,
        "oracle_iters": info[0].iters,
        "oracle_residual": info[0].residual_estimate,
        "sigma_ratio": float(pr.factors[0].sigma[-1] / pr.factors[0].sigma[0]),
        "setup_seconds": t_setup,
        "seconds": time.time() - t0,
        "U": U.tolist(),
        "Omega": W.tolist(),
    }
    with open(os.path.join(HERE, "spheroid1000_sub100_mobility_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(f"iters {info[0].iters}, {out['seconds']:.0f} s")


def batched256_sample_suspensions(wl, count: int = 16):
    """The suspensions of the 256-suspension workload held to oracle solves: the largest, the two with
    the most spheroids (by count), then the sizes nearest to evenly spaced quantiles of the rest."""
    import numpy as np

    sizes = np.diff(wl.body_offsets)
    spheroids = np.array([int(wl.shape_id[wl.body_offsets[s]:wl.body_offsets[s + 1]].sum())
                          for s in range(wl.num_suspensions)])
    chosen = [int(np.argmax(sizes))]
    for s in np.argsort(-spheroids, kind="stable"):
        if int(s) not in chosen:
            chosen.append(int(s))
        if len(chosen) == 3:
            break
    order = [int(s) for s in np.argsort(sizes, kind="stable") if int(s) not in chosen]
    for q in np.linspace(0, len(order) - 1, count - len(chosen)):
        s = order[int(round(q))]
        if s not in chosen:
            chosen.append(s)
    return sorted(chosen)


def batched256_mobility():
    """Oracle solves of 16 of the 256 suspensions, all 4 right-hand sides, GMRES at 1e-12."""
    from oracle.mfs_oracle import split_workload

    wl = make_workload("batched256_mobility")
    chosen = batched256_sample_suspensions(wl)
    t0 = time.time()
    out = {"workload": "batched256_mobility", "description": wl.description, "oracle_gmres_tol": 1e-12,
           "suspensions": {}}
    for s in chosen:
        sub = split_workload(wl, s)
        pr = Problem(sub)
        U, W, iters = [], [], []
        for h in range(wl.nrhs):
            Uh, Wh, info = pr.solve_mobility(sub.F[h], sub.T[h], tol=1e-12)
            U.append(Uh.tolist())
            W.append(Wh.tolist())
            iters.append(info[0].iters)
        out["suspensions"][str(s)] = {"bodies": int(sub.num_bodies), "spheroids": int(sub.shape_id.sum()),
                                      "iters": iters, "U": U, "Omega": W}
        print(f"suspension {s}: {sub.num_bodies} bodies, iters {iters}, {time.time() - t0:.0f} s", flush=True)
    out["seconds"] = time.time() - t0
    with open(os.path.join(HERE, "batched256_mobility_oracle.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    for name in sys.argv[1:] or ["sphere100_mobility"]:
        globals()[name]()
