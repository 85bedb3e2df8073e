"""FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see mfs_oracle.py)."""
from .mfs_oracle import *  # noqa: F401,F403
from .mfs_oracle import Problem, gmres, shape_factors, split_workload, direct_sum  # noqa: F401
