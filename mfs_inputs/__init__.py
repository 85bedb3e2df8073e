"""Seeded synthetic inputs for the MFS elastance and mobility solvers.

This package only *generates* inputs: body-frame point sets, body centres,
orientations (unit quaternions), shape ids and right-hand sides (charges,
forces, torques).  It holds none of the method's arithmetic (no kernels,
no projectors, no pseudo-inverses) and is shared by the FP64 oracle, the
tests and the benchmark so that both sides see bit-identical inputs.
"""

from .geometry import (
    fibonacci_sphere,
    spheroid_lattice,
    spheroid_proxy,
    random_quaternions,
    rsa_in_cube,
    grow_cluster,
)
from .workloads import Workload, make_workload, WORKLOADS

__all__ = [
    "fibonacci_sphere",
    "spheroid_lattice",
    "spheroid_proxy",
    "random_quaternions",
    "rsa_in_cube",
    "grow_cluster",
    "Workload",
    "make_workload",
    "WORKLOADS",
]
