"""Named, seeded workloads with the shapes of the paper's experiments.

Every array is FP64 (positions, right-hand sides) or int32 (ids, offsets).
Body-frame point sets are centred on the body centre; a body's global points
are c_k + R(q_k) X0 with R(q) the rotation of the unit quaternion q = (w,x,y,z)
(quats is None means identity orientations).

Workloads (the sizes are the ones the benchmark and the parity tests use):

* ``two_sphere_elastance``  Laplace, 2 unit spheres, centres 2.5 apart,
  M=600 collocation / N=300 proxy points (R_p = 0.7), charges (+1, -1).
* ``sphere100_mobility``    Stokes, 100 unit spheres by random sequential
  addition in a cube at volume fraction 0.1, min gap 0.1, M=1200, N=600,
  R_p = 0.7, forces and torques i.i.d. N(0,1), seed 2.
* ``spheroid1000_mobility`` Stokes, 1000 prolate spheroids (1,1,2), random
  orientations, grown cluster with true surface-to-surface gaps U[0.05,0.5]
  (each new body at gap g from its nearest neighbour, none closer), M=2000,
  N=1000, Delta_sep = 0.25, force (0,0,-1), zero torque.
* ``sphere200_adjoint``     Stokes, 200 unit spheres at volume fraction 0.15,
  min gap 0.1, M=800, N=400, forces and torques N(0,1).
* ``batched256_mobility``   Stokes, 256 independent suspensions with body
  counts uniform in {2..64}, each body a unit sphere or a (1,1,1.5) spheroid
  (probability 1/2, random orientation), M=600, N=300, Delta_sep = 0.3,
  volume fraction 0.1, min bounding-sphere gap 0.1, 4 right-hand sides.
* ``ellipsoidT5000_mobility``, ``ellipsoidT10000_mobility``  Stokes, Type T
  ellipsoids (0.4, 0.6, 1) inside unit bounding spheres grown with every sphere
  exactly 0.2 from at least one other, random orientations, N_v = 34 (M=839,
  N=660), Delta_sep = 1.05 x 0.125, forces and torques N(0,1) (Sec. 4.2).
* ``sphere100_elastance``  the sphere100 geometry as a Laplace problem, Q ~ N(0,1).
"""

from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np

from .geometry import (
    ellipsoid_grid,
    ellipsoid_proxy,
    ellipsoid_shape_matrices,
    grow_ellipsoid_cluster,
    fibonacci_sphere,
    grow_cluster,
    random_quaternions,
    rsa_in_cube,
    spheroid_lattice,
    spheroid_proxy,
)


@dataclasses.dataclass
class Shape:
    name: str
    semi_axes: tuple  # (a, b, c)
    dsep: float
    proxy: np.ndarray  # (N, 3) body frame
    colloc: np.ndarray  # (M, 3) body frame

    @property
    def n_proxy(self) -> int:
        return self.proxy.shape[0]

    @property
    def n_colloc(self) -> int:
        return self.colloc.shape[0]

    @property
    def bounding_radius(self) -> float:
        return float(max(self.semi_axes))

    @property
    def volume(self) -> float:
        a, b, c = self.semi_axes
        return 4.0 / 3.0 * np.pi * a * b * c


@dataclasses.dataclass
class Workload:
    name: str
    kind: str  # "laplace" or "stokes"
    shapes: list
    centres: np.ndarray  # (P, 3)
    quats: Optional[np.ndarray]  # (P, 4) or None
    shape_id: np.ndarray  # (P,) int32
    body_offsets: np.ndarray  # (S+1,) int32, suspension s owns bodies [off[s], off[s+1])
    Q: Optional[np.ndarray] = None  # (P,) net charges (Laplace)
    F: Optional[np.ndarray] = None  # (nrhs, P, 3) forces (Stokes)
    T: Optional[np.ndarray] = None  # (nrhs, P, 3) torques (Stokes)
    mu: float = 1.0
    seed: int = 0
    description: str = ""

    @property
    def num_bodies(self) -> int:
        return int(self.centres.shape[0])

    def first_suspensions(self, k: int) -> "Workload":
        """The workload restricted to its first k suspensions (bodies [0, body_offsets[k]))."""
        k = min(k, self.num_suspensions)
        nb = int(self.body_offsets[k])
        cut = lambda a: None if a is None else a[..., :nb, :] if a.ndim == 3 else a[:nb]  # noqa: E731
        return Workload(
            name=f"{self.name}[:{k}]", kind=self.kind, shapes=self.shapes, centres=self.centres[:nb],
            quats=None if self.quats is None else self.quats[:nb], shape_id=self.shape_id[:nb],
            body_offsets=self.body_offsets[: k + 1].copy(), Q=cut(self.Q), F=cut(self.F), T=cut(self.T),
            mu=self.mu, seed=self.seed, description=f"first {k} suspensions of {self.name}",
        )

    def first_bodies(self, k: int) -> "Workload":
        """The first k bodies of a one-suspension workload (for a grown cluster: the compact cluster they
        formed before the later bodies were added), with their forces, torques or charges."""
        if self.num_suspensions != 1:
            raise ValueError("first_bodies needs a single suspension")
        k = min(k, self.num_bodies)
        cut = lambda a: None if a is None else a[..., :k, :] if a.ndim == 3 else a[:k]  # noqa: E731
        return Workload(
            name=f"{self.name}[:{k} bodies]", kind=self.kind, shapes=self.shapes, centres=self.centres[:k],
            quats=None if self.quats is None else self.quats[:k], shape_id=self.shape_id[:k],
            body_offsets=np.array([0, k], np.int32), Q=cut(self.Q), F=cut(self.F), T=cut(self.T),
            mu=self.mu, seed=self.seed, description=f"first {k} bodies of {self.name}",
        )

    @property
    def num_suspensions(self) -> int:
        return int(len(self.body_offsets) - 1)

    @property
    def nrhs(self) -> int:
        return 1 if self.F is None else int(self.F.shape[0])

    @property
    def dim(self) -> int:
        return 1 if self.kind == "laplace" else 3

    def counts(self):
        """Per body (M_k, N_k)."""
        m = np.array([self.shapes[s].n_colloc for s in self.shape_id])
        n = np.array([self.shapes[s].n_proxy for s in self.shape_id])
        return m, n

    def off_diagonal_pairs(self) -> int:
        """Number of (target, source) point pairs between distinct bodies of one suspension."""
        m, n = self.counts()
        total = 0
        for s in range(self.num_suspensions):
            b0, b1 = self.body_offsets[s], self.body_offsets[s + 1]
            ms, ns = m[b0:b1], n[b0:b1]
            total += int(ms.sum() * ns.sum() - (ms * ns).sum())
        return total


def sphere_shape(m: int, n: int, radius: float = 1.0, rp: float = 0.7) -> Shape:
    return Shape(
        name=f"sphere_R{radius:g}",
        semi_axes=(radius, radius, radius),
        dsep=radius - rp,
        proxy=fibonacci_sphere(n, rp),
        colloc=fibonacci_sphere(m, radius),
    )


def ellipsoid_shape(n_v: int, a: float, b: float, c: float, dsep: float, colloc_factor: float = 1.15) -> Shape:
    """Triaxial ellipsoid (Sec. 4.2): proxies on the n_v grid moved dsep inward, collocation points
    on the grid with round(1.15 n_v) Gauss-Legendre rings (M ~ 1.3 N)."""
    return Shape(
        name=f"ellipsoid_{a:g}_{b:g}_{c:g}_Nv{n_v}",
        semi_axes=(a, b, c),
        dsep=dsep,
        proxy=ellipsoid_proxy(n_v, a, b, c, dsep),
        colloc=ellipsoid_grid(int(round(colloc_factor * n_v)), a, b, c),
    )


def ellipsoid_cluster(
    count: int = 5000,
    n_v: int = 34,
    semi_axes: tuple = (0.4, 0.6, 1.0),
    dsep: float = 1.05 * 0.125,
    gap: float = 0.2,
    seed: int = 6,
    name: str = "ellipsoidT5000_mobility",
) -> Workload:
    """Type T ellipsoids (semi-axes 0.4, 0.6, 1) in a cluster of unit bounding spheres grown with each
    sphere exactly `gap` from at least one other, random orientations inside the spheres (the footnote
    of Sec. 4.2's P = 10000 example); forces and torques N(0, 1).  dsep: the resistance offset 0.125 of
    Sec. 4.2 times 1.05 for the mobility problem."""
    rng = np.random.default_rng(seed)
    shape = ellipsoid_shape(n_v, *semi_axes, dsep)
    centres = grow_cluster(rng, count, 1.0, gap, gap)
    quats = random_quaternions(rng, count)
    a, b, c = semi_axes
    return Workload(
        name=name,
        kind="stokes",
        shapes=[shape],
        centres=centres,
        quats=quats,
        shape_id=np.zeros(count, np.int32),
        body_offsets=np.array([0, count], np.int32),
        F=rng.standard_normal((1, count, 3)),
        T=rng.standard_normal((1, count, 3)),
        seed=seed,
        description=(
            f"Stokes, {count} ellipsoids ({a:g},{b:g},{c:g}) in unit bounding spheres grown at gap {gap:g}, "
            f"random orientations, N_v={n_v} (M={shape.n_colloc}, N={shape.n_proxy}), Delta_sep={dsep:.5g}, "
            "F, T ~ N(0,1)"
        ),
    )


def spheroid_shape(m: int, n: int, a: float, c: float, dsep: float) -> Shape:
    return Shape(
        name=f"spheroid_{a:g}_{a:g}_{c:g}",
        semi_axes=(a, a, c),
        dsep=dsep,
        proxy=spheroid_proxy(n, a, c, dsep),
        colloc=spheroid_lattice(m, a, c),
    )


def two_sphere_elastance(m: int = 600, n: int = 300, distance: float = 2.5, seed: int = 1) -> Workload:
    centres = np.array([[0.0, 0.0, 0.0], [distance, 0.0, 0.0]])
    return Workload(
        name="two_sphere_elastance",
        kind="laplace",
        shapes=[sphere_shape(m, n)],
        centres=centres,
        quats=None,
        shape_id=np.zeros(2, np.int32),
        body_offsets=np.array([0, 2], np.int32),
        Q=np.array([1.0, -1.0]),
        seed=seed,
        description=f"Laplace elastance, 2 unit spheres {distance} apart, M={m}, N={n}, R_p=0.7, Q=(+1,-1)",
    )


def sphere_suspension(
    count: int = 100,
    m: int = 1200,
    n: int = 600,
    volume_fraction: float = 0.1,
    min_gap: float = 0.1,
    seed: int = 2,
    kind: str = "stokes",
    nrhs: int = 1,
    name: str = "sphere100_mobility",
) -> Workload:
    rng = np.random.default_rng(seed)
    shape = sphere_shape(m, n)
    side = (count * shape.volume / volume_fraction) ** (1.0 / 3.0)
    centres = rsa_in_cube(rng, np.full(count, 1.0), side, min_gap)
    wl = Workload(
        name=name,
        kind=kind,
        shapes=[shape],
        centres=centres,
        quats=None,
        shape_id=np.zeros(count, np.int32),
        body_offsets=np.array([0, count], np.int32),
        seed=seed,
        description=(
            f"{kind}, {count} unit spheres, RSA in a cube of side {side:.4f} (volume fraction "
            f"{volume_fraction}), min gap {min_gap}, M={m}, N={n}, R_p=0.7"
        ),
    )
    if kind == "stokes":
        wl.F = rng.standard_normal((nrhs, count, 3))
        wl.T = rng.standard_normal((nrhs, count, 3))
    else:
        wl.Q = rng.standard_normal(count)
    return wl


def spheroid_cluster(
    count: int = 1000,
    m: int = 2000,
    n: int = 1000,
    a: float = 1.0,
    c: float = 2.0,
    dsep: float = 0.25,
    gap_lo: float = 0.05,
    gap_hi: float = 0.5,
    seed: int = 3,
    name: str = "spheroid1000_mobility",
) -> Workload:
    rng = np.random.default_rng(seed)
    shape = spheroid_shape(m, n, a, c, dsep)
    quats = random_quaternions(rng, count)
    centres = grow_ellipsoid_cluster(rng, ellipsoid_shape_matrices(quats, (a, a, c)), gap_lo, gap_hi)
    F = np.zeros((1, count, 3))
    F[0, :, 2] = -1.0
    return Workload(
        name=name,
        kind="stokes",
        shapes=[shape],
        centres=centres,
        quats=quats,
        shape_id=np.zeros(count, np.int32),
        body_offsets=np.array([0, count], np.int32),
        F=F,
        T=np.zeros((1, count, 3)),
        seed=seed,
        description=(
            f"Stokes, {count} prolate spheroids ({a},{a},{c}), random orientations, grown cluster with "
            f"surface gaps U[{gap_lo},{gap_hi}] (each body at gap g from its nearest neighbour), M={m}, N={n}, "
            f"Delta_sep={dsep}, F=(0,0,-1), T=0"
        ),
    )


def batched_suspensions(
    num_suspensions: int = 256,
    p_lo: int = 2,
    p_hi: int = 64,
    m: int = 600,
    n: int = 300,
    spheroid_c: float = 1.5,
    dsep: float = 0.3,
    volume_fraction: float = 0.1,
    min_gap: float = 0.1,
    nrhs: int = 4,
    seed: int = 5,
    name: str = "batched256_mobility",
) -> Workload:
    rng = np.random.default_rng(seed)
    shapes = [sphere_shape(m, n, 1.0, 1.0 - dsep), spheroid_shape(m, n, 1.0, spheroid_c, dsep)]
    counts = rng.integers(p_lo, p_hi + 1, size=num_suspensions)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    total = int(offsets[-1])
    shape_id = (rng.random(total) < 0.5).astype(np.int32)
    quats = random_quaternions(rng, total)
    centres = np.zeros((total, 3))
    for s in range(num_suspensions):
        b0, b1 = offsets[s], offsets[s + 1]
        ids = shape_id[b0:b1]
        radii = np.array([shapes[i].bounding_radius for i in ids])
        vol = sum(shapes[i].volume for i in ids)
        side = (vol / volume_fraction) ** (1.0 / 3.0)
        # keep random sequential addition far from jamming: the bounding spheres (grown by half the
        # gap) fill at most a quarter of the box their centres may occupy
        excl = sum(4.0 / 3.0 * np.pi * (r + 0.5 * min_gap) ** 3 for r in radii)
        side = max(side, (excl / 0.25) ** (1.0 / 3.0) + 2.0 * radii.max())
        centres[b0:b1] = rsa_in_cube(rng, radii, side, min_gap)
    F = rng.standard_normal((nrhs, total, 3))
    T = rng.standard_normal((nrhs, total, 3))
    return Workload(
        name=name,
        kind="stokes",
        shapes=shapes,
        centres=centres,
        quats=quats,
        shape_id=shape_id,
        body_offsets=offsets,
        F=F,
        T=T,
        seed=seed,
        description=(
            f"Stokes, {num_suspensions} independent suspensions of U{{{p_lo}..{p_hi}}} bodies "
            f"(sphere or (1,1,{spheroid_c}) spheroid), M={m}, N={n}, {nrhs} right-hand sides"
        ),
    )


WORKLOADS: dict = {
    "two_sphere_elastance": two_sphere_elastance,
    "sphere100_mobility": sphere_suspension,
    "spheroid1000_mobility": spheroid_cluster,
    "sphere200_adjoint": lambda **kw: sphere_suspension(
        **{
            "count": 200,
            "m": 800,
            "n": 400,
            "volume_fraction": 0.15,
            "seed": 4,
            "name": "sphere200_adjoint",
            **kw,
        }
    ),
    "batched256_mobility": batched_suspensions,
    "ellipsoidT5000_mobility": ellipsoid_cluster,
    "ellipsoidT10000_mobility": lambda **kw: ellipsoid_cluster(
        **{"count": 10000, "seed": 7, "name": "ellipsoidT10000_mobility", **kw}
    ),
    # the 100-sphere geometry as an elastance problem (Laplace kernel), Q ~ N(0, 1)
    "sphere100_elastance": lambda **kw: sphere_suspension(
        **{"kind": "laplace", "name": "sphere100_elastance", **kw}
    ),
}


def make_workload(name: str, **overrides) -> Workload:
    """Build a named workload; keyword overrides shrink it for tests."""
    builder: Callable = WORKLOADS[name]
    return builder(**overrides)
