"""Point sets and body placements (inputs only; no solver arithmetic).

Discretisation choices follow the paper's setting (Sec. 2, Sec. 4.1, Sec. 4.2):
collocation points X on the physical surface, proxy (source) points Y on an
inner surface offset by Delta_sep along the inward normal.  The paper uses
spherical designs for spheres (Sec. 4.1), which are an external data set;
the paper names Fibonacci grids as the alternative it compared against, so
these generators use Fibonacci lattices:

* sphere of radius R, n points:  z_i = 1 - (2i+1)/n,  phi_i = 2 pi i / Phi^2
  (golden angle, Phi = (1+sqrt 5)/2), i = 0..n-1.
* spheroid with semi-axes (a, a, c): the same lattice made area-uniform, i.e.
  t_i = z_i / c solves A(t_i) / A_total = 1 - (i + 1/2)/n, where A(t) is the
  surface area below height c t; with a == c this reduces to the sphere rule.
* proxy surface: the collocation construction with n = N points, each point
  moved by Delta_sep along the inward unit normal (for a sphere this is the
  concentric sphere of radius R - Delta_sep).
* triaxial ellipsoid (a, b, c) (Sec. 4.2): the parameterisation
  (a sqrt(1-t^2) cos s, b sqrt(1-t^2) sin s, c t) with N_v Gauss-Legendre nodes in t and, on the
  ring at t_i, n_i equispaced s nodes (alternate rings offset by half a step), n_i proportional to
  the ring's perimeter so the surface density is roughly uniform.  The paper gives the total only
  (N ~ 17 + 3.9 N_v + 0.44 N_v^2, at most ~0.75 N_v per ring); here n_i = max(3, round(kappa L_i /
  L_max)) with kappa chosen so that the total matches that count.
"""

from __future__ import annotations

import numpy as np

GOLDEN = (1.0 + np.sqrt(5.0)) / 2.0
GOLDEN_ANGLE = 2.0 * np.pi / GOLDEN**2


def fibonacci_sphere(n: int, radius: float = 1.0) -> np.ndarray:
    """n Fibonacci-lattice points on a sphere of the given radius, shape (n, 3)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = GOLDEN_ANGLE * i
    return radius * np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def _area_primitive(t: np.ndarray, a: float, c: float) -> np.ndarray:
    """Antiderivative of sqrt(c^2 - (c^2 - a^2) t^2) (area density in t, up to 2 pi a)."""
    k2 = c * c - a * a
    if abs(k2) < 1e-14 * c * c:
        return c * t
    if k2 > 0.0:  # prolate
        k = np.sqrt(k2)
        s = np.sqrt(np.maximum(0.0, c * c - k2 * t * t))
        return 0.5 * (t * s + (c * c / k) * np.arcsin(np.clip(k * t / c, -1.0, 1.0)))
    k = np.sqrt(-k2)  # oblate
    s = np.sqrt(c * c + (-k2) * t * t)
    return 0.5 * (t * s + (c * c / k) * np.arcsinh(k * t / c))


def spheroid_lattice(n: int, a: float, c: float) -> np.ndarray:
    """Area-uniform Fibonacci lattice on the spheroid x^2/a^2 + y^2/a^2 + z^2/c^2 = 1."""
    i = np.arange(n, dtype=np.float64)
    frac = 1.0 - (i + 0.5) / n
    f_lo = _area_primitive(np.array(-1.0), a, c)
    f_hi = _area_primitive(np.array(1.0), a, c)
    target = f_lo + frac * (f_hi - f_lo)
    lo = -np.ones(n)
    hi = np.ones(n)
    for _ in range(80):  # bisection: the primitive is strictly increasing on [-1, 1]
        mid = 0.5 * (lo + hi)
        below = _area_primitive(mid, a, c) < target
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    t = 0.5 * (lo + hi)
    rho = a * np.sqrt(np.maximum(0.0, 1.0 - t * t))
    phi = GOLDEN_ANGLE * i
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), c * t], axis=1)


def spheroid_proxy(n: int, a: float, c: float, dsep: float) -> np.ndarray:
    """n proxy points: the spheroid lattice moved dsep along the inward unit normal."""
    p = spheroid_lattice(n, a, c)
    g = p / np.array([a * a, a * a, c * c])
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return p - dsep * g


def random_quaternions(rng: np.random.Generator, count: int) -> np.ndarray:
    """Uniformly distributed unit quaternions (w, x, y, z), shape (count, 4)."""
    q = rng.standard_normal((count, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def rsa_in_cube(
    rng: np.random.Generator,
    radii: np.ndarray,
    side: float,
    min_gap: float,
    max_attempts: int = 2_000_000,
) -> np.ndarray:
    """Random sequential addition of bounding spheres in a cube [0, side]^3.

    Body b has bounding radius radii[b]; its centre is uniform in
    [r_b, side - r_b]^3 and is rejected while it comes closer than
    r_b + r_j + min_gap to an accepted body j.
    """
    radii = np.asarray(radii, dtype=np.float64)
    centres = np.zeros((len(radii), 3))
    attempts = 0
    for b, r in enumerate(radii):
        while True:
            attempts += 1
            if attempts > max_attempts:
                raise RuntimeError("random sequential addition did not finish; lower the volume fraction")
            c = rng.uniform(r, side - r, size=3)
            if b == 0:
                break
            d = np.linalg.norm(centres[:b] - c, axis=1)
            if np.all(d >= radii[:b] + r + min_gap):
                break
        centres[b] = c
    return centres


def grow_cluster(
    rng: np.random.Generator,
    count: int,
    radius: float,
    gap_lo: float,
    gap_hi: float,
) -> np.ndarray:
    """Grow a cluster of bounding spheres (Sec. 4.1 and the footnote of Sec. 4.2).

    Each new sphere travels inward along a random ray through the current
    centroid and stops where it first comes within surface gap g ~ U[gap_lo,
    gap_hi] of an existing sphere, so every body has at least one neighbour at
    gap g and all others farther away.
    """
    centres = np.zeros((count, 3))
    for b in range(1, count):
        g = rng.uniform(gap_lo, gap_hi)
        dist = 2.0 * radius + g
        origin = centres[:b].mean(axis=0)
        while True:
            d = rng.standard_normal(3)
            d /= np.linalg.norm(d)
            rel = origin - centres[:b]
            bb = rel @ d
            cc = np.einsum("ij,ij->i", rel, rel) - dist * dist
            disc = bb * bb - cc
            hit = disc >= 0.0
            if not np.any(hit):
                continue
            t_out = -bb[hit] + np.sqrt(disc[hit])
            t_star = t_out.max()
            if t_star > 0.0:
                break
        centres[b] = origin + t_star * d
    return centres


def _ellipse_perimeter(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Ramanujan's second approximation to the perimeter of an ellipse with semi-axes p, q."""
    h = ((p - q) / np.maximum(p + q, 1e-300)) ** 2
    return np.pi * (p + q) * (1.0 + 3.0 * h / (10.0 + np.sqrt(4.0 - 3.0 * h)))


def ellipsoid_grid(n_v: int, a: float, b: float, c: float) -> np.ndarray:
    """Quasi-uniform grid on the ellipsoid x^2/a^2 + y^2/b^2 + z^2/c^2 = 1 with n_v Gauss-Legendre rings
    (Sec. 4.2), about 17 + 3.9 n_v + 0.44 n_v^2 points."""
    t, _ = np.polynomial.legendre.leggauss(n_v)
    rho = np.sqrt(1.0 - t * t)
    L = _ellipse_perimeter(a * rho, b * rho)
    target = 17.0 + 3.9 * n_v + 0.44 * n_v * n_v

    def counts(kappa):
        return np.maximum(3, np.rint(kappa * L / L.max()).astype(int))

    lo, hi = 1.0, 4.0 * n_v  # the total is nondecreasing in kappa: bisect for the target count
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if counts(mid).sum() < target:
            lo = mid
        else:
            hi = mid
    n_ring = counts(hi)
    pts = []
    for i, (ti, ri, ni) in enumerate(zip(t, rho, n_ring)):
        s = 2.0 * np.pi * (np.arange(ni) + 0.5 * (i % 2)) / ni
        pts.append(np.stack([a * ri * np.cos(s), b * ri * np.sin(s), np.full(ni, c * ti)], axis=1))
    return np.concatenate(pts)


def ellipsoid_proxy(n_v: int, a: float, b: float, c: float, dsep: float) -> np.ndarray:
    """The n_v ellipsoid grid moved dsep along the inward unit normal (Sec. 4.2, normal-shifted proxies)."""
    p = ellipsoid_grid(n_v, a, b, c)
    g = p / np.array([a * a, b * b, c * c])
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return p - dsep * g
