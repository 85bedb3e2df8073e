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


def quaternion_rotations(quats: np.ndarray) -> np.ndarray:
    """Rotation matrices (count, 3, 3) of unit quaternions (w, x, y, z)."""
    q = np.asarray(quats, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def ellipsoid_shape_matrices(quats: np.ndarray, semi_axes) -> np.ndarray:
    """Q_k = R_k diag(a^2, b^2, c^2) R_k^T (count, 3, 3): body k is {c_k + x : x^T Q_k^-1 x <= 1}."""
    R = quaternion_rotations(quats)
    return np.einsum("kij,j,klj->kil", R, np.asarray(semi_axes, dtype=np.float64) ** 2, R)


def ellipsoid_gap(d: np.ndarray, QA: np.ndarray, QB: np.ndarray, n0=None, iters: int = 40, tol: float = 1e-14):
    """Surface-to-surface distance of ellipsoids A (centre 0, shape matrix QA) and B (centre d, QB), batched
    over the leading axis, with the unit normal that realises it.

    For disjoint convex bodies the distance is the largest separation of their support functions,
        gap = max_{|n| = 1}  n . d - sqrt(n^T QA n) - sqrt(n^T QB n),
    a concave function of n maximised on the unit sphere (Riemannian Newton steps from n0 or d/|d|,
    with backtracking).  The value is negative for overlapping bodies.  Returns (gap, n).
    """
    d = np.atleast_2d(np.asarray(d, dtype=np.float64))
    QA = np.asarray(QA, dtype=np.float64).reshape(-1, 3, 3)
    QB = np.asarray(QB, dtype=np.float64).reshape(-1, 3, 3)
    n = d / np.linalg.norm(d, axis=1, keepdims=True) if n0 is None else np.array(n0, dtype=np.float64, ndmin=2)

    def value(n):
        a = np.sqrt(np.einsum("ki,kij,kj->k", n, QA, n))
        b = np.sqrt(np.einsum("ki,kij,kj->k", n, QB, n))
        return np.einsum("ki,ki->k", n, d) - a - b, a, b

    f, a, b = value(n)
    for _ in range(iters):
        An = np.einsum("kij,kj->ki", QA, n)
        Bn = np.einsum("kij,kj->ki", QB, n)
        grad = d - An / a[:, None] - Bn / b[:, None]
        ng = np.einsum("ki,ki->k", n, grad)
        hess = -(QA / a[:, None, None] - np.einsum("ki,kj->kij", An, An) / (a ** 3)[:, None, None]) \
               - (QB / b[:, None, None] - np.einsum("ki,kj->kij", Bn, Bn) / (b ** 3)[:, None, None])
        # orthonormal tangent basis at n
        t = np.where(np.abs(n[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
        e1 = t - np.einsum("ki,ki->k", t, n)[:, None] * n
        e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
        e2 = np.cross(n, e1)
        E = np.stack([e1, e2], axis=2)  # (k, 3, 2)
        g2 = np.einsum("kia,ki->ka", E, grad)
        if np.all(np.linalg.norm(g2, axis=1) <= tol * np.maximum(1.0, np.abs(f))):
            break
        H2 = np.einsum("kia,kij,kjb->kab", E, hess, E) - ng[:, None, None] * np.eye(2)
        try:
            xi = -np.linalg.solve(H2, g2[..., None])[..., 0]
        except np.linalg.LinAlgError:
            xi = g2.copy()
        bad = np.einsum("ka,ka->k", xi, g2) <= 0.0  # not an ascent direction: use the gradient
        xi[bad] = g2[bad]
        step = np.einsum("kia,ka->ki", E, xi)
        nrm = np.linalg.norm(step, axis=1, keepdims=True)
        step = np.where(nrm > 0.5, step * (0.5 / np.maximum(nrm, 1e-300)), step)
        alpha = np.ones(len(n))
        for _ in range(30):  # backtracking: keep the steps that do not decrease the value
            cand = n + alpha[:, None] * step
            cand /= np.linalg.norm(cand, axis=1, keepdims=True)
            fc, ac, bc = value(cand)
            ok = fc >= f - 1e-15 * np.maximum(1.0, np.abs(f))
            if np.all(ok):
                break
            alpha = np.where(ok, alpha, 0.5 * alpha)
        n = np.where(ok[:, None], cand, n)
        f, a, b = np.where(ok, fc, f), np.where(ok, ac, a), np.where(ok, bc, b)
    return f, n


def grow_ellipsoid_cluster(
    rng: np.random.Generator,
    Q: np.ndarray,
    gap_lo: float,
    gap_hi: float,
) -> np.ndarray:
    """Grow a cluster of ellipsoids with true surface gaps (Sec. 4.1, Sec. 4.2).

    Q: (count, 3, 3) shape matrices (orientations drawn beforehand).  Body b draws g ~ U[gap_lo, gap_hi]
    and a random unit direction u, starts far out on the ray from the centroid of the bodies placed so
    far along u, and moves inward until its surface first comes within g of an existing body's surface
    (ellipsoid_gap).  Every body then has a neighbour at surface gap exactly g and no body closer.  The
    stopping point along the ray is, for each body j the ray passes, the outermost root of the convex
    function gap_j(s) - g (Newton from the outside: the tangent never overshoots a convex function's
    root), with bounding spheres limiting the candidates.
    """
    count = Q.shape[0]
    eig = np.linalg.eigvalsh(Q)
    Rmax = np.sqrt(eig[:, -1])  # bounding-sphere radius
    Rmin = np.sqrt(eig[:, 0])   # inscribed-sphere radius
    centres = np.zeros((count, 3))
    for b in range(1, count):
        g = rng.uniform(gap_lo, gap_hi)
        origin = centres[:b].mean(axis=0)
        while True:
            u = rng.standard_normal(3)
            u /= np.linalg.norm(u)
            rel = centres[:b] - origin
            along = rel @ u
            perp2 = np.einsum("ij,ij->i", rel, rel) - along * along
            reach = Rmax[:b] + Rmax[b] + g
            cand = np.nonzero(perp2 < reach * reach)[0]
            if cand.size == 0:
                continue
            s_hi = along[cand] + np.sqrt(reach[cand] ** 2 - perp2[cand])  # bounding spheres g apart
            inner = Rmin[cand] + Rmin[b] + g
            close = perp2[cand] < inner * inner
            # where the inscribed spheres come within g, the true gap is below g: s* is at least there
            s_floor = np.max(np.where(close, along[cand] + np.sqrt(np.maximum(inner ** 2 - perp2[cand], 0.0)),
                                      -np.inf))
            keep = s_hi > s_floor
            cand, s = cand[keep], s_hi[keep].copy()
            active = np.ones(len(cand), bool)
            nrm = None
            root = np.full(len(cand), -np.inf)
            for _ in range(60):
                d = centres[cand] - (origin + s[:, None] * u)
                f, nrm = ellipsoid_gap(d, Q[b][None].repeat(len(cand), 0), Q[cand], n0=nrm)
                slope = -(nrm @ u)  # d gap / d s
                done = np.abs(f - g) <= 1e-13 * max(1.0, g)
                root = np.where(active & done, s, root)
                miss = active & ~done & (slope <= 0.0)  # passed the minimum above g: j never blocks
                active &= ~done & ~miss
                if not np.any(active):
                    break
                s = np.where(active, s - (f - g) / np.where(slope > 0.0, slope, 1.0), s)
            s_star = root.max() if root.size else -np.inf
            if np.isfinite(s_star) and s_star > 0.0:
                break
        centres[b] = origin + s_star * u
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
