"""FP64 CPU oracle of the recompleted MFS elastance and mobility solvers.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module.  The product library
(``paper_2409_04215_gb300``) never imports it, links it or shares code with it.

What it computes (Broms, Barnett, Tornberg, "A Method of Fundamental Solutions
for Large-Scale 3D Elastance and Mobility Problems"), written plainly in FP64
with NumPy/LAPACK and plain-C direct sums (``direct_sum.c``):

* kernels: Laplace G = 1/(4 pi r) (Sec. 2.1, Eq. Skk) and the Stokeslet
  (I + r r^T/r^2)/(8 pi mu r) (Sec. 2.2, Eq. stokeslet);
* rigid-body matrices K_M, K_N with the cross-product matrix (d)_x (Eq. Kdef);
* projectors: elastance L = 1 1^T / N, L_r = 1_M 1_N^T / N (Sec. 3.1, Eq. ansatz);
  mobility L = K_N (K_N^T K_N)^{-1} K_N^T, L_r = K_M K_N^T (Sec. 3.2, Eq. Lrsto);
* one-body block S_L = S^(kk)(I - L) + L_r and its SVD pseudo-inverse applied
  in two steps V (Sigma^+ (U^T gamma)) (Sec. 2.3 Eq. pseudo, Sec. 3.3);
  congruent rotated bodies reuse one SVD: S_L^(k)+ = R_N V Sigma^+ U^T R_M^T
  (Remark "congruent", Eq. Krot);
* completion strengths alpha_0 = q/N 1 (Eq. al0) and lambda_0 = K_N (K_N^T K_N)^{-1}
  [f; t] (Eq. lambda01, lambda02); right-hand side u_0 = sum over ALL body
  pairs S^(kk') lambda_0^(k') (Eq. erhsK, Eq. stou0);
* the preconditioned square system (Eq. 2esysprec): y = gamma + sum_{k' != k}
  S^(kk') (I - L^(k')) S_L^(k')+ gamma^(k'), solved by GMRES from a zero guess
  (Algorithm 1 SOLVE); recovery lambda = S_L^+ gamma and extraction
  U = -K_N^T lambda (Eq. getU) or phi = -mean(alpha) (Eq. vkal);
* the Dirichlet problems, capacitance (Sec. 2.1) and resistance (Sec. 2.2), one-body
  preconditioned with the pseudo-inverse of the bare self block (Sec. 2.3, Eq. 2sysprec,
  Algorithm 1), charges q = sum alpha (Eq. qkgauss), forces [f; t] = K_N^T lambda (Eq. force_def).

Readings where the paper is silent or inconsistent:
the off-diagonal projector acts on the SOURCE body, L^(k') (as Eq. 2esysprec;
the block rows of Prop. 3.2 print L^(k)); viscosity mu defaults to 1; the
truncation eps_trunc defaults to 0 (Sec. 4: no truncation needed in FP64);
GMRES stops when the Arnoldi residual estimate is <= tol * ||b||.

Pins (tests/test_oracle_*.py): isolated-sphere closed forms V = Q/(4 pi a),
U = F/(6 pi mu a), Omega = T/(8 pi mu a^3); the two-sphere potential from the
bispherical and image-charge series; prolate-spheroid drag and capacitance;
the Rotne-Prager far field; exact algebraic identities of the projectors;
direct sums against assembled dense matrices; GMRES against dense LU; SPD and
symmetric mobility/elastance matrices; surface residuals; finite differences
for the adjoint.
"""

from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import List, Optional, Sequence

import numpy as np

PI = np.pi

# ---------------------------------------------------------------------------
# Plain-C direct sums (optional; NumPy fallback below)
# ---------------------------------------------------------------------------

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def _clib():
    global _LIB
    if _LIB is None:
        path = os.path.join(_HERE, "_direct_sum.so")
        if not os.path.exists(path):
            from . import build as _b

            _b.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_laplace_sum.argtypes = [
            ctypes.c_long, dp, ip, ip, ctypes.c_long, dp, ip, ip, dp, ctypes.c_int, dp]
        lib.oracle_stokeslet_sum.argtypes = [
            ctypes.c_long, dp, ip, ip, ctypes.c_long, dp, ip, ip, dp, ctypes.c_int, ctypes.c_double, dp]
        lib.oracle_stokeslet_center_grad.argtypes = [
            ctypes.c_long, dp, ip, ip, dp, ctypes.c_long, dp, ip, ip, dp, ctypes.c_double, ctypes.c_int, dp]
        _LIB = lib
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def direct_sum(kind, x, tgroup, tbody, y, sgroup, sbody, strength, include_self, mu=1.0):
    """sum_j G(x_i - y_j) s_j over same-group pairs (skipping same-body pairs unless include_self)."""
    lib = _clib()
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    s = np.ascontiguousarray(strength, np.float64)
    tg = np.ascontiguousarray(tgroup, np.int32)
    tb = np.ascontiguousarray(tbody, np.int32)
    sg = np.ascontiguousarray(sgroup, np.int32)
    sb = np.ascontiguousarray(sbody, np.int32)
    nt, ns = x.shape[0], y.shape[0]
    if kind == "laplace":
        out = np.zeros(nt)
        lib.oracle_laplace_sum(nt, _dp(x), _ip(tg), _ip(tb), ns, _dp(y), _ip(sg), _ip(sb), _dp(s),
                               int(include_self), _dp(out))
    else:
        out = np.zeros((nt, 3))
        lib.oracle_stokeslet_sum(nt, _dp(x), _ip(tg), _ip(tb), ns, _dp(y), _ip(sg), _ip(sb), _dp(s),
                                 int(include_self), float(mu), _dp(out))
    return out


# ---------------------------------------------------------------------------
# Kernels and one-body matrices
# ---------------------------------------------------------------------------


def quat_to_rotation(q: np.ndarray) -> np.ndarray:
    """Rotation matrix of the unit quaternion q = (w, x, y, z)."""
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def laplace_matrix(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """S_ij = 1 / (4 pi |x_i - y_j|)  (Sec. 2.1, Eq. Skk)."""
    r = np.linalg.norm(X[:, None, :] - Y[None, :, :], axis=2)
    return 1.0 / (4.0 * PI * r)


def stokeslet_matrix(X: np.ndarray, Y: np.ndarray, mu: float = 1.0) -> np.ndarray:
    """3M x 3N matrix whose (i, j) 3x3 block is (I + r r^T/r^2) / (8 pi mu r), r = x_i - y_j (Eq. stokeslet)."""
    r = X[:, None, :] - Y[None, :, :]
    rn = np.linalg.norm(r, axis=2)
    blk = np.eye(3)[None, None] + r[..., :, None] * r[..., None, :] / (rn**2)[..., None, None]
    blk /= (8.0 * PI * mu * rn)[..., None, None]
    M, N = X.shape[0], Y.shape[0]
    return blk.transpose(0, 2, 1, 3).reshape(3 * M, 3 * N)


def cross_matrix(d: np.ndarray) -> np.ndarray:
    """(d)_x of Eq. Kdef: [[0, d3, -d2], [-d3, 0, d1], [d2, -d1, 0]], so (d)_x w = w x d."""
    return np.array([[0.0, d[2], -d[1]], [-d[2], 0.0, d[0]], [d[1], -d[0], 0.0]])


def rigid_body_matrix(pts: np.ndarray, centre: np.ndarray) -> np.ndarray:
    """K (3n x 6) with block rows [I_3, (p_i - c)_x]  (Eq. Kdef)."""
    n = pts.shape[0]
    K = np.zeros((3 * n, 6))
    for i in range(n):
        K[3 * i:3 * i + 3, 0:3] = np.eye(3)
        K[3 * i:3 * i + 3, 3:6] = cross_matrix(pts[i] - centre)
    return K


@dataclasses.dataclass
class ShapeFactors:
    """Per-shape one-body operators in the body frame (Sec. 3.3 and Remark congruent)."""

    kind: str
    S0: np.ndarray  # self block S^(00), dM x dN
    L: np.ndarray  # dN x dN projector
    Lr: np.ndarray  # dM x dN
    SL: np.ndarray  # S_L = S0 (I - L) + Lr
    U: np.ndarray  # dM x r
    sigma: np.ndarray  # r
    Vt: np.ndarray  # r x dN
    sigma_pinv: np.ndarray  # r, 1/sigma or 0 below sigma_1 * eps_trunc
    KN0: Optional[np.ndarray] = None
    KM0: Optional[np.ndarray] = None

    @property
    def cond(self) -> float:
        return float(self.sigma[0] / self.sigma[-1])


def shape_factors(shape, kind: str, mu: float = 1.0, eps_trunc: float = 0.0) -> ShapeFactors:
    X0, Y0 = shape.colloc, shape.proxy
    M, N = X0.shape[0], Y0.shape[0]
    KN0 = KM0 = None
    if kind == "laplace":
        S0 = laplace_matrix(X0, Y0)
        L = np.full((N, N), 1.0 / N)  # Sec. 3.1
        Lr = np.full((M, N), 1.0 / N)  # Eq. ansatz
    else:
        S0 = stokeslet_matrix(X0, Y0, mu)
        KN0 = rigid_body_matrix(Y0, np.zeros(3))
        KM0 = rigid_body_matrix(X0, np.zeros(3))
        L = KN0 @ np.linalg.solve(KN0.T @ KN0, KN0.T)  # Sec. 3.2
        Lr = KM0 @ KN0.T  # Eq. Lrsto
    dN = L.shape[0]
    SL = S0 @ (np.eye(dN) - L) + Lr  # Sec. 3.3
    U, s, Vt = np.linalg.svd(SL, full_matrices=False)  # Eq. pseudo
    keep = s > s[0] * eps_trunc
    sinv = np.where(keep, 1.0 / np.where(keep, s, 1.0), 0.0)
    return ShapeFactors(kind, S0, L, Lr, SL, U, s, Vt, sinv, KN0, KM0)


@dataclasses.dataclass
class DirichletFactors:
    """SVD of the bare self block S^(00) = U Sigma V^T of one shape (Sec. 2.3, Eq. pseudo)."""

    U: np.ndarray  # dM x r
    sigma: np.ndarray  # r
    Vt: np.ndarray  # r x dN
    sigma_pinv: np.ndarray  # r, 1/sigma or 0 below sigma_1 * eps_trunc


def dirichlet_factors(f: ShapeFactors, eps_trunc: float = 0.0) -> DirichletFactors:
    U, s, Vt = np.linalg.svd(f.S0, full_matrices=False)
    keep = s > s[0] * eps_trunc
    sinv = np.where(keep, 1.0 / np.where(keep, s, 1.0), 0.0)
    return DirichletFactors(U, s, Vt, sinv)


# ---------------------------------------------------------------------------
# GMRES (Algorithm 1 SOLVE uses GMRES; zero initial guess, no restart)
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    residual_estimate: float  # |g_{k}| / ||b||
    converged: bool


def gmres(matvec, b: np.ndarray, tol: float = 1e-12, max_iter: int = 200) -> GmresResult:
    """Unrestarted GMRES, Arnoldi by modified Gram-Schmidt with one re-orthogonalisation pass."""
    n = b.shape[0]
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        return GmresResult(np.zeros(n), 0, 0.0, True)
    m = max_iter
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    cs = np.zeros(m)
    sn = np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = beta
    V[0] = b / beta
    k = 0
    converged = False
    for j in range(m):
        w = matvec(V[j])
        for _ in range(2):
            for i in range(j + 1):
                h = float(V[i] @ w)
                H[i, j] += h
                w = w - h * V[i]
        hn = float(np.linalg.norm(w))
        H[j + 1, j] = hn
        if hn > 0.0:
            V[j + 1] = w / hn
        for i in range(j):  # previous Givens rotations
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        den = np.hypot(H[j, j], H[j + 1, j])
        cs[j] = H[j, j] / den
        sn[j] = H[j + 1, j] / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        if abs(g[k]) <= tol * beta or hn == 0.0:
            converged = True
            break
    y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
    x = V[:k].T @ y
    return GmresResult(x, k, abs(g[k]) / beta, converged)


# ---------------------------------------------------------------------------
# The multi-body problem
# ---------------------------------------------------------------------------


class Problem:
    """A workload (mfs_inputs.Workload) discretised for the oracle.

    Vectors on collocation points are per-body arrays of shape (M_k * d,),
    point-major with the d components interleaved; on proxy points (N_k * d,).
    """

    def __init__(self, wl, eps_trunc: float = 0.0, use_c: bool = True):
        self.wl = wl
        self.eps_trunc = eps_trunc
        self._dfactors: Optional[List[DirichletFactors]] = None
        self.kind = wl.kind
        self.d = 1 if wl.kind == "laplace" else 3
        self.mu = float(wl.mu)
        self.P = wl.num_bodies
        self.use_c = use_c
        self.factors = [shape_factors(sh, wl.kind, wl.mu, eps_trunc) for sh in wl.shapes]
        if wl.quats is None:
            self.R = np.broadcast_to(np.eye(3), (self.P, 3, 3)).copy()
        else:
            self.R = np.stack([quat_to_rotation(q) for q in wl.quats])
        self.group = np.zeros(self.P, np.int32)
        for s in range(wl.num_suspensions):
            self.group[wl.body_offsets[s]:wl.body_offsets[s + 1]] = s
        self.X: List[np.ndarray] = []
        self.Y: List[np.ndarray] = []
        for k in range(self.P):
            sh = wl.shapes[wl.shape_id[k]]
            self.X.append(wl.centres[k] + sh.colloc @ self.R[k].T)
            self.Y.append(wl.centres[k] + sh.proxy @ self.R[k].T)

    # -- per-body helpers ---------------------------------------------------
    def shape_of(self, k: int) -> ShapeFactors:
        return self.factors[self.wl.shape_id[k]]

    def suspension_bodies(self, s: int) -> np.ndarray:
        return np.arange(self.wl.body_offsets[s], self.wl.body_offsets[s + 1])

    def rotate_points(self, k: int, v: np.ndarray, transpose: bool) -> np.ndarray:
        """Apply R_k (or R_k^T) to every 3-vector of v (Stokes only; identity for Laplace)."""
        if self.d == 1:
            return v
        R = self.R[k].T if transpose else self.R[k]
        return (v.reshape(-1, 3) @ R.T).reshape(-1)

    def K_N(self, k: int) -> np.ndarray:
        return rigid_body_matrix(self.Y[k], self.wl.centres[k])

    def K_M(self, k: int) -> np.ndarray:
        return rigid_body_matrix(self.X[k], self.wl.centres[k])

    def project(self, k: int, lam: np.ndarray) -> np.ndarray:
        """(I - L^(k)) lam: remove the mean (Sec. 3.1) or the rigid-body part (Sec. 3.2)."""
        if self.d == 1:
            return lam - lam.mean()
        KN = self.K_N(k)
        return lam - KN @ np.linalg.solve(KN.T @ KN, KN.T @ lam)

    def pinv_apply(self, k: int, gamma_k: np.ndarray, project: bool) -> np.ndarray:
        """S_L^(k)+ gamma = R_N V (Sigma^+ (U^T (R_M^T gamma)))  (Eq. pseudo, Remark congruent)."""
        f = self.shape_of(k)
        g = self.rotate_points(k, gamma_k, transpose=True)
        t = f.sigma_pinv * (f.U.T @ g)
        lam = self.rotate_points(k, f.Vt.T @ t, transpose=False)
        return self.project(k, lam) if project else lam

    # -- direct sums --------------------------------------------------------
    def pair_sum(self, bodies: Sequence[int], strengths: Sequence[np.ndarray], include_self: bool,
                 target_bodies: Optional[Sequence[int]] = None,
                 target_rows: Optional[Sequence[np.ndarray]] = None) -> List[np.ndarray]:
        """u^(k) = sum over k' in `bodies` (k' != k unless include_self) of S^(kk') s^(k').

        Targets are the collocation points of `target_bodies` (default: `bodies`),
        optionally only the rows `target_rows[t]` of each.
        """
        if target_bodies is None:
            target_bodies = bodies
        d = self.d
        xs, tg, tb, counts = [], [], [], []
        for t, k in enumerate(target_bodies):
            rows = np.arange(self.X[k].shape[0]) if target_rows is None else np.asarray(target_rows[t])
            xs.append(self.X[k][rows])
            tg.append(np.full(len(rows), self.group[k], np.int32))
            tb.append(np.full(len(rows), k, np.int32))
            counts.append(len(rows))
        ys, sg, sb, ss = [], [], [], []
        for k, s in zip(bodies, strengths):
            ys.append(self.Y[k])
            sg.append(np.full(self.Y[k].shape[0], self.group[k], np.int32))
            sb.append(np.full(self.Y[k].shape[0], k, np.int32))
            ss.append(np.asarray(s).reshape(-1, d) if d == 3 else np.asarray(s).reshape(-1))
        x = np.concatenate(xs)
        y = np.concatenate(ys)
        strength = np.concatenate(ss)
        tgroup, tbody = np.concatenate(tg), np.concatenate(tb)
        sgroup, sbody = np.concatenate(sg), np.concatenate(sb)
        if self.use_c:
            out = direct_sum(self.kind, x, tgroup, tbody, y, sgroup, sbody, strength, include_self, self.mu)
        else:
            out = self._pair_sum_numpy(x, tgroup, tbody, y, sgroup, sbody, strength, include_self)
        res, o = [], 0
        for c in counts:
            res.append(out[o:o + c].reshape(-1).copy())
            o += c
        return res

    def _pair_sum_numpy(self, x, tgroup, tbody, y, sgroup, sbody, strength, include_self):
        d = self.d
        out = np.zeros((x.shape[0], d)) if d == 3 else np.zeros(x.shape[0])
        for kt in np.unique(tbody):
            ti = np.nonzero(tbody == kt)[0]
            for ks in np.unique(sbody):
                if not include_self and ks == kt:
                    continue
                si = np.nonzero(sbody == ks)[0]
                if sgroup[si[0]] != tgroup[ti[0]]:
                    continue
                if d == 1:
                    out[ti] += laplace_matrix(x[ti], y[si]) @ strength[si]
                else:
                    out[ti] += (stokeslet_matrix(x[ti], y[si], self.mu) @ strength[si].reshape(-1)).reshape(-1, 3)
        return out

    # -- the preconditioned operator (Eq. 2esysprec) --------------------------
    def split(self, bodies: Sequence[int], vec: np.ndarray, on: str = "colloc") -> List[np.ndarray]:
        out, o = [], 0
        for k in bodies:
            n = (self.X[k] if on == "colloc" else self.Y[k]).shape[0] * self.d
            out.append(vec[o:o + n])
            o += n
        return out

    def matvec(self, bodies: Sequence[int], gamma: np.ndarray) -> np.ndarray:
        """y = gamma + sum_{k' != k} S^(kk') (I - L^(k')) S_L^(k')+ gamma^(k')  (Eq. 2esysprec)."""
        g = self.split(bodies, gamma)
        lam_hat = [self.pinv_apply(k, gk, project=True) for k, gk in zip(bodies, g)]
        u = self.pair_sum(bodies, lam_hat, include_self=False)
        return gamma + np.concatenate(u)

    def precond_apply(self, bodies: Sequence[int], gamma: np.ndarray, project: bool) -> np.ndarray:
        g = self.split(bodies, gamma)
        return np.concatenate([self.pinv_apply(k, gk, project) for k, gk in zip(bodies, g)])

    # -- adjoint (the paper gives none; derived from Eq. 2esysprec, Eq. stou0, Eq. getU) --------
    #
    # U = E gamma with E = -K_N^T S_L^+ (block diagonal, independent of the centres), and
    # A(c) gamma = b(c) = -u_0(c).  For a loss L(U):  g_gamma = E^T dL/dU,  A^T w = g_gamma,
    # dL = w^T (db - dA gamma) = -sum_{k != k'} w_k^T dS^(kk') mu_k',  mu = lambda_0 + (I - L) S_L^+ gamma,
    # where only the off-diagonal blocks depend on the centres (through r = c_k - c_k' + ...).
    def pinv_apply_T(self, k: int, x: np.ndarray, project: bool) -> np.ndarray:
        """(S_L^(k)+)^T x = R_M U Sigma^+ V^T R_N^T x, after (I - L^(k)) when project (L is symmetric)."""
        f = self.shape_of(k)
        if project:
            x = self.project(k, x)
        t = f.sigma_pinv * (f.Vt @ self.rotate_points(k, x, transpose=True))
        return self.rotate_points(k, f.U @ t, transpose=False)

    def pair_sum_T(self, bodies: Sequence[int], w: Sequence[np.ndarray], include_self: bool) -> List[np.ndarray]:
        """z^(k') = sum_k S^(kk')^T w^(k) at the proxy points (G is symmetric and even in r)."""
        d = self.d
        x = np.concatenate([self.Y[k] for k in bodies])
        tg = np.concatenate([np.full(self.Y[k].shape[0], self.group[k], np.int32) for k in bodies])
        tb = np.concatenate([np.full(self.Y[k].shape[0], k, np.int32) for k in bodies])
        y = np.concatenate([self.X[k] for k in bodies])
        sg = np.concatenate([np.full(self.X[k].shape[0], self.group[k], np.int32) for k in bodies])
        sb = np.concatenate([np.full(self.X[k].shape[0], k, np.int32) for k in bodies])
        s = np.concatenate([np.asarray(v).reshape(-1, d) if d == 3 else np.asarray(v) for v in w])
        out = direct_sum(self.kind, x, tg, tb, y, sg, sb, s, include_self, self.mu)
        res, o = [], 0
        for k in bodies:
            n = self.Y[k].shape[0]
            res.append(out[o:o + n].reshape(-1).copy())
            o += n
        return res

    def matvec_T(self, bodies: Sequence[int], w: np.ndarray) -> np.ndarray:
        """A^T w = w + [((I - L^(k')) S_L^(k')+)^T sum_{k != k'} S^(kk')^T w^(k)]_k'."""
        z = self.pair_sum_T(bodies, self.split(bodies, w), include_self=False)
        return w + np.concatenate([self.pinv_apply_T(k, zk, project=True) for k, zk in zip(bodies, z)])

    def mobility_vjp(self, F: np.ndarray, T: np.ndarray, dU: np.ndarray, dW: np.ndarray, tol: float = 1e-13,
                     max_iter: int = 300):
        """dL/dc [P][3], dL/dF, dL/dT [P][3] for the cotangents dU = dL/dU, dW = dL/dOmega."""
        grad_c = np.zeros((self.P, 3))
        gF = np.zeros((self.P, 3))
        gT = np.zeros((self.P, 3))
        for s in range(self.wl.num_suspensions):
            bodies = list(self.suspension_bodies(s))
            lam0 = [self.lambda0(k, F[k], T[k]) for k in bodies]
            u0 = np.concatenate(self.pair_sum(bodies, lam0, include_self=True))
            gamma = gmres(lambda v: self.matvec(bodies, v), -u0, tol, max_iter).x
            # g_gamma = E^T dL/dU = -(S_L^+)^T K_N [dU; dW]
            gg = np.concatenate([-self.pinv_apply_T(k, self.K_N(k) @ np.concatenate([dU[k], dW[k]]), False)
                                 for k in bodies])
            w = gmres(lambda v: self.matvec_T(bodies, v), gg, tol, max_iter).x
            mu = [l0 + self.pinv_apply(k, gk, project=True)
                  for k, l0, gk in zip(bodies, lam0, self.split(bodies, gamma))]
            grad_c[bodies] -= self.centre_gradient(bodies, self.split(bodies, w), mu)[bodies]
            # dL/dlambda_0 = -S_full^T w (all pairs, Eq. stou0); lambda_0 = K_N G^-1 [f; t]
            z = self.pair_sum_T(bodies, self.split(bodies, w), include_self=True)
            for k, zk in zip(bodies, z):
                KN = self.K_N(k)
                g6 = -np.linalg.solve(KN.T @ KN, KN.T @ zk)
                gF[k], gT[k] = g6[:3], g6[3:]
        return grad_c, gF, gT

    def centre_gradient(self, bodies: Sequence[int], w: Sequence[np.ndarray], mu: Sequence[np.ndarray]):
        """sum over off-diagonal pairs of d/dr [w_i^T G(r_ij) mu_j], +1 to the target body, -1 to the source body."""
        x = np.concatenate([self.X[k] for k in bodies])
        tg = np.concatenate([np.full(self.X[k].shape[0], self.group[k], np.int32) for k in bodies])
        tb = np.concatenate([np.full(self.X[k].shape[0], k, np.int32) for k in bodies])
        y = np.concatenate([self.Y[k] for k in bodies])
        sg = np.concatenate([np.full(self.Y[k].shape[0], self.group[k], np.int32) for k in bodies])
        sb = np.concatenate([np.full(self.Y[k].shape[0], k, np.int32) for k in bodies])
        ww = np.ascontiguousarray(np.concatenate([np.asarray(v).reshape(-1, 3) for v in w]))
        mm = np.ascontiguousarray(np.concatenate([np.asarray(v).reshape(-1, 3) for v in mu]))
        g = np.zeros((self.P, 3))
        lib = _clib()
        xs, ys = np.ascontiguousarray(x), np.ascontiguousarray(y)
        lib.oracle_stokeslet_center_grad(x.shape[0], _dp(xs), _ip(tg), _ip(tb), _dp(ww), y.shape[0], _dp(ys),
                                         _ip(sg), _ip(sb), _dp(mm), float(self.mu), int(self.P), _dp(g))
        return g

    # -- completion (Sec. 3.1, Sec. 3.2) -------------------------------------
    def lambda0(self, k: int, f: np.ndarray, t: np.ndarray) -> np.ndarray:
        """lambda_0 = K_N (K_N^T K_N)^{-1} [f; t]  (Eq. lambda01, lambda02)."""
        KN = self.K_N(k)
        return KN @ np.linalg.solve(KN.T @ KN, np.concatenate([f, t]))

    def alpha0(self, k: int, q: float) -> np.ndarray:
        """alpha_0 = q / N 1_N  (Eq. al0)."""
        n = self.Y[k].shape[0]
        return np.full(n, q / n)

    # -- solves -----------------------------------------------------------------
    def solve_mobility(self, F: np.ndarray, T: np.ndarray, tol: float = 1e-12, max_iter: int = 200):
        """(U, Omega, info) for forces/torques F, T of shape (P, 3) (Prop. 3.2 with Eq. 2esysprec)."""
        U = np.zeros((self.P, 3))
        W = np.zeros((self.P, 3))
        info = []
        for s in range(self.wl.num_suspensions):
            bodies = list(self.suspension_bodies(s))
            lam0 = [self.lambda0(k, F[k], T[k]) for k in bodies]
            u0 = np.concatenate(self.pair_sum(bodies, lam0, include_self=True))  # Eq. stou0
            res = gmres(lambda v: self.matvec(bodies, v), -u0, tol, max_iter)
            lam = self.split(bodies, self.precond_apply(bodies, res.x, project=False), on="proxy")
            for k, lk in zip(bodies, lam):
                uk = -self.K_N(k).T @ lk  # Eq. getU
                U[k], W[k] = uk[:3], uk[3:]
            info.append(res)
        return U, W, info

    def solve_elastance(self, Q: np.ndarray, tol: float = 1e-12, max_iter: int = 200):
        """(phi, info) for net charges Q of shape (P,) (Prop. 3.1 with Eq. 2esysprec)."""
        phi = np.zeros(self.P)
        info = []
        for s in range(self.wl.num_suspensions):
            bodies = list(self.suspension_bodies(s))
            a0 = [self.alpha0(k, Q[k]) for k in bodies]
            u0 = np.concatenate(self.pair_sum(bodies, a0, include_self=True))  # Eq. erhsK
            res = gmres(lambda v: self.matvec(bodies, v), -u0, tol, max_iter)
            alpha = self.split(bodies, self.precond_apply(bodies, res.x, project=False), on="proxy")
            for k, ak in zip(bodies, alpha):
                phi[k] = -ak.mean()  # Eq. vkal
            info.append(res)
        return phi, info

    # -- diagnostics ------------------------------------------------------------
    def total_strengths_mobility(self, bodies, gamma, F, T):
        """mu^(k) = (I - L^(k)) S_L^(k)+ gamma^(k) + lambda_0^(k): the strengths of the representation (Eq. multirep)."""
        g = self.split(bodies, gamma)
        return [self.pinv_apply(k, gk, project=True) + self.lambda0(k, F[k], T[k]) for k, gk in zip(bodies, g)]

    def total_strengths_elastance(self, bodies, gamma, Q):
        """alpha^(k) = (I - L^(k)) S_L^(k)+ gamma^(k) + alpha_0^(k): the strengths of the representation (Eq. erepK)."""
        g = self.split(bodies, gamma)
        return [self.pinv_apply(k, gk, project=True) + self.alpha0(k, Q[k]) for k, gk in zip(bodies, g)]

    def strengths_dirichlet(self, bodies, gamma):
        """alpha^(k) = S^(kk)+ gamma^(k) (Eq. reconbal): the strengths of a Dirichlet solve."""
        return [self.pinv_apply_dirichlet(k, gk) for k, gk in zip(bodies, self.split(bodies, gamma))]

    def evaluate(self, bodies, strengths, points: np.ndarray) -> np.ndarray:
        """u(x) = sum_{k in bodies} sum_j G(x - y_j^(k)) beta_j^(k) at arbitrary points (P_e, 3) (Eq. rep,
        Eq. repS); returns (P_e,) potentials or (P_e, 3) velocities.  Dense kernel matrices: small cases."""
        out = np.zeros(points.shape[0] * self.d)
        for k, bk in zip(bodies, strengths):
            if self.d == 1:
                out += laplace_matrix(points, self.Y[k]) @ bk
            else:
                out += stokeslet_matrix(points, self.Y[k], self.mu) @ bk
        return out if self.d == 1 else out.reshape(-1, 3)

    def evaluate_stress(self, bodies, strengths, points: np.ndarray, normals: np.ndarray):
        """Pressure p and traction T = sigma n of the Stokeslet representation at points with unit normals
        (Eq. traction): per source, p = (r . lambda) / (4 pi r^3) (the pressure fundamental solution
        Pi = 2 r / r^3 with the 1/(8 pi) of Sec. 2.2) and sigma_ik = -3 r_i r_k (r . lambda) / (4 pi r^5),
        r = x - y; both independent of mu.  Returns (p (P_e,), T (P_e, 3))."""
        p = np.zeros(points.shape[0])
        T = np.zeros((points.shape[0], 3))
        for k, bk in zip(bodies, strengths):
            lam = bk.reshape(-1, 3)
            r = points[:, None, :] - self.Y[k][None, :, :]  # (P_e, N, 3)
            rn = np.linalg.norm(r, axis=2)
            rl = np.einsum("ijk,jk->ij", r, lam)
            p += np.sum(rl / rn**3, axis=1) / (4.0 * PI)
            rnrm = np.einsum("ijk,ik->ij", r, normals)
            T += -3.0 / (4.0 * PI) * np.einsum("ij,ijk->ik", rl * rnrm / rn**5, r)
        return p, T

    def surface_field(self, bodies, strengths, targets=None):
        """The representation evaluated at collocation points: all pairs including self."""
        return self.pair_sum(bodies, strengths, include_self=True, target_bodies=targets)

    # -- Dirichlet problems: capacitance (Sec. 2.1) and resistance (Sec. 2.2) -------------
    #
    # One-body right preconditioning with the pseudo-inverse of the bare self block S^(kk)
    # (Sec. 2.3): gamma^(k) = S^(kk) alpha^(k), diagonal blocks replaced by the identity, giving the
    # square system Eq. 2sysprec with the Dirichlet data as right-hand side; alpha = S^+ gamma after.
    def dirichlet_factors(self, k: int) -> "DirichletFactors":
        if self._dfactors is None:
            self._dfactors = [dirichlet_factors(f, self.eps_trunc) for f in self.factors]
        return self._dfactors[self.wl.shape_id[k]]

    def pinv_apply_dirichlet(self, k: int, gamma_k: np.ndarray) -> np.ndarray:
        """S^(kk)+ gamma = R_N V (Sigma^+ (U^T (R_M^T gamma))) from the SVD of S^(00) (Eq. pseudo,
        Remark congruent: S^(kk) = R_M S^(00) R_N^T for a rotated copy)."""
        f = self.dirichlet_factors(k)
        g = self.rotate_points(k, gamma_k, transpose=True)
        t = f.sigma_pinv * (f.U.T @ g)
        return self.rotate_points(k, f.Vt.T @ t, transpose=False)

    def matvec_dirichlet(self, bodies: Sequence[int], gamma: np.ndarray) -> np.ndarray:
        """y = gamma + sum_{k' != k} S^(kk') S^(k'k')+ gamma^(k')  (Eq. 2sysprec; Algorithm 1 MATVEC:
        the self contribution evaluated and subtracted there is simply never added here)."""
        g = self.split(bodies, gamma)
        alpha_hat = [self.pinv_apply_dirichlet(k, gk) for k, gk in zip(bodies, g)]
        return gamma + np.concatenate(self.pair_sum(bodies, alpha_hat, include_self=False))

    def _solve_dirichlet(self, eta_of, tol: float, max_iter: int):
        """Algorithm 1 SOLVE per suspension: gamma = GMRES(MATVEC, eta), alpha^(k) = S^(kk)+ gamma^(k)."""
        strengths: List[Optional[np.ndarray]] = [None] * self.P
        info = []
        for s in range(self.wl.num_suspensions):
            bodies = list(self.suspension_bodies(s))
            eta = np.concatenate([eta_of(k) for k in bodies])
            res = gmres(lambda v: self.matvec_dirichlet(bodies, v), eta, tol, max_iter)
            for k, gk in zip(bodies, self.split(bodies, res.x)):
                strengths[k] = self.pinv_apply_dirichlet(k, gk)
            info.append(res)
        return strengths, info

    def solve_capacitance(self, phi: np.ndarray, tol: float = 1e-12, max_iter: int = 200):
        """(q, info): net charges of conductors held at potentials phi (P,): eta^(k) = phi^(k) 1_M
        (Sec. 2.1), q^(k) = sum_j alpha_j^(k) (Eq. qkgauss)."""
        alpha, info = self._solve_dirichlet(lambda k: np.full(self.X[k].shape[0], float(phi[k])), tol, max_iter)
        return np.array([a.sum() for a in alpha]), info

    def solve_resistance(self, U: np.ndarray, W: np.ndarray, tol: float = 1e-12, max_iter: int = 200):
        """(F, T, info) for rigid-body velocities U, W (P, 3): b = K_M [v; omega] (Sec. 2.2, Eq. Kdef,
        Eq. Kbig), [f; t] = K_N^T lambda (Eq. force_def)."""
        lam, info = self._solve_dirichlet(lambda k: self.K_M(k) @ np.concatenate([U[k], W[k]]), tol, max_iter)
        FT = np.array([self.K_N(k).T @ lk for k, lk in enumerate(lam)])
        return FT[:, :3], FT[:, 3:], info

    def assemble_dense(self, bodies: Sequence[int]) -> np.ndarray:
        """Eq. 2esysprec as a dense matrix, with S^(kk') from explicit kernel matrices (tiny problems only)."""
        d = self.d
        sizes = [self.X[k].shape[0] * d for k in bodies]
        offs = np.concatenate([[0], np.cumsum(sizes)])
        A = np.eye(offs[-1])
        for jj, kp in enumerate(bodies):
            f = self.shape_of(kp)
            if d == 1:
                pinv = f.Vt.T @ (f.sigma_pinv[:, None] * f.U.T)
                proj = np.eye(f.L.shape[0]) - f.L
            else:
                RN = np.kron(np.eye(self.Y[kp].shape[0]), self.R[kp])
                RM = np.kron(np.eye(self.X[kp].shape[0]), self.R[kp])
                pinv = RN @ f.Vt.T @ (f.sigma_pinv[:, None] * f.U.T) @ RM.T
                KN = self.K_N(kp)
                proj = np.eye(KN.shape[0]) - KN @ np.linalg.solve(KN.T @ KN, KN.T)
            B = proj @ pinv
            for ii, k in enumerate(bodies):
                if k == kp:
                    continue
                if d == 1:
                    S = laplace_matrix(self.X[k], self.Y[kp])
                else:
                    S = stokeslet_matrix(self.X[k], self.Y[kp], self.mu)
                A[offs[ii]:offs[ii + 1], offs[jj]:offs[jj + 1]] = S @ B
        return A


def split_workload(wl, s: int):
    """The single-suspension workload of suspension s of a batched workload."""
    b0, b1 = int(wl.body_offsets[s]), int(wl.body_offsets[s + 1])
    sub = dataclasses.replace(
        wl,
        centres=wl.centres[b0:b1].copy(),
        quats=None if wl.quats is None else wl.quats[b0:b1].copy(),
        shape_id=wl.shape_id[b0:b1].copy(),
        body_offsets=np.array([0, b1 - b0], np.int32),
        Q=None if wl.Q is None else wl.Q[b0:b1].copy(),
        F=None if wl.F is None else wl.F[:, b0:b1].copy(),
        T=None if wl.T is None else wl.T[:, b0:b1].copy(),
    )
    return sub
