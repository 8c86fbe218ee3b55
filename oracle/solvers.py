"""Krylov and eigen solvers of the oracle.

* ``pcg``: preconditioned CG (Hestenes-Stiefel), stopped when
  ||r_k||_2 <= rtol ||r_0||_2 (Sec. 4.1, rTOL = 1e-8; k_max = 10000, Sec. 4.2).
* ``inverse_iteration``: the shifted inverse power method of Sec. 2,
  x_{k+1} = A_sigma^{-1} B x_k followed by B-normalisation, each solve by PCG
  with zero initial guess (Sec. 4.2).  Start vector 1/||1||_B (Sec. 4.2).
  Rayleigh quotient R(x) = x^T A x / x^T B x and spectral residual
  r = A x - R(x) B x (Sec. 2).  Stop when
  eta = ||A x - rho B x||_2 / (|rho| ||B x||_2) <= tol_res and
  |rho_k - rho_{k-1}| <= tol_lam |rho_k|.
* ``gmres``: right-preconditioned restarted GMRES (Arnoldi with modified Gram-Schmidt,
  Givens rotations), the Krylov method for the unsymmetric M_RAS2^{-1} (Sec. 2.2); stopped
  when its own residual (the least-squares residual of the Arnoldi relation, |g_{j+1}|)
  satisfies ||r_k||_2 <= rtol ||r_0||_2, as ``pcg`` stops on its recursive residual; restarts
  begin from the true residual.
* ``si_lopcg``: the inexact shift-and-invert preconditioned LOPCG of Algorithm 1:
  outer residual r_o = A x_k - R(x_k) B x_k, inner solve A_sigma w_k = r_o by PCG
  (relative tolerance fixed, or min{0.1, ||r_o||_2} as in Sec. 4.3), or w_k = M^{-1} r_o
  with the Schwarz preconditioner alone (the fused variant of Sec. 4.3); orthogonalised
  Rayleigh-Ritz on span{w_k, x_k, x_{k-1}}; start x_0 = e_1, x_1 = 1/||1||_B (Sec. 4.2).
* ``cell_eigenpair``: lowest eigenpair of the x-periodic cell GEVP (weak cell
  problem, Sec. 2), by a dense generalised symmetric eigensolver; psi > 0,
  psi^T M_# psi = 1.
* ``exact_ground_state``: the plain definition of the result, the lowest
  eigenpair of (K + M_V) x = lambda M x, by a dense solver on tiny grids and by
  inverse iteration with an exact banded Cholesky of A_sigma otherwise.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import q1
from .dd import Decomposition, TwoLevelAS, _band_lower


def dot(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.dot(a, b))


def pcg(A, b, x0=None, prec=None, rtol=1e-8, maxit=10000, history=False):
    """Preconditioned CG.  Returns (x, iterations, list of ||r_k||/||r_0||)."""
    x = np.zeros_like(b) if x0 is None else x0.astype(float).copy()
    r = b - A @ x
    r0 = np.sqrt(dot(r, r))
    hist = [1.0]
    if r0 == 0.0:
        return x, 0, hist
    z = prec(r) if prec is not None else r.copy()
    p = z.copy()
    rho = dot(r, z)
    for k in range(1, maxit + 1):
        q = A @ p
        pq = dot(p, q)
        if not pq > 0.0:
            raise FloatingPointError("p^T A p <= 0: operator or preconditioner not SPD")
        alpha = rho / pq
        x += alpha * p
        r -= alpha * q
        rn = np.sqrt(dot(r, r))
        if history:
            hist.append(rn / r0)
        if rn <= rtol * r0:
            return x, k, hist
        z = prec(r) if prec is not None else r.copy()
        rho_new = dot(r, z)
        beta = rho_new / rho
        p = z + beta * p
        rho = rho_new
    return x, maxit, hist


def gmres(A, b, x0=None, prec=None, rtol=1e-8, restart=30, maxit=10000):
    """Right-preconditioned restarted GMRES: x = x0 + M^{-1} V y minimising ||b - A x||_2 over
    the Krylov space of A M^{-1}.  Returns (x, iterations, list of ||r_k||/||r_0||)."""
    n = b.size
    x = np.zeros(n) if x0 is None else x0.astype(float).copy()
    P = (lambda v: v) if prec is None else prec
    r = b - A @ x
    r0 = np.sqrt(dot(r, r))
    hist = [1.0]
    if r0 == 0.0:
        return x, 0, hist
    its = 0
    while its < maxit:
        beta = np.sqrt(dot(r, r))
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j_done = 0
        for j in range(restart):
            z = P(V[j])
            Z.append(z)
            w = A @ z
            for i in range(j + 1):                 # modified Gram-Schmidt
                H[i, j] = dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.sqrt(dot(w, w))
            V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
            for i in range(j):                     # earlier rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / r0)
            if abs(g[j + 1]) <= rtol * r0 or its >= maxit:
                break
        y = sla.solve_triangular(H[:j_done, :j_done], g[:j_done])
        for i in range(j_done):
            x = x + y[i] * Z[i]
        # stop on the method's own residual |g_{j+1}| (the minimised least-squares residual),
        # as PCG stops on its recursive residual; the cycle restarts from the true residual
        if abs(g[j_done]) <= rtol * r0:
            return x, its, hist
        r = b - A @ x
    return x, its, hist


def _inner_solve(Asig, b, prec, rtol, maxit, krylov, restart):
    if krylov == "gmres":
        return gmres(Asig, b, None, prec, rtol, restart, maxit)
    return pcg(Asig, b, None, prec, rtol, maxit)


def inverse_iteration(Asig, M, sigma, prec=None, x0=None, tol_res=1e-8, tol_lam=1e-10,
                      maxit_outer=100, rtol_inner=1e-8, maxit_inner=10000, krylov="cg", restart=30):
    """Shifted inverse iteration with inexact inner solves (Sec. 2): PCG (krylov="cg", with
    M_AS2^{-1}) or right-preconditioned GMRES (krylov="gmres", with M_RAS2^{-1})."""
    n = Asig.shape[0]
    x = np.ones(n) if x0 is None else x0.astype(float).copy()
    x /= np.sqrt(dot(x, M @ x))
    rho_prev = sigma + dot(x, Asig @ x)
    inner = []
    info = {}
    for k in range(1, maxit_outer + 1):
        b = M @ x
        w, it, _ = _inner_solve(Asig, b, prec, rtol_inner, maxit_inner, krylov, restart)
        inner.append(it)
        x = w / np.sqrt(dot(w, M @ w))
        if x.sum() < 0:
            x = -x
        Mx = M @ x
        lam_shift = dot(x, Asig @ x)          # x^T A_sigma x = rho - sigma
        rho = sigma + lam_shift
        res = Asig @ x - lam_shift * Mx       # = A x - rho M x
        eta = np.sqrt(dot(res, res)) / (abs(rho) * np.sqrt(dot(Mx, Mx)))
        info = dict(eta=eta, drho=abs(rho - rho_prev))
        if eta <= tol_res and abs(rho - rho_prev) <= tol_lam * abs(rho):
            return rho, x, k, inner, info
        rho_prev = rho
    return rho, x, maxit_outer, inner, info


def rayleigh_ritz3(GA, GB, sums, drop=1e-10):
    """Orthogonalised Rayleigh-Ritz (Algorithm 1) on span{s_0, s_1, s_2} from the Gram
    matrices GA = S^T A_sigma S and GB = S^T B S, S = [x_k, w_k, x_{k-1}].

    The basis is B-orthonormalised by Gram-Schmidt (two passes) in the order x_k, w_k,
    x_{k-1}, on coefficient vectors; a direction whose B-norm after orthogonalisation is
    at most ``drop`` times its norm before is dropped.  Returns (theta, c): the lowest
    eigenvalue of the projected pencil (shifted: theta = R(y) - sigma) and the
    coefficients c of its B-normalised Ritz vector y = S c, signed so that sum(y) > 0
    (``sums`` = [sum s_0, sum s_1, sum s_2]).
    """
    GA = np.asarray(GA, dtype=float)
    GB = np.asarray(GB, dtype=float)
    cols = []
    for i in range(3):
        v = np.zeros(3)
        v[i] = 1.0
        n0 = GB[i, i]
        for _ in range(2):
            for t in cols:
                v = v - (t @ GB @ v) * t
        nrm2 = v @ GB @ v
        if n0 > 0.0 and nrm2 > (drop * drop) * n0:
            cols.append(v / np.sqrt(nrm2))
    T = np.column_stack(cols)
    H = T.T @ GA @ T
    H = 0.5 * (H + H.T)
    w, V = np.linalg.eigh(H)
    c = T @ V[:, 0]
    if np.dot(np.asarray(sums, dtype=float), c) < 0.0:
        c = -c
    return float(w[0]), c


def si_lopcg(A, M, sigma, prec=None, x0=None, x1=None, tol_res=1e-8, tol_lam=1e-10,
             maxit_outer=1000, inner="fixed", rtol_inner=1e-8, maxit_inner=10000, krylov="cg", restart=30):
    """Inexact SI-preconditioned LOPCG (Algorithm 1).

    inner = "fixed": PCG on A_sigma w = r_o to relative residual rtol_inner;
    "adaptive": to min{0.1, ||r_o||_2} (Sec. 4.3); "fused": w = M^{-1} r_o, one
    application of the Schwarz preconditioner and no inner Krylov loop (Sec. 4.3).
    Stops like ``inverse_iteration``: eta <= tol_res and |rho_k - rho_{k-1}| <= tol_lam |rho_k|.
    Returns (rho, x, outer steps, inner iterations per step, info).
    """
    n = A.shape[0]
    Asig = (A - sigma * M).tocsr()
    if x0 is None:
        x0 = np.zeros(n)
        x0[0] = 1.0
    xp = x0 / np.sqrt(dot(x0, M @ x0))
    x = np.ones(n) if x1 is None else x1.astype(float).copy()
    x /= np.sqrt(dot(x, M @ x))
    Ax, Mx = Asig @ x, M @ x
    lam = dot(x, Ax)                         # rho - sigma, x^T B x = 1
    rho_prev = np.inf
    inner_its = []
    info = {}
    for k in range(0, maxit_outer + 1):
        rho = sigma + lam
        ro = Ax - lam * Mx                   # = A x - rho B x
        nro = np.sqrt(dot(ro, ro))
        eta = nro / (abs(rho) * np.sqrt(dot(Mx, Mx)))
        info = dict(eta=eta, drho=abs(rho - rho_prev))
        if eta <= tol_res and abs(rho - rho_prev) <= tol_lam * abs(rho):
            return rho, x, k, inner_its, info
        if k == maxit_outer:
            break
        if inner == "fused":
            w, it = prec(ro), 1
        else:
            rt = rtol_inner if inner == "fixed" else min(0.1, nro)
            w, it, _ = _inner_solve(Asig, ro, prec, rt, maxit_inner, krylov, restart)
        inner_its.append(it)
        S = [x, w, xp]
        AS = [Ax, Asig @ w, Asig @ xp]
        MS = [Mx, M @ w, M @ xp]
        GA = np.array([[dot(S[i], AS[j]) for j in range(3)] for i in range(3)])
        GB = np.array([[dot(S[i], MS[j]) for j in range(3)] for i in range(3)])
        GA = 0.5 * (GA + GA.T)
        GB = 0.5 * (GB + GB.T)
        _, c = rayleigh_ritz3(GA, GB, [v.sum() for v in S])
        xn = c[0] * x + c[1] * w + c[2] * xp
        xp = x
        x = xn / np.sqrt(dot(xn, M @ xn))
        Ax, Mx = Asig @ x, M @ x
        rho_prev = rho
        lam = dot(x, Ax)
    return sigma + lam, x, maxit_outer, inner_its, info


def cell_eigenpair(g: q1.Grid, V):
    """(sigma, psi) of the x-periodic cell problem; psi > 0, psi^T M_# psi = 1."""
    K, M, MV = q1.assemble_cell(g, V)
    A = (K + MV).toarray()
    B = M.toarray()
    w, v = sla.eigh(A, B, subset_by_index=[0, 0])
    psi = v[:, 0]
    if psi.sum() < 0:
        psi = -psi
    psi /= np.sqrt(psi @ (B @ psi))
    return float(w[0]), psi


def exact_ground_state(A, M, sigma=None, dense_limit=2500, band=True, tol=1e-15, maxit=400):
    """Lowest eigenpair (lambda_1, x) of A x = lambda M x, x^T M x = 1, sum x > 0.

    Dense generalised eigh up to ``dense_limit`` unknowns; beyond it, inverse
    iteration x <- (A - sigma M)^{-1} M x with an exact banded Cholesky factor
    (sigma below lambda_1, e.g. the cell shift), until the Rayleigh quotient
    is stationary to ``tol``.
    """
    n = A.shape[0]
    if n <= dense_limit:
        w, v = sla.eigh(A.toarray(), M.toarray(), subset_by_index=[0, 0])
        x = v[:, 0]
        if x.sum() < 0:
            x = -x
        return float(w[0]), x / np.sqrt(x @ (M @ x))
    assert sigma is not None
    As = (A - sigma * M).tocsr()
    cb = sla.cholesky_banded(_band_lower(As), lower=True)
    x = np.ones(n)
    x /= np.sqrt(dot(x, M @ x))
    rho_prev = np.inf
    stable = 0
    for _ in range(maxit):
        w = sla.cho_solve_banded((cb, True), M @ x)
        x = w / np.sqrt(dot(w, M @ w))
        rho = sigma + dot(x, As @ x)
        if abs(rho - rho_prev) <= tol * abs(rho):
            stable += 1
            if stable >= 3:
                break
        else:
            stable = 0
        rho_prev = rho
    if x.sum() < 0:
        x = -x
    return rho, x


class Problem:
    """Everything the method builds for one workload, in oracle form."""

    def __init__(self, g: q1.Grid, V, pu: str = "equal", coarse: bool = True, build_prec=True,
                 restricted: bool = False):
        self.g = g
        self.V = V
        self.K, self.M, self.MV = q1.assemble_box(g, V)
        self.A = (self.K + self.MV).tocsr()
        self.sigma, self.psi_cell = cell_eigenpair(g, V)
        self.psi = q1.periodic_extension(g, self.psi_cell)
        self.Asig = (self.A - self.sigma * self.M).tocsr()
        self.dec = Decomposition(g, pu)
        self.prec = TwoLevelAS(self.Asig, self.dec, self.psi, coarse=coarse,
                               restricted=restricted) if build_prec else None

    def solve(self, b, rtol=1e-8, maxit=10000, x0=None, history=False):
        return pcg(self.Asig, b, x0, self.prec, rtol, maxit, history)

    def solve_gmres(self, b, rtol=1e-8, restart=30, maxit=10000, x0=None):
        return gmres(self.Asig, b, x0, self.prec, rtol, restart, maxit)

    def ground_state(self, **kw):
        return inverse_iteration(self.Asig, self.M, self.sigma, self.prec, **kw)

    def ground_state_lopcg(self, **kw):
        return si_lopcg(self.A, self.M, self.sigma, self.prec, **kw)
