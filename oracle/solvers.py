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


def inverse_iteration(Asig, M, sigma, prec=None, x0=None, tol_res=1e-8, tol_lam=1e-10,
                      maxit_outer=100, rtol_inner=1e-8, maxit_inner=10000):
    """Shifted inverse iteration with inexact PCG inner solves (Sec. 2)."""
    n = Asig.shape[0]
    x = np.ones(n) if x0 is None else x0.astype(float).copy()
    x /= np.sqrt(dot(x, M @ x))
    rho_prev = sigma + dot(x, Asig @ x)
    inner = []
    info = {}
    for k in range(1, maxit_outer + 1):
        b = M @ x
        w, it, _ = pcg(Asig, b, None, prec, rtol_inner, maxit_inner)
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

    def __init__(self, g: q1.Grid, V, pu: str = "equal", coarse: bool = True, build_prec=True):
        self.g = g
        self.V = V
        self.K, self.M, self.MV = q1.assemble_box(g, V)
        self.A = (self.K + self.MV).tocsr()
        self.sigma, self.psi_cell = cell_eigenpair(g, V)
        self.psi = q1.periodic_extension(g, self.psi_cell)
        self.Asig = (self.A - self.sigma * self.M).tocsr()
        self.dec = Decomposition(g, pu)
        self.prec = TwoLevelAS(self.Asig, self.dec, self.psi, coarse=coarse) if build_prec else None

    def solve(self, b, rtol=1e-8, maxit=10000, x0=None, history=False):
        return pcg(self.Asig, b, x0, self.prec, rtol, maxit, history)

    def ground_state(self, **kw):
        return inverse_iteration(self.Asig, self.M, self.sigma, self.prec, **kw)
