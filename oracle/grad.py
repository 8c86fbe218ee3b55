"""Gradients of the ground state with respect to the potential (test infrastructure only:
imported by tests, the smoke check and the bench's CPU baseline, never by the CUDA path).

The potential enters the discrete problem only through M_V, assembled with tensor
Gauss-Legendre quadrature from the values V_q at the cell quadrature points (V is periodic,
so every copy of a cell element uses the same V_cell_qp[e, q]):

    M_V = sum over box elements of h^d sum_q W_q V_q N(z_q) N(z_q)^T.

* ``qp_product(g, u, v)``: P[e, q] = sum over the copies of cell element e of
  h^d W_q u_h(z_q) v_h(z_q) -- the derivative of u^T M_V v with respect to V_cell_qp[e, q].
* ``eigenvalue_gradient``: the Hellmann-Feynman identity for A phi = lambda M phi with
  phi^T M phi = 1: d lambda = phi^T dA phi, so d lambda / d V_cell_qp = qp_product(phi, phi).
* ``adjoint_solve`` / ``loss_gradient``: for a loss l(phi) with g = dl/dphi, differentiating
  the eigen-equation and the normalisation gives (A - lambda M) dphi = -(dA - dlambda M) phi
  with phi^T M dphi = 0.  With w the solution of (A - lambda M) w = g - M phi (phi^T g) in the
  M-orthogonal complement of phi (the projected singular system), dl = -w^T dA phi, so
  dl / d V_cell_qp = -qp_product(w, phi).  The oracle solves the singular system exactly
  through the bordered matrix [[A - lambda M, M phi], [phi^T M, 0]] (sparse LU) on small
  grids; on large ones (where the dense border makes sparse LU slow) by CG on the consistent
  singular system preconditioned with the exact banded Cholesky factor of A - sigma M (sigma
  below lambda), to a relative residual of 1e-14, followed by the projection
  w <- w - phi (phi^T M w).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import q1


def qp_product(g: q1.Grid, u: np.ndarray, v: np.ndarray, chunk: int = 1 << 16) -> np.ndarray:
    """[n_cell_elements * Q^d] array (the layout of V_cell_qp) of sum over the copies of each
    cell element of h^d W_q u_h(z_q) v_h(z_q); u, v interior-node vectors of the box."""
    d, h, n, ny, Q = g.d, g.h, g.n, g.ny, g.Q
    xi, pts, locs, B, W = q1.basis_at_points(d, Q)
    nex = g.L * n
    shape = (nex,) * g.p + (ny,)
    nelem = int(np.prod(shape))
    ncell_el = n ** g.p * ny
    out = np.zeros((ncell_el, len(pts)))
    for start in range(0, nelem, chunk):
        eid = np.arange(start, min(nelem, start + chunk))
        idx = np.unravel_index(eid, shape)
        ex, ey = idx[:-1], idx[-1]
        ul = np.zeros((len(eid), len(locs)))
        vl = np.zeros((len(eid), len(locs)))
        for ib, b in enumerate(locs):
            j = ey + b[-1]
            ok = (j >= 1) & (j <= ny - 1)
            lin = np.zeros(len(eid), dtype=np.int64)
            for ax in range(g.p):
                a = ex[ax] + b[ax]
                ok &= (a >= 1) & (a <= nex - 1)
                lin = lin * g.nx + (a - 1)
            lin = lin * (ny - 1) + (j - 1)
            ul[ok, ib] = u[lin[ok]]
            vl[ok, ib] = v[lin[ok]]
        uq = ul @ B.T                              # [elements, Q^d]
        vq = vl @ B.T
        contrib = uq * vq * W[None, :] * h ** d
        cell = np.zeros(len(eid), dtype=np.int64)
        for ax in range(g.p):
            cell = cell * n + (ex[ax] % n)
        cell = cell * ny + ey
        np.add.at(out, cell, contrib)
    return out.reshape(-1)


def eigenvalue_gradient(g: q1.Grid, phi: np.ndarray) -> np.ndarray:
    """d lambda / d V_cell_qp for the M-normalised ground state phi (Hellmann-Feynman)."""
    return qp_product(g, phi, phi)


def adjoint_solve(A, M, lam: float, phi: np.ndarray, gphi: np.ndarray, sigma=None,
                  direct_limit: int = 20000, rtol: float = 1e-14) -> np.ndarray:
    """w with (A - lam M) w = gphi - M phi (phi^T gphi) and phi^T M w = 0."""
    Mphi = M @ phi
    r = gphi - Mphi * float(phi @ gphi)
    n = A.shape[0]
    Al = (A - lam * M).tocsr()
    if n <= direct_limit:
        K = sp.bmat([[Al, sp.csr_matrix(Mphi[:, None])], [sp.csr_matrix(Mphi[None, :]), None]], format="csc")
        sol = spla.spsolve(K, np.concatenate([r, [0.0]]))
        return sol[:n]
    if sigma is None:
        raise ValueError("the iterative adjoint needs a shift sigma below lambda")
    from .dd import _band_lower
    import scipy.linalg as sla
    cb = sla.cholesky_banded(_band_lower((A - sigma * M).tocsr()), lower=True)
    w = np.zeros(n)
    res = r.copy()
    r0 = np.sqrt(res @ res)
    z = sla.cho_solve_banded((cb, True), res)
    p = z.copy()
    rz = res @ z
    for _ in range(1000):
        q = Al @ p
        alpha = rz / (p @ q)
        w += alpha * p
        res -= alpha * q
        if np.sqrt(res @ res) <= rtol * r0:
            break
        z = sla.cho_solve_banded((cb, True), res)
        rz_new = res @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return w - phi * float(phi @ (M @ w))


def loss_gradient(g: q1.Grid, A, M, lam: float, phi: np.ndarray, gphi: np.ndarray, sigma=None) -> np.ndarray:
    """dl / d V_cell_qp for a loss l(phi) with gradient gphi = dl/dphi."""
    w = adjoint_solve(A, M, lam, phi, gphi, sigma=sigma)
    return -qp_product(g, w, phi)
