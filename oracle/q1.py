"""Q1 finite-element assembly (oracle).

Follows Sec. 2 of the paper: the Galerkin discretisation of
  int grad(phi).grad(v) + int V phi v = lambda int phi v
on a mesh made of translated copies of the unit-cell mesh gives the GEVP
A x = lambda B x with A = K + M_V (stiffness plus potential mass) and B = M
(mass).  Here the cell mesh is the uniform Cartesian grid with h = 1/n and
the space is Q1 (tensor bilinear / trilinear), Dirichlet on the whole
boundary of the box (H^1_0).  The cell problem (weak cell problem, Sec. 2)
replaces the x-Dirichlet condition by x-periodicity on (0,1)^p x (0,ell).

Degree-of-freedom order ("D1"): interior nodes only, y fastest, then x_p,
..., x_1 slowest.  For p=1, node (a, j) with 1<=a<=Ln-1, 1<=j<=ny-1 is DOF
(a-1)(ny-1) + (j-1).  Cell DOFs: node (a, j), 0<=a<n, 1<=j<=ny-1 is
a(ny-1) + (j-1) (and ((a1 n + a2)(ny-1) + j-1) for p=2).

Quadrature for int V phi v: tensor Gauss-Legendre with Q points per
direction (the paper does not state its rule), V evaluated at the global
coordinates of the points.
"""
from __future__ import annotations

from dataclasses import dataclass
import itertools

import numpy as np
import scipy.sparse as sp


@dataclass(frozen=True)
class Grid:
    p: int          # expanding directions (1 or 2)
    L: int          # domain length in cells
    n: int          # elements per unit length, h = 1/n
    ny: int         # elements across the fixed direction, ell = ny h
    delta: int = 1  # overlap in element layers
    Q: int = 2      # Gauss points per direction

    @property
    def h(self) -> float:
        return 1.0 / self.n

    @property
    def d(self) -> int:
        return self.p + 1

    @property
    def nx(self) -> int:          # interior nodes per expanding axis
        return self.L * self.n - 1

    @property
    def ndof(self) -> int:
        return self.nx ** self.p * (self.ny - 1)

    @property
    def ncell(self) -> int:       # cell DOFs
        return self.n ** self.p * (self.ny - 1)

    @staticmethod
    def from_workload(w) -> "Grid":
        return Grid(p=w.p, L=w.L, n=w.n, ny=w.ny, delta=w.overlap, Q=w.quad_pts)


def gauss01(Q: int):
    t, wt = np.polynomial.legendre.leggauss(Q)
    return 0.5 * (t + 1.0), 0.5 * wt


def element_matrices(d: int, h: float):
    """Exact Q1 element stiffness and mass on a cube of side h.

    1D: K1 = (1/h)[[1,-1],[-1,1]], M1 = (h/6)[[2,1],[1,2]].  In d dimensions
    K^e = sum_k M1 x .. x K1 (k-th slot) x .. x M1, M^e = M1 x .. x M1
    (Kronecker products; local node (b_1, .., b_d) has index with b_d
    fastest, the last axis being y).
    """
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    M1 = np.array([[2.0, 1.0], [1.0, 2.0]]) * h / 6.0
    Me = M1
    for _ in range(d - 1):
        Me = np.kron(Me, M1)
    Ke = np.zeros((2 ** d, 2 ** d))
    for k in range(d):
        t = np.ones((1, 1))
        for ax in range(d):
            t = np.kron(t, K1 if ax == k else M1)
        Ke += t
    return Ke, Me


def basis_at_points(d: int, Q: int):
    """Values N_b(xi_q) of the 2^d reference Q1 basis at the Q^d Gauss points,
    and the tensor weights W_q (reference cube [0,1]^d)."""
    xi, w = gauss01(Q)
    N1 = np.stack([1.0 - xi, xi], axis=1)            # [Q, 2]
    pts = list(itertools.product(range(Q), repeat=d))
    locs = list(itertools.product(range(2), repeat=d))
    B = np.empty((len(pts), len(locs)))
    W = np.empty(len(pts))
    for iq, q in enumerate(pts):
        W[iq] = np.prod([w[qq] for qq in q])
        for ib, b in enumerate(locs):
            B[iq, ib] = np.prod([N1[q[ax], b[ax]] for ax in range(d)])
    return xi, pts, locs, B, W


def _assemble(g: Grid, V, periodic: bool, chunk: int = 1 << 16):
    """Assemble K, M, M_V over interior DOFs.  periodic=False: the box
    (0,L)^p x (0,ell) with Dirichlet nodes removed; periodic=True: the unit
    cell with x-periodic identification and y-Dirichlet."""
    d, h, n, ny, Q = g.d, g.h, g.n, g.ny, g.Q
    Ke, Me = element_matrices(d, h)
    xi, pts, locs, B, W = basis_at_points(d, Q)
    nex = n if periodic else g.L * n            # elements per x axis
    nodes_x = n if periodic else g.L * n + 1    # node positions per x axis

    # all elements as (ex_1..ex_p, ey), y fastest
    shape = (nex,) * g.p + (ny,)
    nelem = int(np.prod(shape))
    rows, cols, vK, vM, vV = [], [], [], [], []
    for start in range(0, nelem, chunk):
        eid = np.arange(start, min(nelem, start + chunk))
        idx = np.unravel_index(eid, shape)
        ex = idx[:-1]
        ey = idx[-1]
        # global DOF ids of the 2^d local nodes (-1 for Dirichlet nodes)
        gid = np.empty((len(eid), len(locs)), dtype=np.int64)
        for ib, b in enumerate(locs):
            j = ey + b[-1]
            ok = (j >= 1) & (j <= ny - 1)
            lin = np.zeros(len(eid), dtype=np.int64)
            for ax in range(g.p):
                a = ex[ax] + b[ax]
                if periodic:
                    a = a % n
                    lin = lin * n + a
                else:
                    ok &= (a >= 1) & (a <= nodes_x - 2)
                    lin = lin * g.nx + (a - 1)
            lin = lin * (ny - 1) + (j - 1)
            gid[:, ib] = np.where(ok, lin, -1)
        # V at the global coordinates of the quadrature points
        Vq = np.empty((len(eid), len(pts)))
        for iq, q in enumerate(pts):
            coords = [(ex[ax] + xi[q[ax]]) * h for ax in range(g.p)]
            coords.append((ey + xi[q[-1]]) * h)
            Vq[:, iq] = V(*coords)
        # M_V^e[a,b] = h^d sum_q W_q V_q N_a(q) N_b(q)
        MVe = np.einsum("eq,qa,qb->eab", Vq * W[None, :], B, B) * h ** d
        for ia in range(len(locs)):
            for ib in range(len(locs)):
                m = (gid[:, ia] >= 0) & (gid[:, ib] >= 0)
                rows.append(gid[m, ia])
                cols.append(gid[m, ib])
                cnt = int(m.sum())
                vK.append(np.full(cnt, Ke[ia, ib]))
                vM.append(np.full(cnt, Me[ia, ib]))
                vV.append(MVe[m, ia, ib])
    N = g.ncell if periodic else g.ndof
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    K = sp.coo_matrix((np.concatenate(vK), (r, c)), shape=(N, N)).tocsr()
    M = sp.coo_matrix((np.concatenate(vM), (r, c)), shape=(N, N)).tocsr()
    MV = sp.coo_matrix((np.concatenate(vV), (r, c)), shape=(N, N)).tocsr()
    for X in (K, M, MV):
        X.sum_duplicates()
        X.sort_indices()
    return K, M, MV


def assemble_box(g: Grid, V):
    """K, M, M_V of the Dirichlet box problem (discrete weak form, Sec. 2)."""
    return _assemble(g, V, periodic=False)


def assemble_cell(g: Grid, V):
    """K_#, M_#, M_V# of the x-periodic cell problem (weak cell problem, Sec. 2)."""
    return _assemble(g, V, periodic=True)


def periodic_extension(g: Grid, psi_cell: np.ndarray) -> np.ndarray:
    """E_x^# psi restricted to the interior box nodes (Sec. 3.1):
    node (a, j) takes the cell value at (a mod n, j)."""
    n, ny = g.n, g.ny
    a = np.arange(1, g.L * n) % n
    if g.p == 1:
        cell = psi_cell.reshape(n, ny - 1)
        return cell[a, :].reshape(-1).copy()
    cell = psi_cell.reshape(n, n, ny - 1)
    return cell[a[:, None], a[None, :], :].reshape(-1).copy()


def dof_coords(g: Grid):
    """Coordinates of the interior DOFs in D1 order: list of p+1 arrays."""
    h = g.h
    ax = [np.arange(1, g.L * g.n) * h] * g.p + [np.arange(1, g.ny) * h]
    mesh = np.meshgrid(*ax, indexing="ij")
    return [m.reshape(-1) for m in mesh]
