"""Overlapping decomposition, partition of unity, PerFact coarse space and
the two-level additive Schwarz preconditioner (oracle).

Sec. 3.1: the non-overlapping subdomains are the L^p unit cells
Omega_i' = prod_k (i_k - 1, i_k) x (0, ell); Omega_i adds delta element layers
on each x side (clipped at the box).  N_i is the set of interior DOFs strictly
inside the open Omega_i (homogeneous Dirichlet local problems, V_{h,0}(Omega_i)).
R_i restricts to N_i; D_i is a diagonal partition of unity with
sum_i R_i^T D_i R_i = I (Sec. 2.2).

Equal weights (Sec. 2.2): (D_i)_kk = 1 / |M_k|, M_k = {i : k in N_i}.
Distance weights (Sec. 4.1.2): chi_i = I_h(d_i / sum_j d_j) with
d_i(z) = dist(z, dOmega_i minus dOmega) 1_{Omega_i}(z).

Coarse space (Definition 2.1): R_0^T = blockdiag(D_i R_i psi), one column per
subdomain, boundary subdomains included; A_0 = R_0 A_sigma R_0^T.

Preconditioner (two-level additive Schwarz, Sec. 3.1):
  M_AS2^{-1} = R_0^T A_0^{-1} R_0 + sum_i R_i^T A_i^{-1} R_i,
  A_i = R_i A_sigma R_i^T.
With coarse=False this is the one-level M_AS1^{-1} (Sec. 2.2).

Subdomain labels: multi-index (i_1, .., i_p), 0-based, linear index with i_1
slowest (a labelling only; the paper's map n(i) orders them differently).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .q1 import Grid


def axis_ranges(g: Grid):
    """Interior node range [lo, hi] (1-based node index along an x axis) of
    every subdomain: nodes a with (i-1)n - delta < a < i n + delta, clipped to
    1..Ln-1 (i 1-based)."""
    n, L, dl = g.n, g.L, g.delta
    out = []
    for i in range(1, L + 1):
        lo = max(1, (i - 1) * n - dl + 1)
        hi = min(L * n - 1, i * n + dl - 1)
        out.append((lo, hi))
    return out


def axis_multiplicity(g: Grid) -> np.ndarray:
    """|M_k| along one x axis: number of subdomain ranges holding node a, a=1..Ln-1."""
    cnt = np.zeros(g.L * g.n + 1, dtype=np.int64)
    for lo, hi in axis_ranges(g):
        cnt[lo:hi + 1] += 1
    return cnt[1:g.L * g.n]


def axis_distance_weights(g: Grid) -> np.ndarray:
    """Distance partition of unity along one x axis, as a table W[i, a-1]
    for subdomain i (0-based) and node a.  For p=1 this is chi_i itself."""
    n, L, dl, h = g.n, g.L, g.delta, g.h
    a = np.arange(1, L * n)
    x = a * h
    D = np.zeros((L, L * n - 1))
    for i in range(L):
        X_lo = max(0.0, i - dl * h)
        X_hi = min(float(L), i + 1 + dl * h)
        inside = (x > X_lo + 1e-14) & (x < X_hi - 1e-14)
        dist = np.full_like(x, np.inf)
        if X_lo > 0.0:
            dist = np.minimum(dist, x - X_lo)
        if X_hi < L:
            dist = np.minimum(dist, X_hi - x)
        D[i] = np.where(inside, dist, 0.0)
    return D


class Decomposition:
    """Subdomain DOF sets N_i, partition of unity D_i, in D1 order."""

    def __init__(self, g: Grid, pu: str = "equal"):
        self.g = g
        self.pu = pu
        self.ranges = axis_ranges(g)
        self.N = g.L ** g.p
        nx, nyi = g.nx, g.ny - 1
        self.idx = []
        for lin in range(self.N):
            mi = np.unravel_index(lin, (g.L,) * g.p)
            axes = [np.arange(self.ranges[k][0], self.ranges[k][1] + 1) - 1 for k in mi]
            if g.p == 1:
                ids = (axes[0][:, None] * nyi + np.arange(nyi)[None, :]).reshape(-1)
            else:
                ids = ((axes[0][:, None, None] * nx + axes[1][None, :, None]) * nyi
                       + np.arange(nyi)[None, None, :]).reshape(-1)
            self.idx.append(ids)
        self.weights = self._pu_weights()

    def multiplicity(self) -> np.ndarray:
        m = np.zeros(self.g.ndof, dtype=np.int64)
        for ids in self.idx:
            m[ids] += 1
        return m

    def _pu_weights(self):
        g = self.g
        if self.pu == "equal":
            m = self.multiplicity()
            return [1.0 / m[ids] for ids in self.idx]
        if self.pu != "distance":
            raise ValueError(self.pu)
        if self.N == 1:
            return [np.ones(len(self.idx[0]))]
        nx, nyi = g.nx, g.ny - 1
        if g.p == 1:
            Dax = axis_distance_weights(g)
            tot = Dax.sum(axis=0)
            out = []
            for i, ids in enumerate(self.idx):
                a = ids // nyi
                out.append(Dax[i, a] / tot[a])
            return out
        # p = 2: d_i = min over the artificial faces of the box of the
        # perpendicular distance (the projection of an inside point lands on
        # the face), zero outside.
        h, n, L, dl = g.h, g.n, g.L, g.delta
        coords = np.arange(1, L * n) * h
        lo = [max(0.0, i - dl * h) for i in range(L)]
        hi = [min(float(L), i + 1 + dl * h) for i in range(L)]
        X1, X2 = np.meshgrid(coords, coords, indexing="ij")
        dist = np.zeros((self.N, nx, nx))
        for lin in range(self.N):
            i1, i2 = np.unravel_index(lin, (L, L))
            inside = ((X1 > lo[i1] + 1e-14) & (X1 < hi[i1] - 1e-14)
                      & (X2 > lo[i2] + 1e-14) & (X2 < hi[i2] - 1e-14))
            dd = np.full_like(X1, np.inf)
            if lo[i1] > 0:
                dd = np.minimum(dd, X1 - lo[i1])
            if hi[i1] < L:
                dd = np.minimum(dd, hi[i1] - X1)
            if lo[i2] > 0:
                dd = np.minimum(dd, X2 - lo[i2])
            if hi[i2] < L:
                dd = np.minimum(dd, hi[i2] - X2)
            dist[lin] = np.where(inside, dd, 0.0)
        tot = dist.sum(axis=0)
        out = []
        for lin, ids in enumerate(self.idx):
            col = ids // nyi
            a1, a2 = col // nx, col % nx
            out.append(dist[lin, a1, a2] / tot[a1, a2])
        return out

    def coarse_basis(self, psi_ext: np.ndarray) -> sp.csc_matrix:
        """R_0^T = blockdiag(D_i R_i psi) as an n x N sparse matrix (Def. 2.1)."""
        rows, cols, vals = [], [], []
        for i, (ids, w) in enumerate(zip(self.idx, self.weights)):
            rows.append(ids)
            cols.append(np.full(len(ids), i))
            vals.append(w * psi_ext[ids])
        n = self.g.ndof
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(n, self.N)).tocsc()


def _band_lower(A: sp.spmatrix):
    """Lower band storage ab[k, j] = A[j + k, j] (LAPACK 'L' layout)."""
    C = A.tocoo()
    m = C.row >= C.col
    r, c, v = C.row[m], C.col[m], C.data[m]
    bw = int((r - c).max()) if len(r) else 0
    ab = np.zeros((bw + 1, A.shape[0]))
    ab[r - c, c] = v
    return ab


class TwoLevelAS:
    """z = M_AS2^{-1} r (or M_AS1^{-1} r with coarse=False), Sec. 3.1; with restricted=True
    the restricted variant M_RAS2^{-1} (M_RAS1^{-1}): the local solutions are weighted by the
    partition of unity before the extension, sum_i R_i^T D_i A_i^{-1} R_i r (eq. of the
    one-level preconditioners), the coarse correction added the same way.

    Every subdomain gets its own local matrix and its own banded Cholesky
    factor (no sharing between equal subdomains); A_0 is factorised densely.
    """

    def __init__(self, Asig: sp.csr_matrix, dec: Decomposition, psi_ext: np.ndarray,
                 coarse: bool = True, restricted: bool = False):
        self.dec = dec
        self.coarse = coarse
        self.restricted = restricted
        self.local = []
        for ids in dec.idx:
            Ai = Asig[ids][:, ids]
            cb = sla.cholesky_banded(_band_lower(Ai), lower=True)
            self.local.append((ids, cb))
        if coarse:
            self.Z = dec.coarse_basis(psi_ext)
            A0 = (self.Z.T @ (Asig @ self.Z)).toarray()
            self.A0 = 0.5 * (A0 + A0.T)
            self.A0fac = sla.cho_factor(self.A0, lower=True)

    def local_part(self, r: np.ndarray) -> np.ndarray:
        z = np.zeros_like(r)
        for i, (ids, cb) in enumerate(self.local):
            yi = sla.cho_solve_banded((cb, True), r[ids])
            if self.restricted:
                yi = self.dec.weights[i] * yi
            z[ids] += yi
        return z

    def coarse_part(self, r: np.ndarray) -> np.ndarray:
        c = self.Z.T @ r
        u0 = sla.cho_solve(self.A0fac, c)
        return self.Z @ u0

    def __call__(self, r: np.ndarray) -> np.ndarray:
        z = self.local_part(r)
        if self.coarse:
            z += self.coarse_part(r)
        return z
