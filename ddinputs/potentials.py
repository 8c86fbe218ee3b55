"""Workload descriptions and potentials (inputs only, no solver arithmetic)."""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One synthetic eigenproblem: geometry (0,L)^p x (0,ell), mesh h = 1/n.

    ``kind`` selects the potential family (see :func:`potential`);
    ``seed`` feeds the random coefficients where the family has any.
    """
    name: str
    p: int
    L: int
    n: int
    ell: float = 1.0
    overlap: int = 1
    quad_pts: int = 2
    kind: str = "zero"
    seed: int = 0
    params: dict = field(default_factory=dict, compare=False, hash=False)

    @property
    def ny(self) -> int:
        v = self.ell * self.n
        iv = int(round(v))
        if abs(v - iv) > 1e-9:
            raise ValueError("ell * n must be an integer")
        return iv

    @property
    def dofs(self) -> int:
        return (self.L * self.n - 1) ** self.p * (self.ny - 1)

    def with_(self, **kw) -> "Workload":
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)


def _cos_series_coeffs(seed: int, terms: int = 4):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 20.0, terms)
    b = rng.uniform(-0.5, 0.5, terms)
    return a, b


def potential(w: Workload):
    """Return V as a vectorised callable V(x, y) (p=1) or V(x1, x2, y) (p=2).

    Families:
      zero      V = 0                       (closed-form Q1 spectrum)
      const     V = c                       (pure spectral shift)
      cos1      V = 10 (1 + cos 2 pi x)(1 + 0.5 sin pi y)
      cos4      V = sum_j a_j cos(2 pi j x)(1 + b_j y), a_j ~ U(0,20),
                b_j ~ U(-1/2, 1/2) drawn from default_rng(seed) (a first, then b)
      sin4      V = 100 sin^4(pi x) sin^4(pi y)  (the formula printed in Sec. 4.1)
      wells     V = -30 (1 + y) sum_c exp(-|x - c|^2 / (2 * 0.15^2)),
                c over the lattice (Z + 1/2)^2 within max-norm distance 3
      asym3     V = 10 (4 + sin 2pi x1 + sin 4pi x1 + 2 sin 2pi x2 + 2 sin 4pi x2 + y)
                (the unsymmetric potential of Sec. 4.3)
      theta8    V = sum_{j=1..8} theta_j cos(2 pi j x)(1 + 0.3 y), theta from
                w.params["theta"], else theta_seed(w.seed) (the differentiable workload)
    """
    k = w.kind
    if k == "zero":
        return (lambda x, y: np.zeros_like(np.asarray(x, dtype=float))) if w.p == 1 else \
               (lambda x1, x2, y: np.zeros_like(np.asarray(x1, dtype=float)))
    if k == "const":
        c = float(w.params.get("c", 3.0))
        return (lambda x, y: np.full_like(np.asarray(x, dtype=float), c)) if w.p == 1 else \
               (lambda x1, x2, y: np.full_like(np.asarray(x1, dtype=float), c))
    if k == "cos1":
        assert w.p == 1
        return lambda x, y: 10.0 * (1.0 + np.cos(2 * np.pi * x)) * (1.0 + 0.5 * np.sin(np.pi * y))
    if k == "cos4":
        if "a" in w.params:
            a, b = np.asarray(w.params["a"], dtype=float), np.asarray(w.params["b"], dtype=float)
        else:
            a, b = _cos_series_coeffs(w.seed)
        if w.p == 1:
            def V(x, y):
                x = np.asarray(x, dtype=float)
                out = np.zeros_like(x)
                for j in range(4):
                    out += a[j] * np.cos(2 * np.pi * (j + 1) * x) * (1.0 + b[j] * y)
                return out
            return V

        def V3(x1, x2, y):
            x1 = np.asarray(x1, dtype=float)
            out = np.zeros_like(x1)
            for j in range(4):
                out += a[j] * np.cos(2 * np.pi * (j + 1) * x1) * np.cos(2 * np.pi * (j + 1) * x2) * (1.0 + b[j] * y)
            return out
        return V3
    if k == "sin4":
        assert w.p == 1
        return lambda x, y: 100.0 * np.sin(np.pi * x) ** 4 * np.sin(np.pi * y) ** 4
    if k == "wells":
        assert w.p == 2
        s2 = 2 * 0.15 ** 2

        def Vw(x1, x2, y):
            x1 = np.asarray(x1, dtype=float)
            x2 = np.asarray(x2, dtype=float)
            f1 = x1 - np.floor(x1)
            f2 = x2 - np.floor(x2)
            acc = np.zeros_like(x1)
            for c1 in range(-3, 4):
                for c2 in range(-3, 4):
                    acc += np.exp(-((f1 - (c1 + 0.5)) ** 2 + (f2 - (c2 + 0.5)) ** 2) / s2)
            return -30.0 * (1.0 + y) * acc
        return Vw
    if k == "asym3":
        assert w.p == 2
        return lambda x1, x2, y: 10.0 * (4 + np.sin(2 * np.pi * x1) + np.sin(4 * np.pi * x1)
                                         + 2 * np.sin(2 * np.pi * x2) + 2 * np.sin(4 * np.pi * x2) + y)
    if k == "theta8":
        assert w.p == 1
        th = np.asarray(w.params.get("theta", theta_seed(w.seed)[0]), dtype=float)

        def Vt(x, y):
            x = np.asarray(x, dtype=float)
            out = np.zeros_like(x)
            for j in range(len(th)):
                out += th[j] * theta8_basis(j, x, y)
            return out
        return Vt
    raise ValueError(f"unknown potential kind {k!r}")


def batch_workloads(seed: int = 4242, count: int = 64, L_min: int = 16, L_max: int = 2048, n: int = 32,
                    overlap: int = 4):
    """The batched workload: ``count`` independent 2D instances (h = 1/n, ell = 1) with
    L_i = round(exp(U(ln L_min, ln L_max))) and each its own 4-term cosine potential
    (a ~ U(0, 20), b ~ U(-1/2, 1/2) as in cfg2), all drawn from default_rng(seed): the L_i
    first, then (a_i, b_i) instance by instance."""
    rng = np.random.default_rng(seed)
    Ls = np.rint(np.exp(rng.uniform(np.log(L_min), np.log(L_max), count))).astype(int)
    out = []
    for i, L in enumerate(Ls):
        a = rng.uniform(0.0, 20.0, 4)
        b = rng.uniform(-0.5, 0.5, 4)
        out.append(Workload(f"cfg4_{i}", p=1, L=int(L), n=n, overlap=overlap, kind="cos4",
                            params={"a": a.tolist(), "b": b.tolist()}))
    return out


def theta8_basis(j: int, x, y):
    """g_j(x, y) = cos(2 pi (j+1) x)(1 + 0.3 y), the j-th basis potential of theta8 (0-based)."""
    return np.cos(2 * np.pi * (j + 1) * np.asarray(x, dtype=float)) * (1.0 + 0.3 * np.asarray(y, dtype=float))


def theta_seed(seed: int, terms: int = 8):
    """(theta, theta_target) of the differentiable workload: theta ~ N(0, 25) and
    theta_target = theta + N(0, 1), drawn from default_rng(seed) in that order."""
    rng = np.random.default_rng(seed)
    th = rng.normal(0.0, 5.0, terms)
    tt = th + rng.normal(0.0, 1.0, terms)
    return th, tt


def theta8_qp_basis(w: Workload) -> np.ndarray:
    """[8, n_qp] values of the basis potentials g_j at the cell quadrature points, in the
    layout of sample_cell_qp (so that V_cell_qp = theta @ basis)."""
    return np.stack([sample_cell_qp(w, lambda x, y, j=j: theta8_basis(j, x, y)) for j in range(8)])


def gauss_legendre_01(Q: int):
    """Gauss-Legendre points and weights mapped to [0, 1] (numpy's leggauss)."""
    t, wt = np.polynomial.legendre.leggauss(Q)
    return 0.5 * (t + 1.0), 0.5 * wt


def sample_cell_qp(w: Workload, V=None) -> np.ndarray:
    """Sample V on the unit cell at tensor Gauss-Legendre points.

    Layout (the ``V_cell_qp`` input of ``dd_setup``): element-major, elements
    ordered (ex, ey) for p=1 / (ex1, ex2, ey) for p=2 with ey fastest; inside
    an element the Q^d points are ordered (qx, qy) / (qx1, qx2, qy), qy fastest.
    Element (ex, ey) covers [ex h, (ex+1) h] x [ey h, (ey+1) h].
    """
    if V is None:
        V = potential(w)
    n, ny, Q = w.n, w.ny, w.quad_pts
    h = 1.0 / n
    xi, _ = gauss_legendre_01(Q)
    if w.p == 1:
        ex, ey, qx, qy = np.meshgrid(np.arange(n), np.arange(ny), np.arange(Q), np.arange(Q), indexing="ij")
        x = (ex + xi[qx]) * h
        y = (ey + xi[qy]) * h
        return np.ascontiguousarray(V(x, y).reshape(-1), dtype=np.float64)
    e1, e2, ey, q1, q2, qy = np.meshgrid(np.arange(n), np.arange(n), np.arange(ny),
                                         np.arange(Q), np.arange(Q), np.arange(Q), indexing="ij")
    x1 = (e1 + xi[q1]) * h
    x2 = (e2 + xi[q2]) * h
    y = (ey + xi[qy]) * h
    return np.ascontiguousarray(V(x1, x2, y).reshape(-1), dtype=np.float64)


# The workloads.  "cfg1".."cfg3" are the three configurations the method is
# measured on; the small ones are parity cases that the oracle finishes quickly.
WORKLOADS = {
    "cfg1": Workload("cfg1", p=1, L=8, n=16, overlap=2, kind="cos1"),
    "cfg1_v0": Workload("cfg1_v0", p=1, L=8, n=16, overlap=2, kind="zero"),
    "cfg2": Workload("cfg2", p=1, L=2048, n=32, overlap=4, kind="cos4", seed=2311),
    "cfg2_small": Workload("cfg2_small", p=1, L=64, n=32, overlap=4, kind="cos4", seed=2311),
    "cfg3": Workload("cfg3", p=2, L=64, n=16, overlap=2, kind="wells"),
    "cfg3_small": Workload("cfg3_small", p=2, L=4, n=8, overlap=2, kind="wells"),
    # the d=3 well lattice at its full cell resolution and overlap on a 3 x 3 cell box: the
    # same nine local matrices and cell problem as the 64 x 64 box
    "cfg3_mid": Workload("cfg3_mid", p=2, L=3, n=16, overlap=2, kind="wells"),
    "e1": Workload("e1", p=1, L=8, n=30, overlap=1, kind="sin4"),
    # differentiable workload: theta ~ N(0, 25), 8 cosine modes times (1 + 0.3 y)
    "cfg5": Workload("cfg5", p=1, L=256, n=32, overlap=4, kind="theta8", seed=5),
    "cfg5_small": Workload("cfg5_small", p=1, L=8, n=16, overlap=2, kind="theta8", seed=5),
}
