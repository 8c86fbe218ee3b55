"""Pins of the oracle against facts that do not come from the oracle itself.

Each test names the passage of the paper (or the piece of mathematics) it
checks.  A dropped term, a wrong sign or index, or a transposed operand in the
oracle's assembly, decomposition, preconditioner or solvers fails one of them.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from ddinputs import WORKLOADS, Workload, potential
from oracle import q1, solvers
from oracle.dd import Decomposition, TwoLevelAS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def mu(theta, h):
    """1D Q1 Dirichlet/periodic generalised eigenvalue for the discrete sine
    or Fourier mode of angle theta: (6/h^2)(1 - cos theta)/(2 + cos theta).
    (K1 = tridiag(-1,2,-1)/h, M1 = h tridiag(1,4,1)/6 act on sin(k a theta)
    by the factors 2(1-cos)/h and h(4+2cos)/6.)"""
    return 6.0 / h ** 2 * (1.0 - np.cos(theta)) / (2.0 + np.cos(theta))


def grid(p, L, n, ny, delta=1, Q=2):
    return q1.Grid(p=p, L=L, n=n, ny=ny, delta=delta, Q=Q)


def zeroV(p):
    return (lambda x, y: 0.0 * x) if p == 1 else (lambda x1, x2, y: 0.0 * x1)


# --- closed-form Q1 spectrum for V = 0 (motivation Sec. 1.2, Q1 analogue) ----

@pytest.mark.parametrize("p,L,n,ny", [(1, 3, 4, 5), (1, 5, 6, 4), (2, 2, 4, 4), (2, 3, 3, 3)])
def test_v0_box_spectrum_closed_form(p, L, n, ny):
    g = grid(p, L, n, ny)
    K, M, MV = q1.assemble_box(g, zeroV(p))
    w = sla.eigh(K.toarray(), M.toarray(), eigvals_only=True)
    h = g.h
    ks = [np.arange(1, L * n)] * p + [np.arange(1, ny)]
    lens = [L] * p + [ny * h]
    mesh = np.meshgrid(*[mu(k * np.pi * h / ln, h) for k, ln in zip(ks, lens)], indexing="ij")
    expect = np.sort(sum(mesh).reshape(-1))
    assert np.allclose(np.sort(w), expect, rtol=1e-11, atol=1e-9)
    assert np.abs(MV.toarray()).max() == 0.0


@pytest.mark.parametrize("p,n,ny", [(1, 8, 8), (1, 6, 12), (2, 4, 5)])
def test_v0_cell_shift_closed_form(p, n, ny):
    """Cell problem (Sec. 2): x-periodic modes have theta = 2 pi k h, so the
    lowest is k = 0 and sigma = mu(pi h / ell); psi = const in x times
    sin(pi y / ell)."""
    g = grid(p, 2, n, ny)
    sigma, psi = solvers.cell_eigenpair(g, zeroV(p))
    h = g.h
    ell = ny * h
    assert sigma == pytest.approx(mu(np.pi * h / ell, h), rel=1e-12)
    prof = np.sin(np.pi * np.arange(1, ny) * h / ell)
    cells = psi.reshape(-1, ny - 1)
    for row in cells:
        assert np.allclose(row / row.sum(), prof / prof.sum(), atol=1e-12)
    K, M, MV = q1.assemble_cell(g, zeroV(p))
    assert psi @ (M @ psi) == pytest.approx(1.0, rel=1e-13)
    assert (psi > 0).all()


def test_v0_ground_state_and_qosi_ratio():
    """lambda_1 and lambda_2 of the box for V=0 in closed form; the shifted
    ratio (lambda_1 - sigma)/(lambda_2 - sigma) tends to 1/4 (Sec. 1.2, QOSI
    shift) and the full eigensolver (inverse iteration + PCG + M_AS2) reaches
    lambda_1 to 1e-10."""
    L, n, ny = 16, 8, 8
    g = grid(1, L, n, ny, delta=2)
    P = solvers.Problem(g, zeroV(1))
    h = g.h
    lam1 = mu(np.pi * h / L, h) + mu(np.pi * h, h)
    lam2 = mu(2 * np.pi * h / L, h) + mu(np.pi * h, h)
    lam, x, k, inner, info = P.ground_state()
    assert lam == pytest.approx(lam1, rel=1e-10)
    ratio = (lam1 - P.sigma) / (lam2 - P.sigma)
    assert abs(ratio - 0.25) < 0.01
    le, xe = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma, dense_limit=0)
    assert le == pytest.approx(lam1, rel=1e-12)


def test_constant_potential_shift():
    """A constant V = c shifts every eigenvalue by c (Sec. 1, remark after A2)."""
    c = 3.25
    g = grid(1, 4, 6, 6, delta=2)
    s0, _ = solvers.cell_eigenpair(g, zeroV(1))
    sc, _ = solvers.cell_eigenpair(g, lambda x, y: c + 0.0 * x)
    assert sc - s0 == pytest.approx(c, rel=1e-12)
    K, M, MV = q1.assemble_box(g, lambda x, y: c + 0.0 * x)
    assert np.allclose(MV.toarray(), c * M.toarray(), rtol=1e-13, atol=1e-15)
    l0, _ = solvers.exact_ground_state(K, M)
    lc, _ = solvers.exact_ground_state(K + MV, M)
    assert lc - l0 == pytest.approx(c, rel=1e-11)


# --- assembly against Simpson-rule integrals of separable functions ----------

def _simpson_1d(vals_nodes, vfun, h, npts):
    """int v(x) (I_h f)^2 dx and int (I_h f)'^2 dx over [0, npts*h] for nodal
    values f (including the zero end nodes), by Simpson's rule per element
    (exact for the cubic integrand v * (linear)^2 with v linear)."""
    I2 = 0.0
    Id = 0.0
    for e in range(npts):
        x0, x1 = e * h, (e + 1) * h
        f0, f1 = vals_nodes[e], vals_nodes[e + 1]
        fm = 0.5 * (f0 + f1)
        xm = 0.5 * (x0 + x1)
        I2 += h / 6 * (vfun(x0) * f0 ** 2 + 4 * vfun(xm) * fm ** 2 + vfun(x1) * f1 ** 2)
        Id += (f1 - f0) ** 2 / h
    return I2, Id


@pytest.mark.parametrize("Q", [2, 3])
def test_assembly_separable_integrals(Q):
    L, n, ny = 3, 4, 5
    g = grid(1, L, n, ny, Q=Q)
    h = g.h
    v1 = lambda x: 1.5 + 0.7 * x
    v2 = lambda y: 2.0 - 0.4 * y
    V = lambda x, y: v1(x) * v2(y)
    K, M, MV = q1.assemble_box(g, V)
    rng = np.random.default_rng(7)
    f = np.concatenate([[0.0], rng.standard_normal(L * n - 1), [0.0]])
    gg = np.concatenate([[0.0], rng.standard_normal(ny - 1), [0.0]])
    u = (f[1:-1, None] * gg[None, 1:-1]).reshape(-1)
    Fv, Fd = _simpson_1d(f, v1, h, L * n)
    Gv, Gd = _simpson_1d(gg, v2, h, ny)
    F1, _ = _simpson_1d(f, lambda x: 1.0, h, L * n)
    G1, _ = _simpson_1d(gg, lambda y: 1.0, h, ny)
    assert u @ (MV @ u) == pytest.approx(Fv * Gv, rel=1e-12)
    assert u @ (M @ u) == pytest.approx(F1 * G1, rel=1e-12)
    assert u @ (K @ u) == pytest.approx(Fd * G1 + F1 * Gd, rel=1e-12)


def test_assembly_symmetric_and_3d_separable():
    g = grid(2, 2, 3, 4)
    V = lambda x1, x2, y: (1 + x1) * (2 - 0.5 * x2) * (1 + 0.25 * y)
    K, M, MV = q1.assemble_box(g, V)
    for X in (K, M, MV):
        assert abs(X - X.T).max() < 1e-15
    h = g.h
    rng = np.random.default_rng(3)
    fs = [np.concatenate([[0.0], rng.standard_normal(m - 1), [0.0]]) for m in (g.L * g.n, g.L * g.n, g.ny)]
    u = (fs[0][1:-1, None, None] * fs[1][None, 1:-1, None] * fs[2][None, None, 1:-1]).reshape(-1)
    vs = [lambda x: 1 + x, lambda x: 2 - 0.5 * x, lambda y: 1 + 0.25 * y]
    ones = lambda x: 1.0
    parts = [_simpson_1d(f, v, h, len(f) - 1) for f, v in zip(fs, vs)]
    plain = [_simpson_1d(f, ones, h, len(f) - 1) for f in fs]
    assert u @ (MV @ u) == pytest.approx(np.prod([a for a, _ in parts]), rel=1e-12)
    stiff = sum(plain[k][1] * np.prod([plain[j][0] for j in range(3) if j != k]) for k in range(3))
    assert u @ (K @ u) == pytest.approx(stiff, rel=1e-12)


# --- cell eigenpair and periodic extension (Sec. 2, factorisation Sec. 2.3) --

def test_cell_eigenpair_brute_force_and_translation_invariance():
    """psi solves the cell GEVP (brute-force residual) and its periodic
    extension is annihilated by A_sigma on every row whose stencil does not
    reach the x-boundary: those rows of the box operator are translated rows
    of the periodic cell operator."""
    w = Workload("t", p=1, L=4, n=8, overlap=2, kind="cos1")
    g = q1.Grid.from_workload(w)
    V = potential(w)
    sigma, psi = solvers.cell_eigenpair(g, V)
    Kc, Mc, MVc = q1.assemble_cell(g, V)
    r = (Kc + MVc) @ psi - sigma * (Mc @ psi)
    assert np.abs(r).max() < 1e-10 * sigma
    K, M, MV = q1.assemble_box(g, V)
    Asig = K + MV - sigma * M
    pe = q1.periodic_extension(g, psi)
    res = (Asig @ pe).reshape(g.nx, g.ny - 1)
    assert np.abs(res[1:-1]).max() < 1e-10 * np.abs(pe).max() * sigma
    assert np.abs(res[0]).max() > 1e-3  # boundary rows differ (Dirichlet)


def test_exact_ground_state_banded_vs_dense():
    w = Workload("t", p=1, L=6, n=6, overlap=2, kind="cos1")
    g = q1.Grid.from_workload(w)
    P = solvers.Problem(g, potential(w), build_prec=False)
    ld, xd = solvers.exact_ground_state(P.A, P.M)
    lb, xb = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma, dense_limit=0)
    assert lb == pytest.approx(ld, rel=1e-13)
    assert np.abs(xb - xd).max() < 1e-8


def test_factorisation_principle_gap():
    """lambda_L - sigma > 0 and (lambda_L - sigma) L^2 stays bounded
    (factorisation principle, lambda_u in O(1/L^2), Sec. 2.3)."""
    vals = []
    for L in (4, 8, 16):
        w = Workload("t", p=1, L=L, n=8, overlap=2, kind="cos1")
        g = q1.Grid.from_workload(w)
        P = solvers.Problem(g, potential(w), build_prec=False)
        lam, _ = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma, dense_limit=0)
        assert lam > P.sigma
        vals.append((lam - P.sigma) * L ** 2)
    assert max(vals) / min(vals) < 1.5


# --- decomposition, partition of unity, preconditioner (Sec. 2.2, 2.3, 3.1) --

@pytest.mark.parametrize("pu", ["equal", "distance"])
@pytest.mark.parametrize("p,L,n,delta", [(1, 5, 8, 2), (1, 3, 6, 1), (2, 3, 6, 2), (1, 1, 6, 2)])
def test_partition_of_unity(pu, p, L, n, delta):
    g = grid(p, L, n, 4, delta=delta)
    dec = Decomposition(g, pu)
    s = np.zeros(g.ndof)
    for ids, w in zip(dec.idx, dec.weights):
        assert (w >= 0).all() and (w <= 1 + 1e-15).all()
        s[ids] += w
    assert np.allclose(s, 1.0, atol=1e-14)
    # interior subdomain size (n + 2 delta - 1)^p (ny - 1) when L >= 3
    if L >= 3:
        mid = (L // 2) * (L ** (p - 1)) + (L // 2 if p == 2 else 0)
        assert len(dec.idx[mid]) == (n + 2 * delta - 1) ** p * (g.ny - 1)


def test_subdomains_are_open_overlapping_boxes():
    """N_i holds nodes strictly inside ((i-1) - delta h, i + delta h) (Sec. 3.1)."""
    g = grid(1, 4, 8, 4, delta=2)
    dec = Decomposition(g)
    nyi = g.ny - 1
    for i, ids in enumerate(dec.idx):
        a = np.unique(ids // nyi) + 1
        x = a * g.h
        lo, hi = i - 2 * g.h, i + 1 + 2 * g.h
        assert (x > lo).all() and (x < hi).all()
        allx = np.arange(1, g.L * g.n) * g.h
        assert len(a) == ((allx > lo + 1e-12) & (allx < hi - 1e-12)).sum()


def _weights_by_node(dec, nyi):
    """{subdomain: {node column: weight}} from the decomposition's D_i, checking that every
    y node of a column carries the same weight (the partition of unity is a function of the
    expanding coordinates only)."""
    out = []
    for ids, w in zip(dec.idx, dec.weights):
        col = {}
        for k, c in enumerate(ids // nyi):
            if c in col:
                assert w[k] == col[c]
            col[c] = w[k]
        out.append(col)
    return out


def test_distance_pu_p1_linear_ramp():
    """Distance partition of unity (Sec. 4.1.2), p = 1: across the overlap zone of the
    interface x = t the weights of the two neighbouring subdomains fall and rise linearly,
    chi = d_i / (d_i + d_j) with d measured to the artificial faces x = t -/+ delta h only
    (faces on the box boundary, the ends and y = 0, ell, do not count).  delta = 3: the
    left subdomain's weight at x = t + k h, k = -2..2, is 5/6, 2/3, 1/2, 1/3, 1/6; every
    node outside an overlap zone belongs to one subdomain with weight 1."""
    L, n, delta = 4, 8, 3
    g = grid(1, L, n, 4, delta=delta)
    dec = Decomposition(g, "distance")
    W = _weights_by_node(dec, g.ny - 1)
    left = {-2: 5 / 6, -1: 2 / 3, 0: 1 / 2, 1: 1 / 3, 2: 1 / 6}
    for t in range(1, L):
        for k, wl in left.items():
            col = t * n + k - 1          # 0-based interior column of node a = t n + k
            assert W[t - 1][col] == pytest.approx(wl, abs=1e-14)
            assert W[t][col] == pytest.approx(1.0 - wl, abs=1e-14)
    for i in range(L):
        for col, wv in W[i].items():
            a = col + 1
            if all(abs(a - t * n) >= delta for t in range(1, L)):
                assert wv == 1.0


def test_distance_pu_p2_corner_zone_and_physical_boundary():
    """Distance partition of unity (Sec. 4.1.2), p = 2, delta = 3, h = 1/8.  d_i is the
    distance to the artificial part of the subdomain's boundary (the faces not on the box
    boundary), so near the interior vertex (1, 1) four subdomains share a node with weights
    fixed by the distances to their inner faces (worked by hand below), while along the
    overlap zone of x_1 = 1 next to the box face x_2 = 0 the two covering subdomains keep
    the 1-D ramp: the physical face x_2 = 0 is not a face to measure to, and the subdomains
    are clipped at the box (no face at x_2 = -delta h either)."""
    L, n, delta = 3, 8, 3
    g = grid(2, L, n, 3, delta=delta)
    dec = Decomposition(g, "distance")
    nx, nyi = g.nx, g.ny - 1
    W = _weights_by_node(dec, nyi)
    sub = {(i1, i2): i1 * L + i2 for i1 in range(L) for i2 in range(L)}
    # node (8 + u, 8 + v): weights of subdomains (0,0), (1,0), (0,1), (1,1)
    corner = {(0, 0): (1 / 4, 1 / 4, 1 / 4, 1 / 4),
              (-1, 0): (3 / 10, 1 / 5, 3 / 10, 1 / 5),
              (-2, -2): (5 / 8, 1 / 8, 1 / 8, 1 / 8),
              (2, -1): (1 / 8, 1 / 2, 1 / 8, 1 / 4),
              (-1, 2): (1 / 8, 1 / 8, 1 / 2, 1 / 4)}
    for (u, v), ws in corner.items():
        col = (n + u - 1) * nx + (n + v - 1)
        for key, wv in zip(((0, 0), (1, 0), (0, 1), (1, 1)), ws):
            assert W[sub[key]][col] == pytest.approx(wv, abs=1e-14)
    # next to the face x_2 = 0 (a_2 = 1): the ramp of the x_1 = 1 overlap zone
    for u, wl in {-2: 5 / 6, -1: 2 / 3, 0: 1 / 2, 1: 1 / 3, 2: 1 / 6}.items():
        col = (n + u - 1) * nx + 0
        assert W[sub[(0, 0)]][col] == pytest.approx(wl, abs=1e-14)
        assert W[sub[(1, 0)]][col] == pytest.approx(1.0 - wl, abs=1e-14)


@pytest.mark.parametrize("pu", ["equal", "distance"])
@pytest.mark.parametrize("p", [1, 2])
def test_coarse_basis_sums_to_periodic_cell_function(p, pu):
    """Definition 2.1 with the partition of unity of Sec. 2.2: the columns D_i R_i psi of
    R_0^T extended by zero add up to the periodic extension E^# psi itself
    (sum_i R_i^T D_i R_i = I), and A_sigma annihilates that sum on every row whose stencil
    stays away from the x-ends of the box (those rows are translated rows of the periodic
    cell problem whose eigenpair is (sigma, psi))."""
    if p == 1:
        w = Workload("t", p=1, L=5, n=8, overlap=2, kind="cos1")
    else:
        w = Workload("t", p=2, L=3, n=6, overlap=2, kind="asym3")
    g = q1.Grid.from_workload(w)
    P = solvers.Problem(g, potential(w), pu=pu, build_prec=False)
    Z = P.dec.coarse_basis(P.psi)
    assert Z.shape == (g.ndof, g.L ** g.p)
    s = Z @ np.ones(Z.shape[1])
    assert np.abs(s - P.psi).max() <= 1e-14 * np.abs(P.psi).max()
    res = P.Asig @ s
    nyi = g.ny - 1
    if p == 1:
        inner = res.reshape(g.nx, nyi)[1:-1]
    else:
        inner = res.reshape(g.nx, g.nx, nyi)[1:-1, 1:-1]
    assert np.abs(inner).max() <= 1e-10 * P.sigma * np.abs(P.psi).max()
    assert np.abs(res).max() > 1e-6 * P.sigma * np.abs(P.psi).max()   # the x-end rows do not vanish


def test_cfg1_independent_probe_values():
    """The smallest workload (p = 1, L = 8, h = 1/16, V = 10(1 + cos 2 pi x)(1 + sin(pi y)/2)):
    the oracle's cell shift sigma and exact ground state lambda_1, lambda_2 against an
    independent dense generalised eigensolve recorded in tests/golden/cfg1_probe.json
    (12 digits), and the same for V = 0."""
    with open(os.path.join(GOLDEN, "cfg1_probe.json")) as f:
        ref = json.load(f)
    w = WORKLOADS["cfg1"]
    g = q1.Grid.from_workload(w)
    for V, r in ((potential(w), ref), (zeroV(1), ref["v0"])):
        P = solvers.Problem(g, V, build_prec=False)
        assert P.sigma == pytest.approx(r["sigma"], rel=1e-11, abs=0)
        lam, _ = solvers.exact_ground_state(P.A, P.M)
        assert lam == pytest.approx(r["lambda1"], rel=1e-11, abs=0)
    import scipy.linalg as sla2
    P = solvers.Problem(g, potential(w), build_prec=False)
    ev = sla2.eigh(P.A.toarray(), P.M.toarray(), eigvals_only=True, subset_by_index=[0, 1])
    assert ev[1] == pytest.approx(ref["lambda2"], rel=1e-11, abs=0)


@pytest.mark.parametrize("coarse", [False, True])
def test_preconditioner_symmetric_positive(coarse):
    w = Workload("t", p=1, L=5, n=8, overlap=2, kind="cos1")
    g = q1.Grid.from_workload(w)
    P = solvers.Problem(g, potential(w), coarse=coarse)
    rng = np.random.default_rng(1)
    u, v = rng.standard_normal((2, g.ndof))
    assert u @ P.prec(v) == pytest.approx(v @ P.prec(u), rel=1e-11)
    assert u @ P.prec(u) > 0


def test_preconditioner_parts_match_definition():
    """Local part = sum_i R_i^T A_i^{-1} R_i (dense inverses); coarse part =
    Z A_0^{-1} Z^T with Z = blockdiag(D_i R_i psi) (Def. 2.1), checked with
    dense linear algebra on a tiny grid."""
    w = Workload("t", p=1, L=3, n=6, overlap=2, kind="cos1")
    g = q1.Grid.from_workload(w)
    P = solvers.Problem(g, potential(w))
    A = P.Asig.toarray()
    n = g.ndof
    Pl = np.zeros((n, n))
    for ids in P.dec.idx:
        Pl[np.ix_(ids, ids)] += np.linalg.inv(A[np.ix_(ids, ids)])
    Z = np.zeros((n, g.L))
    for i, (ids, wts) in enumerate(zip(P.dec.idx, P.dec.weights)):
        Z[ids, i] = wts * P.psi[ids]
    Pc = Z @ np.linalg.inv(Z.T @ A @ Z) @ Z.T
    rng = np.random.default_rng(5)
    r = rng.standard_normal(n)
    assert np.allclose(P.prec(r), (Pl + Pc) @ r, rtol=1e-10, atol=1e-12)
    # coarse operator of p=1 is tridiagonal for delta < n/2
    A0 = Z.T @ A @ Z
    assert np.abs(np.triu(A0, 2)).max() < 1e-14 * np.abs(A0).max()


def test_single_subdomain_special_case():
    """L = 1: the one subdomain is the whole domain, so M_AS1^{-1} = A^{-1}
    (CG stops after 1 iteration) and M_AS2^{-1} = A^{-1} + rank one, whose
    preconditioned operator has eigenvalues {1, 2} (2 iterations)."""
    g = grid(1, 1, 10, 10, delta=1)
    V = lambda x, y: 5 + 0.0 * x
    b = np.full(g.ndof, g.h ** 2)
    for coarse, expect in ((False, 1), (True, 2)):
        P = solvers.Problem(g, V, coarse=coarse)
        _, it, _ = P.solve(b, x0=np.ones(g.ndof))
        assert it == expect


@pytest.mark.slow
def test_l_robust_iterations_source_problem():
    """Sec. 4.1: CG + M_AS2 iteration counts stay bounded in L while the
    one-level M_AS1 counts grow (source problem f = 1, initial guess 1,
    rTOL = 1e-8, N = L subdomains, delta = 1; h = 1/10 as in Table 1)."""
    counts = {False: [], True: []}
    Ls = (4, 16, 64)
    for coarse in (False, True):
        for L in Ls:
            w = Workload("e1", p=1, L=L, n=10, overlap=1, kind="sin4")
            g = q1.Grid.from_workload(w)
            P = solvers.Problem(g, potential(w), coarse=coarse)
            b = np.full(g.ndof, g.h ** 2)
            _, it, _ = P.solve(b, x0=np.ones(g.ndof))
            counts[coarse].append(it)
    as1, as2 = counts[False], counts[True]
    assert as1[-1] > 2 * as2[-1]
    assert as1[-1] > 3 * as1[0]
    assert as2[-1] <= as2[1] + 20


def test_outer_iterations_independent_of_L():
    """QOSI (Sec. 1.1): the shifted inverse iteration needs O(1) outer steps."""
    outs = []
    for L in (4, 16):
        w = Workload("t", p=1, L=L, n=8, overlap=2, kind="cos1")
        g = q1.Grid.from_workload(w)
        P = solvers.Problem(g, potential(w))
        lam, x, k, inner, info = P.ground_state()
        le, _ = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma, dense_limit=0)
        assert lam == pytest.approx(le, rel=1e-10)
        outs.append(k)
    assert abs(outs[0] - outs[1]) <= 2


def test_printed_cell_shift_is_recorded_unpinned():
    """Sec. 4.1 prints sigma ~ 19.32644 for V = 100 sin^4(pi x) sin^4(pi y),
    h = 1/30.  The printed formula does not give that value; the fixture
    records it as unpinned.  What is checked: our value is quadrature-stable
    (Q = 2 vs Q = 4 agree to 1e-5 relative)."""
    with open(os.path.join(GOLDEN, "paper_sec41_sigma.json")) as f:
        gold = json.load(f)
    assert gold["status"] == "unpinned"
    w = Workload("e1", p=1, L=1, n=30, kind="sin4")
    g2 = q1.Grid.from_workload(w)
    g4 = q1.Grid.from_workload(w.with_(quad_pts=4))
    s2, _ = solvers.cell_eigenpair(g2, potential(w))
    s4, _ = solvers.cell_eigenpair(g4, potential(w))
    assert abs(s2 - s4) / s4 < 1e-5
    assert abs(s2 - gold["sigma_printed"]) > 1.0


# --- SI-LOPCG (Algorithm 1) and the inner-tolerance strategies of Sec. 4.3 ------------

def test_rayleigh_ritz3_brute_force():
    """The orthogonalised Rayleigh-Ritz step returns the minimum of the Rayleigh quotient
    over the span (brute force: the lowest eigenvalue of the projected pencil from an
    explicit B-orthonormal basis), a B-normalised Ritz vector with that quotient and
    positive sum; an exactly dependent third vector is dropped."""
    rng = np.random.default_rng(41)
    n = 30
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n)
    R = rng.standard_normal((n, n))
    B = R @ R.T + n * np.eye(n)
    S = rng.standard_normal((n, 3))
    GA, GB = S.T @ A @ S, S.T @ B @ S
    theta, c = solvers.rayleigh_ritz3(GA, GB, S.sum(axis=0))
    Lb = np.linalg.cholesky(B)
    Qs, _ = np.linalg.qr(Lb.T @ S)                  # B-orthonormal basis: S' = Lb^-T Qs
    Sb = np.linalg.solve(Lb.T, Qs)
    ref = np.linalg.eigvalsh(Sb.T @ A @ Sb)[0]
    assert theta == pytest.approx(ref, rel=1e-12)
    y = S @ c
    assert y @ B @ y == pytest.approx(1.0, rel=1e-12)
    assert y @ A @ y == pytest.approx(theta, rel=1e-12)
    assert y.sum() > 0
    # dependent third vector: same as the two-vector problem
    S2 = np.column_stack([S[:, 0], S[:, 1], 2.0 * S[:, 0] - 3.0 * S[:, 1]])
    t2, c2 = solvers.rayleigh_ritz3(S2.T @ A @ S2, S2.T @ B @ S2, S2.sum(axis=0))
    ref2 = sla.eigh(S[:, :2].T @ A @ S[:, :2], S[:, :2].T @ B @ S[:, :2], eigvals_only=True)[0]
    assert t2 == pytest.approx(ref2, rel=1e-10)
    assert c2[2] == 0.0


@pytest.mark.parametrize("inner", ["fixed", "adaptive", "fused"])
def test_si_lopcg_reaches_ground_state(inner):
    """All three inner strategies of Sec. 4.3 reach the exact ground state (dense
    generalised eigensolver) to 1e-10 with residual eta <= 1e-8, and the Ritz values
    never increase (x_k lies in the next search space)."""
    w = Workload("t", p=1, L=6, n=8, overlap=2, kind="cos1")
    P = solvers.Problem(q1.Grid.from_workload(w), potential(w))
    le, _ = solvers.exact_ground_state(P.A, P.M, dense_limit=5000)
    rhos = []
    orig = solvers.rayleigh_ritz3

    def spy(GA, GB, sums, drop=1e-10):
        t, c = orig(GA, GB, sums, drop)
        rhos.append(P.sigma + t)
        return t, c

    solvers.rayleigh_ritz3 = spy
    try:
        lam, x, k, inner_its, info = P.ground_state_lopcg(inner=inner)
    finally:
        solvers.rayleigh_ritz3 = orig
    assert lam == pytest.approx(le, rel=1e-10)
    assert info["eta"] <= 1e-8
    assert x @ (P.M @ x) == pytest.approx(1.0, rel=1e-12) and x.sum() > 0
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(rhos, rhos[1:]))


def test_si_lopcg_v0_closed_form():
    """V = 0: SI-LOPCG with the fused strategy reaches the closed-form lambda_1."""
    L, n, ny = 12, 8, 8
    g = grid(1, L, n, ny, delta=2)
    P = solvers.Problem(g, zeroV(1))
    h = g.h
    lam1 = mu(np.pi * h / L, h) + mu(np.pi * h, h)
    lam, x, k, inner, info = P.ground_state_lopcg(inner="fused")
    assert lam == pytest.approx(lam1, rel=1e-10)


def test_inner_tolerance_strategies_order():
    """Sec. 4.3: the adaptive inner tolerance min{0.1, ||r_o||} needs fewer inner
    iterations in total than the fixed 1e-8, and the fused variant (the Schwarz
    preconditioner in place of the inner solve) fewer still; all reach the same
    eigenvalue."""
    w = Workload("t", p=1, L=16, n=16, overlap=2, kind="cos1")
    P = solvers.Problem(q1.Grid.from_workload(w), potential(w))
    tot, lams = {}, {}
    for inner in ("fixed", "adaptive", "fused"):
        lam, x, k, its, info = P.ground_state_lopcg(inner=inner)
        tot[inner] = sum(its)
        lams[inner] = lam
    assert tot["adaptive"] < tot["fixed"]
    assert tot["fused"] < tot["adaptive"]
    assert lams["adaptive"] == pytest.approx(lams["fixed"], rel=1e-10)
    assert lams["fused"] == pytest.approx(lams["fixed"], rel=1e-10)


def test_source_sweep_goldens_are_the_oracles():
    """The stored iteration counts of tests/golden/source_sweeps.json (the reference of the
    GPU sweeps of Sec. 4.1) are what the oracle computes now: a few entries recomputed."""
    with open(os.path.join(GOLDEN, "source_sweeps.json")) as f:
        gold = json.load(f)
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(GOLDEN, "make_source_sweeps.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    f3 = gold["fig3"]
    for L in (4, 8):
        i = f3["L"].index(L)
        assert mk.source_count(L, 30, 1, False, "equal") == f3["as1"][i]
        assert mk.source_count(L, 30, 1, True, "equal") == f3["as2"][i]
    row = [r for r in gold["table1"]["cases"] if r["n"] == 10 and r["delta"] == 2][0]
    assert mk.source_count(4, 10, 2, True, "distance") == row["as2"][0]
    assert mk.source_count(4, 10, 2, False, "distance") == row["as1"][0]
