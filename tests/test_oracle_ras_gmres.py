"""Pins of the oracle's restricted Schwarz preconditioner (M_RAS2^{-1}) and right-preconditioned
GMRES against dense formulas, exact cases, and the boundedness in L of the inner iteration
counts (Sec. 4.2 table)."""
import numpy as np
import pytest

from ddinputs import Workload, potential
from oracle import q1, solvers
from oracle.dd import Decomposition, TwoLevelAS


def _problem(w, **kw):
    return solvers.Problem(q1.Grid.from_workload(w), potential(w), **kw)


@pytest.mark.parametrize("w", [
    Workload("t", p=1, L=4, n=6, overlap=2, kind="cos1"),
    Workload("t", p=2, L=3, n=4, overlap=1, kind="asym3"),
])
def test_ras2_matches_dense_formula(w):
    """M_RAS2^{-1} r = sum_i R_i^T D_i (R_i A R_i^T)^{-1} R_i r + Z A_0^{-1} Z^T r with every
    matrix dense (brute force)."""
    P = _problem(w, restricted=True)
    A = P.Asig.toarray()
    n = A.shape[0]
    r = np.random.default_rng(2).standard_normal(n)
    z = np.zeros(n)
    for ids, D in zip(P.dec.idx, P.dec.weights):
        Ri = np.zeros((len(ids), n))
        Ri[np.arange(len(ids)), ids] = 1.0
        z += Ri.T @ (D * np.linalg.solve(Ri @ A @ Ri.T, Ri @ r))
    Z = P.prec.Z.toarray()
    z += Z @ np.linalg.solve(Z.T @ A @ Z, Z.T @ r)
    assert np.allclose(P.prec(r), z, rtol=1e-10, atol=1e-12 * np.abs(z).max())


def test_ras_single_subdomain_is_exact_inverse():
    """L = 1: one subdomain covering all unknowns, D = I: M_RAS1^{-1} = A^{-1} and GMRES
    converges in one iteration."""
    w = Workload("t", p=1, L=1, n=8, overlap=2, kind="cos1")
    P = _problem(w, coarse=False, restricted=True)
    b = np.random.default_rng(1).standard_normal(P.g.ndof)
    x, it, hist = solvers.gmres(P.Asig, b, None, P.prec, 1e-12, 30)
    assert it == 1
    assert np.linalg.norm(P.Asig @ x - b) <= 1e-11 * np.linalg.norm(b)


def test_gmres_against_direct_solve_and_monotone():
    """Unpreconditioned and preconditioned GMRES reach the direct solution; the residual
    history never increases; with restart >= n it terminates in at most n steps."""
    rng = np.random.default_rng(3)
    n = 40
    A = rng.standard_normal((n, n)) + n * np.eye(n)        # unsymmetric, well conditioned
    b = rng.standard_normal(n)
    x_ref = np.linalg.solve(A, b)
    x, it, hist = solvers.gmres(A, b, None, None, 1e-12, restart=n)
    assert it <= n
    assert np.allclose(x, x_ref, rtol=1e-10, atol=1e-12)
    assert all(b2 <= a2 * (1 + 1e-12) for a2, b2 in zip(hist, hist[1:]))
    Mi = np.diag(1.0 / np.diag(A))
    x2, it2, _ = solvers.gmres(A, b, None, lambda v: Mi @ v, 1e-12, restart=5)
    assert np.allclose(x2, x_ref, rtol=1e-10, atol=1e-12)


def test_gmres_ras2_counts_comparable_to_cg_as2_and_bounded_in_L():
    """Sec. 4.2: GMRES with RAS2 stays bounded as L grows, like CG with AS2 (source problem
    A_sigma u = M 1, delta = 1).  The paper's table has GMRES+RAS2 slightly below CG+AS2 on
    its unstructured mesh; on this structured Q1 grid the two counts agree within a few
    iterations (measured 18/18, 28/29, 30/30 at L = 16, 32, 64), so that is what is pinned."""
    counts = {}
    for L in (16, 32, 64):
        w = Workload("t", p=1, L=L, n=8, overlap=1, kind="cos1")
        Pa = _problem(w)
        Pr = _problem(w, restricted=True)
        b = Pa.M @ np.ones(Pa.g.ndof)
        _, it_cg, _ = Pa.solve(b, rtol=1e-8)
        _, it_gm, _ = Pr.solve_gmres(b, rtol=1e-8, restart=200)
        counts[L] = (it_cg, it_gm)
        assert abs(it_gm - it_cg) <= max(2, it_cg // 5)
    for k in (0, 1):
        assert counts[64][k] <= counts[32][k] + 5


def test_ground_state_with_gmres_ras2_inner():
    """Inverse iteration and SI-LOPCG with GMRES + RAS2 inner solves reach the exact ground
    state."""
    w = Workload("t", p=1, L=6, n=8, overlap=2, kind="cos1")
    P = _problem(w, restricted=True)
    le, _ = solvers.exact_ground_state(P.A, P.M, dense_limit=5000)
    lam, x, k, inner, info = solvers.inverse_iteration(P.Asig, P.M, P.sigma, P.prec, krylov="gmres")
    assert lam == pytest.approx(le, rel=1e-10)
    lam2, x2, k2, inner2, info2 = solvers.si_lopcg(P.A, P.M, P.sigma, P.prec, inner="adaptive", krylov="gmres")
    assert lam2 == pytest.approx(le, rel=1e-10)
    lam3, *_ = solvers.si_lopcg(P.A, P.M, P.sigma, P.prec, inner="fused")
    assert lam3 == pytest.approx(le, rel=1e-10)
