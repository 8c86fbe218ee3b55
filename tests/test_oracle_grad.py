"""Pins of the oracle's potential gradients (Hellmann-Feynman element reduction and the
adjoint of the projected singular system) against what fixes them independently: the
assembled M_V (bilinear identity), the constant-shift closed form, the defining equations
of the adjoint, and central finite differences of exact eigen-solves."""
import numpy as np
import pytest
import scipy.linalg as sla

from ddinputs import Workload, potential, sample_cell_qp, theta_seed, theta8_qp_basis
from oracle import grad, q1, solvers


def _exact(A, M):
    w, v = sla.eigh(A.toarray(), M.toarray(), subset_by_index=[0, 0])
    x = v[:, 0]
    if x.sum() < 0:
        x = -x
    return float(w[0]), x / np.sqrt(x @ (M @ x))


@pytest.mark.parametrize("w", [
    Workload("t", p=1, L=3, n=6, overlap=1, kind="cos1"),
    Workload("t", p=1, L=2, n=5, ell=1.4, overlap=1, kind="cos4", seed=3),
    Workload("t", p=2, L=2, n=4, overlap=1, kind="asym3"),
])
def test_qp_product_bilinear_identity(w):
    """sum_{e,q} V_cell_qp[e,q] qp_product(u, v)[e,q] = u^T M_V v with M_V assembled by the
    oracle from V at global coordinates (periodic, so equal up to rounding)."""
    g = q1.Grid.from_workload(w)
    K, M, MV = q1.assemble_box(g, potential(w))
    rng = np.random.default_rng(7)
    u, v = rng.standard_normal(g.ndof), rng.standard_normal(g.ndof)
    Vqp = sample_cell_qp(w)
    lhs = float(Vqp @ grad.qp_product(g, u, v))
    rhs = float(u @ (MV @ v))
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12 * np.abs(MV).sum())
    # symmetric in (u, v); the all-ones potential gives the mass form
    assert np.allclose(grad.qp_product(g, u, v), grad.qp_product(g, v, u), rtol=0, atol=1e-15)
    assert float(np.ones_like(Vqp) @ grad.qp_product(g, u, v)) == pytest.approx(float(u @ (M @ v)), rel=1e-12)


def test_eigenvalue_gradient_constant_shift():
    """V + c shifts lambda by c: the derivative along the all-ones direction is phi^T M phi = 1."""
    w = Workload("t", p=1, L=4, n=6, overlap=1, kind="cos1")
    g = q1.Grid.from_workload(w)
    K, M, MV = q1.assemble_box(g, potential(w))
    lam, phi = _exact(K + MV, M)
    gl = grad.eigenvalue_gradient(g, phi)
    assert float(gl.sum()) == pytest.approx(1.0, rel=1e-12)
    assert np.all(gl >= 0.0)


def test_adjoint_solution_defining_equations():
    w = Workload("t", p=1, L=4, n=6, overlap=1, kind="cos1")
    g = q1.Grid.from_workload(w)
    K, M, MV = q1.assemble_box(g, potential(w))
    A = (K + MV).tocsr()
    lam, phi = _exact(A, M)
    gphi = np.random.default_rng(3).standard_normal(g.ndof)
    wv = grad.adjoint_solve(A, M, lam, phi, gphi)
    r = gphi - (M @ phi) * (phi @ gphi)
    assert np.linalg.norm((A - lam * M) @ wv - r) <= 1e-10 * np.linalg.norm(r)
    assert abs(phi @ (M @ wv)) <= 1e-12 * np.linalg.norm(wv)


def test_adjoint_iterative_matches_direct():
    """The iterative adjoint (CG preconditioned by the exact factor of A - sigma M) equals
    the direct bordered solve."""
    w = Workload("t", p=1, L=6, n=8, overlap=1, kind="cos1")
    P = solvers.Problem(q1.Grid.from_workload(w), potential(w), build_prec=False)
    lam, phi = _exact(P.A, P.M)
    gphi = np.random.default_rng(5).standard_normal(P.g.ndof)
    wd = grad.adjoint_solve(P.A, P.M, lam, phi, gphi)
    wi = grad.adjoint_solve(P.A, P.M, lam, phi, gphi, sigma=P.sigma, direct_limit=0)
    assert np.abs(wi - wd).max() <= 1e-11 * np.abs(wd).max()


def _solve_theta(w, theta):
    wt = w.with_(params={"theta": theta})
    g = q1.Grid.from_workload(wt)
    K, M, MV = q1.assemble_box(g, potential(wt))
    A = (K + MV).tocsr()
    lam, phi = _exact(A, M)
    return g, A, M, lam, phi


def test_gradients_match_central_differences():
    """d lambda / d theta and d l / d theta for l = ||phi - phi_target||_M^2 (the
    differentiable workload's loss) against Richardson-extrapolated central differences
    (steps 2e-4 and 1e-4) of exact dense eigen-solves, to 1e-6 relative (gradient-vector norm)."""
    w = Workload("t", p=1, L=3, n=8, overlap=2, kind="theta8", seed=5)
    th, tt = theta_seed(5)
    Bq = theta8_qp_basis(w)
    g, A, M, lam, phi = _solve_theta(w, th)
    _, _, _, _, phi_t = _solve_theta(w, tt)
    dlam = Bq @ grad.eigenvalue_gradient(g, phi)
    gphi = 2.0 * (M @ (phi - phi_t))
    dl = Bq @ grad.loss_gradient(g, A, M, lam, phi, gphi)

    def loss(theta):
        _, _, Mm, lm, ph = _solve_theta(w, theta)
        e = ph - phi_t
        return lm, float(e @ (Mm @ e))

    def central(j, eps):
        tp, tm = th.copy(), th.copy()
        tp[j] += eps
        tm[j] -= eps
        (lp, fp), (lm_, fm) = loss(tp), loss(tm)
        return (lp - lm_) / (2 * eps), (fp - fm) / (2 * eps)

    # Richardson extrapolation of two central differences (steps 2e-4 and 1e-4) cancels the
    # O(eps^2) truncation term, leaving O(eps^4) plus rounding noise of ~1e-16 / 1e-4.  The
    # agreement is measured on the gradient vector, max_j |fd_j - g_j| / max_j |g_j|: a
    # component near zero carries only that noise, which no step can remove
    fd = np.array([[(4 * a1 - a2) / 3 for a1, a2 in zip(central(j, 1e-4), central(j, 2e-4))] for j in range(8)])
    assert np.abs(fd[:, 0] - dlam).max() <= 1e-6 * np.abs(dlam).max()
    assert np.abs(fd[:, 1] - dl).max() <= 1e-6 * np.abs(dl).max()
