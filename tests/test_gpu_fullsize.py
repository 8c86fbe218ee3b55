"""Parity at the full size of the bench workload (L = 2048, h = 1/32, delta = 4:
2,031,585 unknowns, 2048 subdomains), in the launch configuration bench.py times.

The oracle handles this size in tens of seconds: its CSR operators, its M_AS2^{-1} with
2048 banded factorisations, and the exact ground state by banded-Cholesky inverse
iteration on A_sigma.  Every output is compared in full (no sampling needed).
"""
import numpy as np
import pytest

import paper_2311_08757_gb300 as dd
from ddinputs import WORKLOADS
from oracle import solvers
from tests.gpu_util import gpu_vec, host, make_solver, oracle_problem, rel_err, sigma_tol

pytestmark = pytest.mark.gpu

W = WORKLOADS["cfg2"]


@pytest.fixture(scope="module")
def oracle():
    P = oracle_problem(W)
    lam_ex, _ = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma, dense_limit=0)
    return P, lam_ex


@pytest.fixture(scope="module", params=["fp64", "bf16"])
def gpu(request):
    es = make_solver(W, precision=request.param)
    es.prepare()
    yield request.param, es
    es.close()


def test_fullsize_cell_shift(oracle, gpu):
    P, _ = oracle
    prec, es = gpu
    assert abs(es.info["sigma"] - P.sigma) <= sigma_tol(P)


def test_fullsize_operator(oracle, gpu):
    P, _ = oracle
    _, es = gpu
    x = np.random.default_rng(21).standard_normal(W.dofs)
    y = gpu_vec(np.zeros(W.dofs))
    dd.dd_apply_operator(es.ctx, dd.DD_OP_ASIGMA, gpu_vec(x), y)
    assert rel_err(host(y), P.Asig @ x) < 1e-12


def test_fullsize_coarse_matrix(oracle, gpu):
    P, _ = oracle
    _, es = gpu
    N = W.L
    A0 = np.zeros((N, N))
    dd.dd_coarse_matrix(es.ctx, A0)
    assert rel_err(A0, P.prec.A0) < 1e-12


def test_fullsize_preconditioner(oracle, gpu):
    """At L = 2048 the coarse matrix is ill conditioned (kappa(A_0) ~ 1.7e6: its smallest
    eigenvalue carries the near-null mode psi of A_sigma), so two correct roundings of A_0
    and of its solve differ by about eps kappa(A_0) in the coarse correction; the FP64
    tolerance is 50 eps kappa(A_0), the rounded (BF16) form keeps its 2e-2."""
    P, _ = oracle
    prec, es = gpu
    r = np.random.default_rng(22).standard_normal(W.dofs)
    z = gpu_vec(np.zeros(W.dofs))
    dd.dd_apply_preconditioner(es.ctx, gpu_vec(r), z)
    ev = np.linalg.eigvalsh(P.prec.A0)
    tol = max(1e-10, 50 * np.finfo(float).eps * ev[-1] / ev[0])
    assert rel_err(host(z), P.prec(r)) < (tol if prec == "fp64" else 2e-2)


def test_fullsize_ground_state(oracle, gpu):
    P, lam_ex = oracle
    prec, es = gpu
    x = gpu_vec(np.ones(W.dofs))
    lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
    assert abs(lam - lam_ex) <= 1e-10 * abs(lam_ex)
    xh = host(x)
    Mx = P.M @ xh
    eta = np.linalg.norm(P.A @ xh - lam * Mx) / (abs(lam) * np.linalg.norm(Mx))
    assert eta <= 1e-8 + 1e-12   # the stop rule's 1e-8, plus the rounding of recomputing eta
    assert xh @ Mx == pytest.approx(1.0, rel=1e-12)


def test_fullsize_coarse_solve_by_dense_inverse(oracle):
    """The other coarse-solve form at full size (the default for p = 1 is cyclic reduction)."""
    P, _ = oracle
    es = make_solver(W, precision="fp64")
    try:
        dd.dd_set_option(es.ctx, dd.DD_OPT_COARSE_SOLVE, 2)
        es.prepare()
        r = np.random.default_rng(24).standard_normal(W.dofs)
        z = gpu_vec(np.zeros(W.dofs))
        dd.dd_apply_preconditioner(es.ctx, gpu_vec(r), z)
        ev = np.linalg.eigvalsh(P.prec.A0)
        tol = max(1e-10, 50 * np.finfo(float).eps * ev[-1] / ev[0])
        assert rel_err(host(z), P.prec(r)) < tol
    finally:
        es.close()
