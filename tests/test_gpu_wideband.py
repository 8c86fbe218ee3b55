"""Bands wider than the shared-memory window (b > 160) at a size the oracle solves in
seconds: p = 2, L = 2, n = 10, ell = 1.5 (ny - 1 = 14), overlap 2.  The local matrices have
half bandwidth 11 * 14 + 15 = 169 and the shifted cell operator 2 * 10 * 14 + 2 * 14 + 1 =
309, so both the FP64 factors (plain method) and the FP32 factors (mixed form, cell
preconditioner) go through the blocked panel factorisation.  Checked against the oracle:
the cell pair, the FP64 preconditioner to 1e-10, the BF16 one to its rounding, and the ground
state of both forms to the 1e-10 eigenvalue target."""
import numpy as np
import pytest

import paper_2311_08757_gb300 as dd
from ddinputs import Workload
from oracle import solvers
from tests.gpu_util import gpu_vec, host, make_solver, oracle_problem, rel_err, sigma_tol

pytestmark = pytest.mark.gpu

W = Workload("p2_wide", p=2, L=2, n=10, ell=1.5, overlap=2, kind="asym3")


@pytest.fixture(scope="module")
def oracle():
    P = oracle_problem(W)
    lam, _ = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma, dense_limit=0)
    return P, lam


def test_bands_exceed_the_window():
    with make_solver(W) as es:
        info = dd.dd_query(es.ctx)
    assert info["band_local"] == 11 * 14 + 15 > 160
    assert 2 * W.n * (W.ny - 1) + 2 * (W.ny - 1) + 1 > 160


def test_cell_pair(oracle):
    P, _ = oracle
    import torch
    with make_solver(W) as es:
        psi = torch.zeros(P.psi_cell.size, dtype=torch.float64, device="cuda:0")
        sigma = dd.dd_cell_eigenpair(es.ctx, psi)
    assert abs(sigma - P.sigma) <= sigma_tol(P)
    assert rel_err(host(psi), P.psi_cell) < 1e-8


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("bf16", 2e-2)])
def test_preconditioner(oracle, prec, tol):
    P, _ = oracle
    rng = np.random.default_rng(8)
    r = rng.standard_normal(W.dofs)
    with make_solver(W, precision=prec) as es:
        es.prepare()
        z = gpu_vec(np.zeros(W.dofs))
        dd.dd_apply_preconditioner(es.ctx, gpu_vec(r), z)
    assert rel_err(host(z), P.prec(r)) < tol


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_ground_state(oracle, prec):
    P, lam_ex = oracle
    with make_solver(W, precision=prec) as es:
        es.prepare()
        x = gpu_vec(np.ones(W.dofs))
        lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
    assert abs(lam - lam_ex) <= 1e-10 * abs(lam_ex)
    xh = host(x)
    Mx = P.M @ xh
    assert np.linalg.norm(P.A @ xh - lam * Mx) / (abs(lam) * np.linalg.norm(Mx)) <= 1.5e-8
