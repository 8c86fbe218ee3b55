"""Parity of the CUDA path (through the C ABI) with the oracle, FP64 local solves.

Workloads span several subdomain types, ragged sizes (ny - 1 not a multiple of the
padding, n not a power of two), p = 1 and p = 2, L = 1 and L = 2, both partitions of
unity and the one-level ablation.  Floating-point tolerances: operators and the
preconditioner are FP64 with O(10) terms per entry, so 1e-12 relative (max norm) is
loose by two orders; eigenvalues must meet the 1e-10 relative target.
"""
import numpy as np
import pytest

import paper_2311_08757_gb300 as dd
from ddinputs import Workload, WORKLOADS
from tests.gpu_util import sigma_tol, gpu_vec, host, make_solver, oracle_problem, rel_err
from oracle import solvers

pytestmark = pytest.mark.gpu

CASES = {
    "cfg1": WORKLOADS["cfg1"],
    "cfg2_small": WORKLOADS["cfg2_small"],
    "p2_small": WORKLOADS["cfg3_small"],
    "cfg3_mid": WORKLOADS["cfg3_mid"],
    "p2_types": Workload("p2_types", p=2, L=3, n=6, overlap=2, kind="asym3"),
    "ragged": Workload("ragged", p=1, L=5, n=10, ell=1.2, overlap=3, kind="cos4", seed=7),
    "L1": Workload("L1", p=1, L=1, n=10, overlap=2, kind="cos1"),
    "L2": Workload("L2", p=1, L=2, n=8, overlap=3, kind="cos1"),
    "v0": WORKLOADS["cfg1_v0"],
}


@pytest.fixture(scope="module")
def built():
    out = {}
    for name, w in CASES.items():
        es = make_solver(w)
        es.prepare()
        out[name] = (w, es, oracle_problem(w))
    yield out
    for w, es, P in out.values():
        es.close()


@pytest.mark.parametrize("name", list(CASES))
def test_operators(built, name):
    w, es, P = built[name]
    rng = np.random.default_rng(11)
    x = rng.standard_normal(w.dofs)
    xg = gpu_vec(x)
    y = gpu_vec(np.zeros(w.dofs))
    for op, Aref in ((dd.DD_OP_A, P.A), (dd.DD_OP_MASS, P.M), (dd.DD_OP_ASIGMA, P.Asig)):
        dd.dd_apply_operator(es.ctx, op, xg, y)
        assert rel_err(host(y), Aref @ x) < 1e-12, op


@pytest.mark.parametrize("name", list(CASES))
def test_cell_eigenpair(built, name):
    w, es, P = built[name]
    import torch
    psi = torch.zeros(P.psi_cell.size, dtype=torch.float64, device="cuda:0")
    sigma = dd.dd_cell_eigenpair(es.ctx, psi)
    dd.dd_coarse_build(es.ctx)
    assert abs(sigma - P.sigma) <= sigma_tol(P)
    assert rel_err(host(psi), P.psi_cell) < 1e-8


@pytest.mark.parametrize("name", [k for k in CASES if k != "L1"])
def test_coarse_matrix(built, name):
    w, es, P = built[name]
    N = w.L ** w.p
    A0 = np.zeros((N, N))
    dd.dd_coarse_matrix(es.ctx, A0)
    assert rel_err(A0, P.prec.A0) < 1e-11


@pytest.mark.parametrize("name", list(CASES))
def test_preconditioner(built, name):
    w, es, P = built[name]
    rng = np.random.default_rng(3)
    r = rng.standard_normal(w.dofs)
    z = gpu_vec(np.zeros(w.dofs))
    dd.dd_apply_preconditioner(es.ctx, gpu_vec(r), z)
    assert rel_err(host(z), P.prec(r)) < 1e-10


@pytest.mark.parametrize("coarse,pu", [(0, "equal"), (1, "distance"), (0, "distance")])
@pytest.mark.parametrize("name", ["cfg1", "p2_types", "L2"])
def test_preconditioner_variants(name, coarse, pu):
    w = CASES[name]
    P = oracle_problem(w, coarse=bool(coarse), pu=pu)
    with make_solver(w, coarse=coarse, pu=pu) as es:
        es.prepare()
        rng = np.random.default_rng(5)
        r = rng.standard_normal(w.dofs)
        z = gpu_vec(np.zeros(w.dofs))
        dd.dd_apply_preconditioner(es.ctx, gpu_vec(r), z)
        assert rel_err(host(z), P.prec(r)) < 1e-10


@pytest.mark.parametrize("name", list(CASES))
def test_pcg_solve(built, name):
    """Same iteration count as the oracle's PCG (+-1 for rounding order) and a true
    relative residual at the requested tolerance."""
    w, es, P = built[name]
    rng = np.random.default_rng(17)
    b = rng.standard_normal(w.dofs)
    x = gpu_vec(np.zeros(w.dofs))
    it, rel = dd.dd_pcg_solve(es.ctx, gpu_vec(b), x, rtol=1e-8, maxit=2000)
    _, it_ref, _ = solvers.pcg(P.Asig, b, None, P.prec, 1e-8, 2000)
    assert abs(it - it_ref) <= 1
    xh = host(x)
    true_rel = np.linalg.norm(b - P.Asig @ xh) / np.linalg.norm(b)
    assert true_rel < 2e-8
    assert rel < 1e-8


@pytest.mark.parametrize("name", list(CASES))
def test_ground_state(built, name):
    w, es, P = built[name]
    x = gpu_vec(np.ones(w.dofs))
    lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
    lam_ex, x_ex = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma,
                                              dense_limit=3000 if w.dofs <= 3000 else 0)
    assert abs(lam - lam_ex) <= 1e-10 * abs(lam_ex)
    xh = host(x)
    assert xh.sum() > 0
    assert xh @ (P.M @ xh) == pytest.approx(1.0, rel=1e-12)
    Mx = P.M @ xh
    eta = np.linalg.norm(P.A @ xh - lam * Mx) / (abs(lam) * np.linalg.norm(Mx))
    assert eta <= 1.5e-8
    lam_o, _, k_o, inner_o, _ = P.ground_state()
    assert abs(outer - k_o) <= 1
    assert abs(mx - max(inner_o)) <= 1


def test_host_buffers_match_device(built):
    w, es, P = built["cfg1"]
    rng = np.random.default_rng(2)
    b = rng.standard_normal(w.dofs)
    xd = gpu_vec(np.zeros(w.dofs))
    xh = np.zeros(w.dofs)
    dd.dd_pcg_solve(es.ctx, gpu_vec(b), xd)
    dd.dd_pcg_solve(es.ctx, b, xh)
    assert np.array_equal(host(xd), xh)


def test_eigenpair_convenience():
    w = CASES["cfg1"]
    import torch
    from ddinputs import sample_cell_qp
    V = sample_cell_qp(w)
    phi = np.zeros(w.dofs)
    lam, sigma = dd.dd_eigenpair(dd.grid_from_workload(w), V, phi_out=phi)
    P = oracle_problem(w, build_prec=False)
    lam_ex, _ = solvers.exact_ground_state(P.A, P.M)
    assert abs(lam - lam_ex) <= 1e-10 * lam_ex
    assert phi.sum() > 0 and abs(phi @ (P.M @ phi) - 1) < 1e-12
    torch.cuda.synchronize()


def test_status_codes():
    from ddinputs import sample_cell_qp
    w = CASES["cfg1"]
    V = sample_cell_qp(w)
    bad = [dict(n=2), dict(overlap=8), dict(overlap=0), dict(quad_pts=5), dict(L=0)]
    for kw in bad:
        g = dd.grid_from_workload(w)
        for k, v in kw.items():
            setattr(g, k, v)
        with pytest.raises(dd.DDError) as e:
            dd.dd_setup(g, V)
        assert e.value.code == dd.DD_EINVAL
    g = dd.grid_from_workload(w)
    g.q = 2
    with pytest.raises(dd.DDError):
        dd.dd_setup(g, V)
    with pytest.raises(dd.DDError) as e:
        dd.dd_setup(dd.grid_from_workload(w), V[:-1])
    assert e.value.code == dd.DD_EINVAL
    Vn = V.copy()
    Vn[5] = np.nan
    with pytest.raises(dd.DDError) as e:
        dd.dd_setup(dd.grid_from_workload(w), Vn)
    assert e.value.code == dd.DD_ENAN
    ctx = dd.dd_setup(dd.grid_from_workload(w), V)
    try:
        with pytest.raises(dd.DDError) as e:
            dd.dd_pcg_solve(ctx, np.ones(w.dofs), np.zeros(w.dofs))
        assert e.value.code == dd.DD_ESTATE
        dd.dd_cell_eigenpair(ctx)
        dd.dd_coarse_build(ctx)
        with pytest.raises(dd.DDError) as e:
            dd.dd_pcg_solve(ctx, np.ones(w.dofs), np.zeros(w.dofs), rtol=1e-14, maxit=3)
        assert e.value.code == dd.DD_EMAXIT
    finally:
        dd.dd_destroy(ctx)


def test_zero_rhs_and_options(built):
    w, es, P = built["cfg2_small"]
    x = gpu_vec(np.zeros(w.dofs))
    it, rel = dd.dd_pcg_solve(es.ctx, gpu_vec(np.zeros(w.dofs)), x)
    assert it == 0 and np.abs(host(x)).max() == 0.0
    rng = np.random.default_rng(9)
    b = rng.standard_normal(w.dofs)
    res = []
    for graph, every in ((1, 8), (0, 3), (1, 1)):
        dd.dd_set_option(es.ctx, dd.DD_OPT_USE_GRAPH, graph)
        dd.dd_set_option(es.ctx, dd.DD_OPT_CHECK_EVERY, every)
        xx = gpu_vec(np.zeros(w.dofs))
        it, _ = dd.dd_pcg_solve(es.ctx, gpu_vec(b), xx)
        res.append((it, host(xx)))
    assert res[0][0] == res[1][0] == res[2][0]
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][1], res[2][1])
    dd.dd_set_option(es.ctx, dd.DD_OPT_USE_GRAPH, 1)
    dd.dd_set_option(es.ctx, dd.DD_OPT_CHECK_EVERY, 8)


@pytest.mark.parametrize("name", ["cfg1", "p2_types", "ragged", "L2"])
def test_local_rhs_per_warp_bit_exact(built, name):
    """Subdomains of one type solved together by one warp (1, 2 or 4 at a time) take the same
    operations per vector as one at a time, so the preconditioner is bit-identical, and it
    matches the oracle."""
    w, es, P = built[name]
    rng = np.random.default_rng(17)
    r = gpu_vec(rng.standard_normal(w.dofs))
    out = []
    for k in (1, 2, 4, 0):
        dd.dd_set_option(es.ctx, dd.DD_OPT_LOCAL_RHS, k)
        z = gpu_vec(np.zeros(w.dofs))
        dd.dd_apply_preconditioner(es.ctx, r, z)
        out.append(host(z))
    for z in out[1:]:
        assert np.array_equal(z, out[0])
    assert rel_err(out[0], P.prec(host(r))) < 1e-10
    with pytest.raises(dd.DDError):
        dd.dd_set_option(es.ctx, dd.DD_OPT_LOCAL_RHS, 3)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("name", ["cfg1", "cfg2_small", "ragged", "L2", "L1"])
def test_coarse_solve_forms(name, mode):
    """Both forms of the p = 1 coarse solve (cyclic reduction, dense inverse) give the oracle's
    preconditioner."""
    w = CASES[name]
    P = oracle_problem(w)
    es = make_solver(w)
    try:
        dd.dd_set_option(es.ctx, dd.DD_OPT_COARSE_SOLVE, mode)
        es.prepare()
        r = np.random.default_rng(23).standard_normal(w.dofs)
        z = gpu_vec(np.zeros(w.dofs))
        dd.dd_apply_preconditioner(es.ctx, gpu_vec(r), z)
        assert rel_err(host(z), P.prec(r)) < 1e-10
    finally:
        es.close()
