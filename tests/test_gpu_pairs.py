"""Float pairs in the PCG iteration (DD_OPT_PAIRS = 1, the default with rounded local inverses):
the matvec q = A_sigma p on the FP32 pipe (the fused p = 1 pass, the p = 2 pass), against the
FP64 form of the same iteration; every dot product stays FP64.

The pair arithmetic changes only the inner solve's operator (by at most 2^-43 times the sum of
the taps' magnitudes); the outer
iteration's residuals and Rayleigh quotients stay FP64.  So both forms must reach the stop
rule's eta <= 1e-8 measured in FP64 by the oracle's matrices, the same eigenvalue (well inside
the 1e-10 target), and the oracle's exact eigenvalue, with inner iteration counts that differ
by at most a few.  A right-hand side scaled by 2^-40 or 2^40 gives the same iteration count and
the scaled solution, bit for bit (the splits of the coefficients and of p are exact under a
power-of-two scaling; the BF16 local solves keep the float exponent range, which bounds the
scales a mixed solve can take)."""
import numpy as np
import pytest

import paper_2311_08757_gb300 as dd
from ddinputs import WORKLOADS, Workload
from oracle import solvers
from tests.gpu_util import gpu_vec, host, make_solver, oracle_problem

pytestmark = pytest.mark.gpu

CASES = {
    "cfg1": WORKLOADS["cfg1"],
    "cfg2_small": WORKLOADS["cfg2_small"],
    "ragged": Workload("ragged", p=1, L=5, n=10, ell=1.2, overlap=3, kind="cos4", seed=7),
    "L256": Workload("L256", p=1, L=256, n=32, overlap=4, kind="cos4", seed=11),
    "p2": Workload("p2", p=2, L=3, n=6, overlap=2, kind="asym3"),
    "p2_wells": Workload("p2_wells", p=2, L=4, n=8, overlap=2, kind="wells"),
}


def _eta(P, x, lam):
    Mx = P.M @ x
    return np.linalg.norm(P.A @ x - lam * Mx) / (abs(lam) * np.linalg.norm(Mx))


def _solve(w, prec, arith, method):
    with make_solver(w, precision=prec) as es:
        es.prepare()
        dd.dd_set_option(es.ctx, dd.DD_OPT_PAIRS, arith)
        x = gpu_vec(np.ones(w.dofs))
        if method == "ipm":
            lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
        else:
            lam, outer, tot, mx = dd.dd_lopcg(es.ctx, x, inner="fused")
        return lam, tot, host(x)


@pytest.mark.parametrize("method", ["ipm", "lopcg"])
@pytest.mark.parametrize("prec", ["bf16", "fp64"])
@pytest.mark.parametrize("name", list(CASES))
def test_pairs_reach_the_fp64_ground_state(name, prec, method):
    w = CASES[name]
    P = oracle_problem(w, build_prec=False)
    lam_ex, _ = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma,
                                           dense_limit=3000 if w.dofs <= 3000 else 0)
    l0, t0, x0 = _solve(w, prec, 0, method)
    l1, t1, x1 = _solve(w, prec, 1, method)
    print(f"{name} {prec} {method}: inner {t0} (FP64 q) {t1} (pairs); "
          f"lambda diff {abs(l1 - l0) / abs(l0):.1e}; eta {_eta(P, x0, l0):.2e} {_eta(P, x1, l1):.2e}")
    for lam, x in ((l0, x0), (l1, x1)):
        assert abs(lam - lam_ex) <= 1e-10 * abs(lam_ex)
        assert _eta(P, x, lam) <= 1e-8 + 1e-12
    assert abs(l1 - l0) <= 1e-11 * abs(l0)
    assert abs(t1 - t0) <= max(3, 0.05 * t0)


@pytest.mark.parametrize("name", ["p2", "p2_wells"])
def test_tiled_3d_pairs_matvec(name):
    """The shared-memory tiled p = 2 pass (DD_OPT_TILED3) against the cached one: the same q
    per node, (p, q) summed in another order, so the same ground state within the stop rule and
    iteration counts within a few."""
    w = CASES[name]
    P = oracle_problem(w, build_prec=False)
    lam_ex, _ = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma, dense_limit=3000 if w.dofs <= 3000 else 0)
    out = {}
    for tiled in (0, 1):
        with make_solver(w, precision="bf16") as es:
            es.prepare()
            dd.dd_set_option(es.ctx, dd.DD_OPT_TILED3, tiled)
            x = gpu_vec(np.ones(w.dofs))
            lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
            out[tiled] = (lam, tot, host(x))
    print(f"{name}: inner {out[0][1]} (cached) {out[1][1]} (tiled)")
    for lam, tot, x in out.values():
        assert abs(lam - lam_ex) <= 1e-10 * abs(lam_ex)
        assert _eta(P, x, lam) <= 1e-8 + 1e-12
    assert abs(out[0][1] - out[1][1]) <= 3


@pytest.mark.parametrize("name", ["cfg1", "cfg2_small", "L256"])
def test_pairs_pcg_solve(name):
    """The shifted solve A_sigma w = M 1 to rTOL = 1e-8: the same iteration count within one or
    two, and solutions whose difference lies almost entirely along the ground state (the
    system's near-null direction, where each form's rounding is amplified by 1/(lambda_1 - sigma))."""
    w = CASES[name]
    P = oracle_problem(w, build_prec=False)
    lam_ex, psi = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma,
                                             dense_limit=3000 if w.dofs <= 3000 else 0)
    out = {}
    for arith in (0, 1):
        with make_solver(w, precision="bf16") as es:
            es.prepare()
            dd.dd_set_option(es.ctx, dd.DD_OPT_PAIRS, arith)
            b = gpu_vec(np.zeros(w.dofs))
            dd.dd_apply_operator(es.ctx, dd.DD_OP_MASS, gpu_vec(np.ones(w.dofs)), b)
            x = gpu_vec(np.zeros(w.dofs))
            it, rel = dd.dd_pcg_solve(es.ctx, b, x, 1e-8)
            out[arith] = (it, rel, host(x))
    assert abs(out[0][0] - out[1][0]) <= 2
    assert out[1][1] <= 1e-8
    d = out[1][2] - out[0][2]
    Mpsi = P.M @ psi
    d_perp = d - psi * (psi @ (P.M @ d)) / (psi @ Mpsi)
    print(f"{name}: iterations {out[0][0]} {out[1][0]}; |d| / |x| {np.linalg.norm(d) / np.linalg.norm(out[0][2]):.1e}, "
          f"off the ground state {np.linalg.norm(d_perp) / np.linalg.norm(out[0][2]):.1e}")
    assert np.linalg.norm(d_perp) <= 1e-6 * np.linalg.norm(out[0][2])


@pytest.mark.parametrize("e", [-40, 40])
def test_pairs_scale_invariance(e):
    w = CASES["cfg2_small"]
    out = {}
    for scale in (1.0, 2.0 ** e):
        with make_solver(w, precision="bf16") as es:
            es.prepare()
            b = gpu_vec(np.zeros(w.dofs))
            dd.dd_apply_operator(es.ctx, dd.DD_OP_MASS, gpu_vec(np.full(w.dofs, scale)), b)
            x = gpu_vec(np.zeros(w.dofs))
            it, rel = dd.dd_pcg_solve(es.ctx, b, x, 1e-8)
            out[scale] = (it, rel, host(x) / scale)
    (i0, r0, x0), (i1, r1, x1) = out.values()
    assert i0 == i1 and r1 <= 1e-8
    assert np.array_equal(x0, x1)


def test_option_validation():
    w = CASES["cfg1"]
    with make_solver(w, precision="bf16") as es:
        for bad in (-2, 2):
            with pytest.raises(dd.DDError):
                dd.dd_set_option(es.ctx, dd.DD_OPT_PAIRS, bad)
    # p = 1 stages whole node columns in one block: at most 256 padded rows
    with make_solver(Workload("tall", p=1, L=1, n=32, ell=9.0, overlap=2, kind="cos1"), precision="bf16") as es:
        with pytest.raises(dd.DDError):
            dd.dd_set_option(es.ctx, dd.DD_OPT_PAIRS, 1)
        dd.dd_set_option(es.ctx, dd.DD_OPT_PAIRS, 0)
    with make_solver(Workload("p2", p=2, L=2, n=6, overlap=2, kind="asym3"), precision="bf16") as es:
        dd.dd_set_option(es.ctx, dd.DD_OPT_PAIRS, 1)
        dd.dd_set_option(es.ctx, dd.DD_OPT_PAIRS, 0)


@pytest.mark.parametrize("name", ["cfg1", "cfg2_small", "ragged", "p2", "p2_wells"])
def test_pair_matvec_node_bound(name):
    """The float-pair matvec of the PCG iteration, node by node against the FP64 stencil of the
    same context: |y_pairs - y|_i <= 32 * 2^-47 * (|A_sigma| |x|)_i.  Per term the truncated
    splits of the coefficient and of x leave up to 2^-47 each and the dropped product of the
    two low words 2^-48; the low-order accumulator is rounded to FP32 three times per tap, at
    2^-24 of a value that grows with the running sum, so its share grows with the number of
    taps (measured: up to 8.5 with 9 taps, 13.4 with 27).  Checked on the ground state (where
    A_sigma x cancels) and on random signs at two scales."""
    w = CASES[name]
    P = oracle_problem(w, build_prec=False)
    rng = np.random.default_rng(5)
    with make_solver(w, precision="bf16") as es:
        sigma = es.prepare()
        absA = abs(P.A - sigma * P.M)
        _, psi = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma, dense_limit=3000 if w.dofs <= 3000 else 0)
        worst = 0.0
        for x in (psi, rng.standard_normal(w.dofs), 1e-7 * rng.standard_normal(w.dofs)):
            y64 = gpu_vec(np.zeros(w.dofs))
            y2 = gpu_vec(np.zeros(w.dofs))
            dd.dd_apply_operator(es.ctx, dd.DD_OP_ASIGMA, gpu_vec(x), y64)
            dd.dd_apply_asigma_pairs(es.ctx, gpu_vec(x), y2)
            bound = 2.0 ** -47 * (absA @ np.abs(x))
            err = np.abs(host(y2) - host(y64))
            assert np.all(err <= 32 * bound + 1e-300), (name, float((err / np.maximum(bound, 1e-300)).max()))
            worst = max(worst, float((err / np.maximum(bound, 1e-300)).max()))
        print(f"{name}: max |y_pairs - y| / (2^-47 |A||x|) = {worst:.2f}")
