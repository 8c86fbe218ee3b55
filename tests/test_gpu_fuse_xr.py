"""The x, r update of a p = 1 PCG iteration fused into the restriction packing
(DD_OPT_FUSE_XR, opt-in, with BF16/TF32 local inverses).

Each subdomain's block forms r - alpha q with the same FMA as the separate x/r update, the
owner of each node column updates x and adds to (r, r), and the prolong-sum stores r - alpha q.
So x and r take the same values in every iteration as with the separate update; only (r, r)
is summed in another order, which can move the stop test by an iteration at most.  Where the
iteration counts agree, the solutions are bit-identical."""
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
    "L1": Workload("L1", p=1, L=1, n=8, overlap=2, kind="cos1"),
}


def _eta(P, x, lam):
    Mx = P.M @ x
    return np.linalg.norm(P.A @ x - lam * Mx) / (abs(lam) * np.linalg.norm(Mx))


@pytest.mark.parametrize("pairs", [1, 0])
@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("name", list(CASES))
def test_fused_xr_update(name, prec, pairs):
    w = CASES[name]
    P = oracle_problem(w, build_prec=False)
    lam_ex, _ = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma,
                                           dense_limit=3000 if w.dofs <= 3000 else 0)
    out = {}
    for fuse in (0, 1):
        with make_solver(w, precision=prec) as es:
            es.prepare()
            dd.dd_set_option(es.ctx, dd.DD_OPT_PAIRS, pairs)
            dd.dd_set_option(es.ctx, dd.DD_OPT_FUSE_XR, fuse)
            b = gpu_vec(np.zeros(w.dofs))
            dd.dd_apply_operator(es.ctx, dd.DD_OP_MASS, gpu_vec(np.ones(w.dofs)), b)
            y = gpu_vec(np.zeros(w.dofs))
            it, rel = dd.dd_pcg_solve(es.ctx, b, y, 1e-8)
            x = gpu_vec(np.ones(w.dofs))
            lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
            out[fuse] = (it, rel, host(y), lam, tot, host(x))
    (i0, r0, y0, l0, t0, x0), (i1, r1, y1, l1, t1, x1) = out[0], out[1]
    print(f"{name} {prec} pairs={pairs}: PCG {i0} {i1}, inner totals {t0} {t1}")
    assert abs(i0 - i1) <= 1 and r1 <= 1e-8
    if i0 == i1:
        assert np.array_equal(y0, y1)
    for lam, x in ((l0, x0), (l1, x1)):
        assert abs(lam - lam_ex) <= 1e-10 * abs(lam_ex)
        assert _eta(P, x, lam) <= 1e-8 + 1e-12
    assert abs(t0 - t1) <= 3
    if t0 == t1:
        assert l0 == l1 and np.array_equal(x0, x1)


def test_fused_xr_option_validation():
    with make_solver(CASES["cfg1"], precision="fp64") as es:
        with pytest.raises(dd.DDError):
            dd.dd_set_option(es.ctx, dd.DD_OPT_FUSE_XR, 1)
        dd.dd_set_option(es.ctx, dd.DD_OPT_FUSE_XR, 0)
        dd.dd_set_option(es.ctx, dd.DD_OPT_FUSE_XR, -1)
    with make_solver(Workload("p2", p=2, L=2, n=6, overlap=2, kind="asym3"), precision="bf16") as es:
        with pytest.raises(dd.DDError):
            dd.dd_set_option(es.ctx, dd.DD_OPT_FUSE_XR, 1)
    with make_solver(CASES["cfg1"], precision="bf16") as es:
        for bad in (-2, 2):
            with pytest.raises(dd.DDError):
                dd.dd_set_option(es.ctx, dd.DD_OPT_FUSE_XR, bad)
        dd.dd_set_option(es.ctx, dd.DD_OPT_FUSED_PQ, 0)   # the two-kernel p update: no fused x/r update
        with pytest.raises(dd.DDError):
            dd.dd_set_option(es.ctx, dd.DD_OPT_FUSE_XR, 1)
