"""SI-LOPCG (Algorithm 1) through the C ABI against the oracle: the iterate after three
Rayleigh-Ritz steps of each inner strategy of Sec. 4.3, and the exact ground state to 1e-10
with residual eta <= 1e-8 at convergence, in FP64 and in the mixed forms.  Full step counts
are only bounded: they depend on rounding (see test_lopcg_fp64_matches_oracle)."""
import numpy as np
import pytest

import paper_2311_08757_gb300 as dd
from ddinputs import Workload, WORKLOADS
from oracle import solvers
from tests.gpu_util import gpu_vec, host, make_solver, oracle_problem, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    "cfg1": WORKLOADS["cfg1"],
    "cfg2_small": WORKLOADS["cfg2_small"],
    "p2_small": WORKLOADS["cfg3_small"],
    "ragged": Workload("ragged", p=1, L=5, n=10, ell=1.2, overlap=3, kind="cos4", seed=7),
    "v0": WORKLOADS["cfg1_v0"],
}


@pytest.fixture(scope="module")
def oracles():
    out = {}
    for name, w in CASES.items():
        P = oracle_problem(w)
        lam_ex, _ = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma,
                                               dense_limit=3000 if w.dofs <= 3000 else 0)
        out[name] = (P, lam_ex)
    return out


def _eta(P, x, lam):
    Mx = P.M @ x
    return np.linalg.norm(P.A @ x - lam * Mx) / (abs(lam) * np.linalg.norm(Mx))


@pytest.mark.parametrize("inner", ["fixed", "adaptive", "fused"])
@pytest.mark.parametrize("name", list(CASES))
def test_lopcg_fp64_matches_oracle(oracles, name, inner):
    P, lam_ex = oracles[name]
    w = CASES[name]
    with make_solver(w) as es:
        es.prepare()
        x = gpu_vec(np.ones(w.dofs))
        lam, outer, tot, mx = dd.dd_lopcg(es.ctx, x, inner)
    lam_o, x_o, k_o, its_o, _ = P.ground_state_lopcg(inner=inner)
    assert abs(lam - lam_ex) <= 1e-10 * abs(lam_ex)
    xh = host(x)
    assert _eta(P, xh, lam) <= 1.5e-8
    assert xh @ (P.M @ xh) == pytest.approx(1.0, rel=1e-12) and xh.sum() > 0
    # the step count: the stop waits for eta at a threshold as tight as the inner solves, and
    # the fused variant's long linear tail drifts by rounding in the direction x_k - x_{k-1}
    # (oracle reruns with 1e-13 relative perturbations of w: 7-8 steps for the fixed and
    # 27-34 for the fused strategy on p2_small), so only a sanity bound here; the
    # trajectory itself is compared step by step below
    assert k_o // 2 <= outer <= 2 * k_o + 2
    if inner == "fused":
        assert tot == outer


@pytest.mark.parametrize("inner", ["fixed", "adaptive", "fused"])
@pytest.mark.parametrize("name", ["cfg1", "cfg2_small", "p2_small", "ragged"])
def test_lopcg_first_steps_match_oracle(oracles, name, inner):
    """Before rounding is amplified, the iterates agree: x_4 after three Rayleigh-Ritz steps
    (the call stops with DD_EMAXIT and returns its last iterate) against the oracle's."""
    P, lam_ex = oracles[name]
    w = CASES[name]
    with make_solver(w) as es:
        es.prepare()
        x = gpu_vec(np.ones(w.dofs))
        with pytest.raises(dd.DDError) as e:
            dd.dd_lopcg(es.ctx, x, inner, maxit_outer=3)
        assert e.value.code == dd.DD_EMAXIT
    _, x_o, k_o, its_o, _ = P.ground_state_lopcg(inner=inner, maxit_outer=3)
    assert k_o == 3
    assert rel_err(host(x), x_o) < (1e-9 if inner == "fused" else 1e-7)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("inner", ["fixed", "adaptive", "fused"])
@pytest.mark.parametrize("name", ["cfg1", "cfg2_small", "p2_small"])
def test_lopcg_mixed_reaches_ground_state(oracles, name, inner, prec):
    P, lam_ex = oracles[name]
    w = CASES[name]
    with make_solver(w, precision=prec) as es:
        es.prepare()
        x = gpu_vec(np.ones(w.dofs))
        lam, outer, tot, mx = dd.dd_lopcg(es.ctx, x, inner)
    assert abs(lam - lam_ex) <= 1e-10 * abs(lam_ex)
    assert _eta(P, host(x), lam) <= 1.5e-8


def test_lopcg_host_buffer_and_errors(oracles):
    P, lam_ex = oracles["cfg1"]
    w = CASES["cfg1"]
    with make_solver(w) as es:
        es.prepare()
        xh = np.ones(w.dofs)
        lam, outer, tot, mx = dd.dd_lopcg(es.ctx, xh, "fused")
        assert abs(lam - lam_ex) <= 1e-10 * abs(lam_ex)
        assert _eta(P, xh, lam) <= 1.5e-8
        with pytest.raises(dd.DDError) as e:
            dd.dd_lopcg(es.ctx, gpu_vec(np.ones(w.dofs)), 7)
        assert e.value.code == dd.DD_EINVAL
        with pytest.raises(dd.DDError) as e:
            dd.dd_lopcg(es.ctx, gpu_vec(np.ones(w.dofs)), "fused", maxit_outer=2)
        assert e.value.code == dd.DD_EMAXIT
        with pytest.raises(dd.DDError) as e:
            dd.dd_lopcg(es.ctx, gpu_vec(np.zeros(w.dofs)), "fused")
        assert e.value.code in (dd.DD_ENOTSPD, dd.DD_ENAN)
        # the context stays usable
        lam2, *_ = dd.dd_lopcg(es.ctx, gpu_vec(np.ones(w.dofs)), "adaptive")
        assert abs(lam2 - lam_ex) <= 1e-10 * abs(lam_ex)
