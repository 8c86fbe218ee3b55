"""The PCG solution update deferred to the next p update (DD_OPT_X_LAG, on by default).

With the option the x/r update only forms r - alpha q and (r, r); iteration k + 1's p update,
which reads p_k anyway, applies x += alpha_k p_k to the nodes it owns, and one kernel applies
the last iteration's update after the loop.  Every entry of x receives the same FMAs on the
same operands in the same order as when the x/r update makes them, so solutions, iteration
counts, eigenvalues and eigenvectors must be bit-identical with the option on and off, on
every path of the iteration: the fused p = 1 pass (float pairs and FP64), the two-kernel p
update, the p = 2 passes, CUDA graphs or eager launches, a solve stopped by maxit, and the
outer inverse iteration built on these solves."""
import numpy as np
import pytest

import paper_2311_08757_gb300 as dd
from ddinputs import WORKLOADS, Workload
from tests.gpu_util import gpu_vec, host, make_solver

pytestmark = pytest.mark.gpu

CASES = {
    "cfg1": WORKLOADS["cfg1"],
    "cfg2_small": WORKLOADS["cfg2_small"],
    "ragged": Workload("ragged", p=1, L=5, n=10, ell=1.2, overlap=3, kind="cos4", seed=7),
    "L1": Workload("L1", p=1, L=1, n=8, overlap=2, kind="cos1"),
    "p2": Workload("p2", p=2, L=3, n=6, overlap=2, kind="asym3"),
}

# (precision, extra options): the default pass of each precision, FP64 matvec with rounded
# inverses, the two-kernel p update, eager launches
VARIANTS = [
    ("bf16", {}),
    ("fp64", {}),
    ("bf16", {dd.DD_OPT_PAIRS: 0}),
    ("tf32", {dd.DD_OPT_FUSED_PQ: 0}),
    ("bf16", {dd.DD_OPT_USE_GRAPH: 0}),
]


def _run(w, prec, opts, lag, maxit=10000, rtol=1e-8):
    with make_solver(w, precision=prec) as es:
        es.prepare()
        for k, v in opts.items():
            if k == dd.DD_OPT_FUSED_PQ and w.p == 2:
                continue
            dd.dd_set_option(es.ctx, k, v)
        dd.dd_set_option(es.ctx, dd.DD_OPT_X_LAG, lag)
        b = gpu_vec(np.zeros(w.dofs))
        dd.dd_apply_operator(es.ctx, dd.DD_OP_MASS, gpu_vec(np.ones(w.dofs)), b)
        y = gpu_vec(np.zeros(w.dofs))
        it, rel = dd.dd_pcg_solve(es.ctx, b, y, rtol, maxit, allow_maxit=True)
        y2 = gpu_vec(np.linspace(-1.0, 1.0, w.dofs))   # a nonzero initial guess
        it2, rel2 = dd.dd_pcg_solve(es.ctx, b, y2, rtol, maxit, allow_maxit=True)
        x = gpu_vec(np.ones(w.dofs))
        lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
        return (it, rel, host(y), it2, rel2, host(y2), lam, outer, tot, host(x))


@pytest.mark.parametrize("variant", range(len(VARIANTS)))
@pytest.mark.parametrize("name", list(CASES))
def test_deferred_x_update_is_bit_identical(name, variant):
    w = CASES[name]
    prec, opts = VARIANTS[variant]
    on = _run(w, prec, opts, 1)
    off = _run(w, prec, opts, 0)
    it, rel, y, it2, rel2, y2, lam, outer, tot, x = on
    print(f"{name} {prec} {opts}: PCG {it} / {it2}, inner total {tot}, lambda {lam!r}")
    assert rel <= 1e-8 and rel2 <= 1e-8
    for a, b in zip(on, off):
        if isinstance(a, np.ndarray):
            assert np.array_equal(a, b)
        else:
            assert a == b


@pytest.mark.parametrize("name", ["cfg1", "p2"])
def test_deferred_x_update_at_maxit(name):
    """A solve stopped by maxit returns the same iterate (the final update also runs then)."""
    w = CASES[name]
    for maxit in (1, 2, 5):
        on = _run(w, "bf16", {}, 1, maxit=maxit)
        off = _run(w, "bf16", {}, 0, maxit=maxit)
        assert on[0] == off[0] == maxit
        assert np.array_equal(on[2], off[2]) and np.array_equal(on[5], off[5])
        assert np.any(on[2] != 0.0)


def test_x_lag_option_validation():
    with make_solver(CASES["cfg1"], precision="bf16") as es:
        for bad in (-1, 2):
            with pytest.raises(dd.DDError):
                dd.dd_set_option(es.ctx, dd.DD_OPT_X_LAG, bad)
