"""Programmatic dependent launch of the PCG chain (DD_OPT_PDL): the kernels wait for their
predecessor's results before reading anything, so launching them early changes no bit of the
iterates: the same eigenpair, iteration counts and solution with the option on and off, in
the FP64 and the mixed forms, with and without CUDA graphs."""
import numpy as np
import pytest

import paper_2311_08757_gb300 as dd
from ddinputs import WORKLOADS, Workload
from tests.gpu_util import gpu_vec, host, make_solver

pytestmark = pytest.mark.gpu

CASES = {
    "cfg1": WORKLOADS["cfg1"],
    "cfg2_small": WORKLOADS["cfg2_small"],
    "p2": Workload("p2", p=2, L=3, n=6, overlap=2, kind="asym3"),
}


@pytest.mark.parametrize("graph", [1, 0])
@pytest.mark.parametrize("prec", ["bf16", "fp64"])
@pytest.mark.parametrize("name", list(CASES))
def test_pdl_same_bits(name, prec, graph):
    w = CASES[name]
    out = {}
    for pdl in (0, 1):
        with make_solver(w, precision=prec) as es:
            es.prepare()
            dd.dd_set_option(es.ctx, dd.DD_OPT_PDL, pdl)
            dd.dd_set_option(es.ctx, dd.DD_OPT_USE_GRAPH, graph)
            x = gpu_vec(np.ones(w.dofs))
            lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
            b = gpu_vec(np.zeros(w.dofs))
            dd.dd_apply_operator(es.ctx, dd.DD_OP_MASS, gpu_vec(np.ones(w.dofs)), b)
            y = gpu_vec(np.zeros(w.dofs))
            it, rel = dd.dd_pcg_solve(es.ctx, b, y, 1e-8)
            out[pdl] = (lam, outer, tot, host(x), it, rel, host(y))
    a, b = out[0], out[1]
    assert a[0] == b[0] and a[1:3] == b[1:3] and a[4:6] == b[4:6]
    assert np.array_equal(a[3], b[3]) and np.array_equal(a[6], b[6])


def test_pdl_option_validation():
    with make_solver(CASES["cfg1"]) as es:
        for bad in (-1, 2):
            with pytest.raises(dd.DDError):
                dd.dd_set_option(es.ctx, dd.DD_OPT_PDL, bad)
