"""The prolong-sum of a p = 1 box computes each node's owners and their packed rows in closed
form (subdomain i spans columns max(1, i n - delta + 1) .. min(Ln - 1, (i+1) n + delta - 1) and
is packed row i) instead of reading them from index tables; set-up checks the formula against
the tables.  Both ways give the same bits: the preconditioner, and the ground state."""
import numpy as np
import pytest

import paper_2311_08757_gb300 as dd
from ddinputs import WORKLOADS, Workload
from tests.gpu_util import gpu_vec, host, make_solver

pytestmark = pytest.mark.gpu

CASES = {
    "L1": Workload("L1", p=1, L=1, n=8, overlap=2, kind="cos1"),
    "L2": Workload("L2", p=1, L=2, n=8, overlap=3, kind="cos1"),
    "L3": Workload("L3", p=1, L=3, n=10, overlap=1, kind="cos4", seed=3),
    "cfg2_small": WORKLOADS["cfg2_small"],
}


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_closed_form_owners_equal_tables(name, prec):
    w = CASES[name]
    r = gpu_vec(np.random.default_rng(31).standard_normal(w.dofs))
    out = {}
    for tables in (0, 1):
        with make_solver(w, precision=prec) as es:
            es.prepare()
            dd.dd_set_option(es.ctx, dd.DD_OPT_PROLONG_TABLES, tables)
            z = gpu_vec(np.zeros(w.dofs))
            dd.dd_apply_preconditioner(es.ctx, r, z)
            x = gpu_vec(np.ones(w.dofs))
            lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
            out[tables] = (host(z), lam, tot, host(x))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]
    assert np.array_equal(out[0][3], out[1][3])
