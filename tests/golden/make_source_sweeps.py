"""Writes source_sweeps.json: CG iteration counts of the oracle on the source problem of
Sec. 4.1 and inner PCG counts of its inverse iteration, the reference for the GPU sweeps.

* Fig. 3 (Sec. 4.1.1): a_sigma(u, v) = (1, v) on (0, L) x (0, 1), the printed potential
  V = 10^2 (sin^2 pi x)^2 (sin^2 pi y)^2, h = 1/30, delta = 1, N = L subdomains, CG from the
  initial guess 1 to ||r_k|| <= 1e-8 ||r_0||, one-level M_AS1 and two-level M_AS2 (equal
  weights), L = 2 ... 256.
* Table 1 (Sec. 4.1.2): the same problem with the distance partition of unity for
  h in {1/10, 1/20, 1/30} and delta in {1, 2, 3} (the table's L values are not in the text;
  4, 16 and 64 here).
* Inverse iteration (Sec. 2) on the 4-term cosine potential of the headline workload
  (h = 1/32, delta = 4, seed 2311) for L = 2, 8, 32: outer steps and inner PCG iterations.

Only the oracle is called.  About a minute on one core (one BLAS thread):
    OMP_NUM_THREADS=1 python tests/golden/make_source_sweeps.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from ddinputs import WORKLOADS, Workload, potential  # noqa: E402
from oracle import q1, solvers  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "source_sweeps.json")


def source_count(L, n, delta, coarse, pu, near=False):
    """CG iterations to ||r_k|| <= 1e-8 ||r_0||; with near=True also the first iteration at
    which ||r_k|| <= 3e-8 ||r_0||: CG residual norms can hover within a factor of 3 of the
    threshold for several iterations, and there rounding alone (even the BLAS thread count of
    the dense coarse factorisation) moves the first crossing."""
    w = Workload("e1", p=1, L=L, n=n, overlap=delta, kind="sin4")
    g = q1.Grid.from_workload(w)
    P = solvers.Problem(g, potential(w), pu=pu, coarse=coarse)
    b = np.full(g.ndof, g.h ** 2)        # (f, v_h) for f = 1: the integral of each Q1 hat function
    _, it, hist = P.solve(b, x0=np.ones(g.ndof), history=True)
    if not near:
        return int(it)
    return int(it), int(next(k for k, h in enumerate(hist) if h <= 3e-8))


def main():
    out = {"citation": "Sec. 4.1 (Fig. 3 and Table 1: CG iteration counts, rTOL = 1e-8, initial guess 1) and "
                       "Sec. 2 (inverse iteration); written by tests/golden/make_source_sweeps.py from the oracle alone",
           "near_stop": "as1_near / as2_near: first iteration with ||r_k|| <= 3e-8 ||r_0||",
           "fig3": {"n": 30, "delta": 1, "pu": "equal", "L": [], "as1": [], "as2": [], "as1_near": [],
                    "as2_near": []},
           "table1": {"pu": "distance", "L": [4, 16, 64], "cases": []},
           "eigen": {"workload": "cfg2 potential", "n": 32, "delta": 4, "L": [], "outer": [], "inner_total": [],
                     "inner_max": []}}
    for L in (2, 4, 8, 16, 32, 64, 128, 256):
        out["fig3"]["L"].append(L)
        for key, coarse in (("as1", False), ("as2", True)):
            it, near = source_count(L, 30, 1, coarse, "equal", near=True)
            out["fig3"][key].append(it)
            out["fig3"][key + "_near"].append(near)
        print("fig3", L, out["fig3"]["as1"][-1], out["fig3"]["as2"][-1], flush=True)
    for n in (10, 20, 30):
        for delta in (1, 2, 3):
            row = {"n": n, "delta": delta, "as1": [], "as2": [], "as1_near": [], "as2_near": []}
            for L in out["table1"]["L"]:
                for key, coarse in (("as1", False), ("as2", True)):
                    it, near = source_count(L, n, delta, coarse, "distance", near=True)
                    row[key].append(it)
                    row[key + "_near"].append(near)
            out["table1"]["cases"].append(row)
            print("table1", n, delta, row["as1"], row["as2"], flush=True)
    base = WORKLOADS["cfg2"]
    for L in (2, 8, 32):
        w = base.with_(name=f"cfg2_l{L}", L=L)
        g = q1.Grid.from_workload(w)
        P = solvers.Problem(g, potential(w))
        lam, x, k, inner, info = P.ground_state()
        out["eigen"]["L"].append(L)
        out["eigen"]["outer"].append(int(k))
        out["eigen"]["inner_total"].append(int(np.sum(inner)))
        out["eigen"]["inner_max"].append(int(np.max(inner)))
        print("eigen", L, k, inner, flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
