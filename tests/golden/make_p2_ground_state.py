"""Writes p2_ground_state.json: the exact discrete ground state of the d = 3 Gaussian-well
workload on a 6 x 6-cell box, from the oracle alone.

The box is the d = 3 workload (p = 2, h = 1/16, delta = 2, V = -30 (1 + y) sum over the well
lattice) shrunk to L = 6: 95 x 95 x 15 = 135,375 unknowns and 36 subdomains, of which 16 are
interior, 16 edge and 4 corner subdomains, so every local-matrix type of the full workload
occurs more than once.  The value is the plain definition of the result (Sec. 2, discrete weak
form): the lowest eigenpair of (K + M_V) x = lambda M x, here by inverse iteration with an exact
banded Cholesky factor of A_sigma, converged until the Rayleigh quotient is stationary to
1e-15.  About 30 s on one core:  python tests/golden/make_p2_ground_state.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from ddinputs import WORKLOADS, potential  # noqa: E402
from oracle import q1, solvers  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "p2_ground_state.json")


def main():
    w = WORKLOADS["cfg3"].with_(name="cfg3_l6", L=6)
    g = q1.Grid.from_workload(w)
    P = solvers.Problem(g, potential(w), build_prec=False)
    lam, x = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma, dense_limit=0)
    r = P.A @ x - lam * (P.M @ x)
    eta = float((r @ r) ** 0.5 / (abs(lam) * float((P.M @ x) @ (P.M @ x)) ** 0.5))
    out = {"citation": "Sec. 2 (discrete weak form): lowest eigenpair of the Q1 pencil (K + M_V, M); written by "
                       "tests/golden/make_p2_ground_state.py from the oracle alone",
           "workload": {"p": 2, "L": 6, "n": 16, "ell": 1.0, "overlap": 2, "quad_pts": 2, "kind": "wells",
                        "dofs": int(w.dofs)},
           "sigma": float(P.sigma), "lambda1": float(lam), "eta": eta}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
