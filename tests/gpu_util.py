"""Helpers of the GPU parity tests: run the CUDA path through the C ABI binding and
the oracle on the same seeded inputs."""
import numpy as np

import paper_2311_08757_gb300 as dd
from ddinputs import Workload, potential, sample_cell_qp
from oracle import q1, solvers


def torch_dev():
    import torch
    return torch.device("cuda:0")


def gpu_vec(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")


def host(t):
    return t.detach().cpu().numpy()


def make_solver(w: Workload, precision="fp64", coarse=1, pu="equal"):
    import torch
    V = torch.from_numpy(sample_cell_qp(w)).to("cuda:0")
    grid = dd.grid_from_workload(w, precision=dd.PRECISIONS[precision], coarse=coarse,
                                 pu_kind=dd.DD_PU_EQUAL if pu == "equal" else dd.DD_PU_DISTANCE)
    return dd.Eigensolver(grid, V)


def oracle_problem(w: Workload, coarse=True, pu="equal", build_prec=True):
    g = q1.Grid.from_workload(w)
    return solvers.Problem(g, potential(w), pu=pu, coarse=coarse, build_prec=build_prec)


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def sigma_tol(P):
    """Tolerance on the cell shift sigma.  In FP64 the smallest eigenvalue of the cell pencil
    is fixed only to about eps * lambda_max absolutely (the rounding of A psi, whose entries
    are of size lambda_max |psi|, against sigma M psi), by any method: the dense solver of
    the oracle and the inverse iteration of the GPU each land within a few such units."""
    import scipy.sparse.linalg as spla
    K, M, MV = q1.assemble_cell(P.g, P.V)
    lmax = float(spla.eigsh((K + MV).tocsc(), k=1, M=M.tocsc(), which="LA", return_eigenvectors=False)[0])
    return max(1e-12 * max(1.0, abs(P.sigma)), 8 * np.finfo(float).eps * lmax)
