"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle.

This module holds no arithmetic of the eigensolver.  It only describes the
workloads (grid sizes, overlap, quadrature order) and the potentials V as
closed-form callables, and samples a callable at Gauss-Legendre points of the
unit cell -- the input format of ``dd_setup``.

The potentials follow the periodic, bounded class the paper assumes
(Sec. 1, assumptions A1-A2: V is 1-periodic in every expanding coordinate and
essentially bounded).  Their concrete forms are synthetic stand-ins for the
paper's examples (Sec. 4.1 uses V = 100 sin^4(pi x) sin^4(pi y)); the paper
uses no dataset.
"""
from .potentials import (  # noqa: F401
    Workload, WORKLOADS, potential, sample_cell_qp, gauss_legendre_01, theta_seed, theta8_basis,
    theta8_qp_basis, batch_workloads,
)
