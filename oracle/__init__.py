"""Plain, slow FP64 CPU oracle for the two-level Schwarz eigensolver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The CUDA library never calls it and shares no code with it.

It restates, in numpy/scipy, what the method of Theisen & Stamm
(arXiv 2311.08757) computes:

* ``q1``      Q1 finite elements on (0,L)^p x (0,ell): K, M, M_V (Sec. 2,
              discrete weak form) and the x-periodic cell operator (Sec. 2,
              weak cell problem).
* ``dd``      one overlapping subdomain per unit cell, partitions of unity,
              the PerFact coarse space R_0^T = blockdiag(D_i R_i psi)
              (Definition 2.1) and the two-level additive Schwarz
              preconditioner M_AS2^{-1} (Sec. 3.1).
* ``solvers`` preconditioned CG (Sec. 4.1 stopping rule), shifted inverse
              iteration (Sec. 2), the cell eigenpair and the exact ground
              state used as the plain definition of the result.

Pins (checked by the CPU tests, not by re-running this code): the closed-form
Q1 spectrum for V = 0, spectral shift by constant V, dense brute force on tiny
grids, Simpson-rule integrals of separable V, symmetry and partition-of-unity
identities, the exact-inverse special case L = 1 and the L-robust iteration
counts of Sec. 4.1.  The printed cell shift of Sec. 4.1 (sigma ~ 19.32644) is
not reproduced by the printed potential and stays parity unpinned.
"""
