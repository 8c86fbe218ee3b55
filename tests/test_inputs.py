"""The seeded input generators: the workload sizes of the hot-path scope table, the
periodicity every potential must have (assumption A1 of Sec. 1), the draw order of the
random coefficients, and the sample layout that dd_setup reads."""
import numpy as np
import pytest

from ddinputs import WORKLOADS, Workload, batch_workloads, potential, sample_cell_qp, theta_seed


def test_workload_sizes():
    # interior unknowns (L n - 1)^p (n_y - 1) and subdomains L^p
    assert WORKLOADS["cfg1"].dofs == 127 * 15 == 1905
    assert WORKLOADS["cfg2"].dofs == 65535 * 31 == 2_031_585
    assert WORKLOADS["cfg3"].dofs == 1023 ** 2 * 15 == 15_697_935
    assert WORKLOADS["cfg2"].L ** WORKLOADS["cfg2"].p == 2048
    assert WORKLOADS["cfg3"].L ** WORKLOADS["cfg3"].p == 4096


@pytest.mark.parametrize("name", ["cfg1", "cfg2", "cfg3", "e1", "cfg5"])
def test_potentials_are_one_periodic(name):
    w = WORKLOADS[name]
    V = potential(w)
    rng = np.random.default_rng(1)
    y = rng.uniform(0, w.ell, 200)
    if w.p == 1:
        x = rng.uniform(0, 1, 200)
        for k in (1, 3, -2):
            assert np.allclose(V(x + k, y), V(x, y), rtol=1e-12, atol=1e-12)
    else:
        x1, x2 = rng.uniform(0, 1, 200), rng.uniform(0, 1, 200)
        base = V(x1, x2, y)
        for k1, k2 in ((1, 0), (0, 1), (2, -3)):
            assert np.allclose(V(x1 + k1, x2 + k2, y), base, rtol=1e-12, atol=1e-12)


def test_cosine_coefficients_draw_order():
    rng = np.random.default_rng(2311)
    a = rng.uniform(0.0, 20.0, 4)
    b = rng.uniform(-0.5, 0.5, 4)
    V = potential(WORKLOADS["cfg2"])
    x, y = np.array([0.0]), np.array([0.25])
    assert V(x, y)[0] == pytest.approx(float(np.sum(a * (1 + b * 0.25))), rel=1e-14)


def test_wells_lattice_symmetry_and_sign():
    V = potential(WORKLOADS["cfg3"])
    rng = np.random.default_rng(2)
    x1, x2, y = rng.uniform(0, 1, 100), rng.uniform(0, 1, 100), rng.uniform(0, 1, 100)
    v = V(x1, x2, y)
    assert np.all(v < 0)
    assert np.allclose(V(x2, x1, y), v, rtol=1e-12)          # the lattice is symmetric in x1, x2
    assert np.allclose(V(1 - x1, x2, y), v, rtol=1e-12)      # and under x1 -> 1 - x1
    # deepest at the well centre (1/2, 1/2); the (1 + y) factor scales it
    c = V(np.array([0.5]), np.array([0.5]), np.array([0.0]))[0]
    assert c < V(np.array([0.0]), np.array([0.0]), np.array([0.0]))[0]
    assert V(np.array([0.5]), np.array([0.5]), np.array([1.0]))[0] == pytest.approx(2 * c, rel=1e-14)


@pytest.mark.parametrize("name", ["cfg1", "cfg3_small"])
def test_sample_layout_and_size(name):
    w = WORKLOADS[name]
    s = sample_cell_qp(w)
    assert s.dtype == np.float64 and s.flags["C_CONTIGUOUS"]
    assert s.size == w.ny * w.n ** w.p * w.quad_pts ** (w.p + 1)
    # element-major, y element fastest, then the points with qy fastest: the first Q^d values
    # are element 0's points, the next Q^d are the element above it (ey = 1)
    V = potential(w)
    h, Q = 1.0 / w.n, w.quad_pts
    xi = 0.5 * (np.polynomial.legendre.leggauss(Q)[0] + 1.0)
    npt = Q ** (w.p + 1)
    if w.p == 1:
        want0 = [V(np.array([xi[qx] * h]), np.array([xi[qy] * h]))[0] for qx in range(Q) for qy in range(Q)]
        want1 = [V(np.array([xi[qx] * h]), np.array([(1 + xi[qy]) * h]))[0] for qx in range(Q) for qy in range(Q)]
    else:
        want0 = [V(np.array([xi[a] * h]), np.array([xi[b] * h]), np.array([xi[c] * h]))[0]
                 for a in range(Q) for b in range(Q) for c in range(Q)]
        want1 = [V(np.array([xi[a] * h]), np.array([xi[b] * h]), np.array([(1 + xi[c]) * h]))[0]
                 for a in range(Q) for b in range(Q) for c in range(Q)]
    assert np.allclose(s[:npt], want0, rtol=1e-14)
    assert np.allclose(s[npt:2 * npt], want1, rtol=1e-14)


def test_generators_are_deterministic():
    w = WORKLOADS["cfg2_small"]
    assert np.array_equal(sample_cell_qp(w), sample_cell_qp(w))
    b1, b2 = batch_workloads(), batch_workloads()
    assert [x.L for x in b1] == [x.L for x in b2]
    assert all(x.params == y.params for x, y in zip(b1, b2))
    assert len(b1) == 64 and all(16 <= x.L <= 2048 for x in b1)
    th, tt = theta_seed(5)
    rng = np.random.default_rng(5)
    th2 = rng.normal(0.0, 5.0, 8)
    assert np.array_equal(th, th2) and np.array_equal(tt, th2 + rng.normal(0.0, 1.0, 8))


def test_workload_rejects_non_integer_cell_height():
    with pytest.raises(ValueError):
        Workload("bad", p=1, L=2, n=16, ell=1.03).ny
