"""Potential gradients through the C ABI (dd_potential_gradient) and the torch.autograd
wrapper: parity with the oracle's Hellmann-Feynman reduction and adjoint solve, and central
finite differences of GPU eigen-solves on the differentiable workload (8 cosine modes,
theta ~ N(0, 25), loss ||phi - phi_target||_M^2)."""
import numpy as np
import pytest

import paper_2311_08757_gb300 as dd
from ddinputs import WORKLOADS, Workload, theta_seed, theta8_qp_basis, sample_cell_qp
from oracle import grad, solvers
from tests.gpu_util import gpu_vec, host, make_solver, oracle_problem, rel_err

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_res=1e-11, tol_lam=1e-14, rtol_inner=1e-12)


def _oracle_state(w):
    P = oracle_problem(w, build_prec=False)
    lam, phi = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma, dense_limit=3000 if w.dofs <= 3000 else 0)
    return P, lam, phi


@pytest.mark.parametrize("name", ["cfg5_small", "p2"])
@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_gradient_matches_oracle(name, prec):
    w = WORKLOADS[name] if name in WORKLOADS else Workload("p2", p=2, L=3, n=6, overlap=2, kind="asym3")
    P, lam, phi = _oracle_state(w)
    th, tt = theta_seed(5)
    if w.kind == "theta8":
        _, _, phi_t = _oracle_state(w.with_(params={"theta": tt}))
    else:
        phi_t = np.random.default_rng(4).standard_normal(w.dofs) * 0.01 + phi
    gphi = 2.0 * (P.M @ (phi - phi_t))
    ref_lam = grad.eigenvalue_gradient(P.g, phi)
    ref_l = grad.loss_gradient(P.g, P.A, P.M, lam, phi, gphi, sigma=P.sigma)
    with make_solver(w, precision=prec) as es:
        es.prepare()
        nV = ref_lam.size
        dV = gpu_vec(np.zeros(nV))
        it = dd.dd_potential_gradient(es.ctx, gpu_vec(phi), lam, 1.0, None, dV)
        assert it == 0
        assert rel_err(host(dV), ref_lam) < 1e-12
        dV2 = np.zeros(nV)                      # host output buffer
        it = dd.dd_potential_gradient(es.ctx, phi, lam, 0.0, gphi, dV2, rtol=1e-11)
        assert it > 0
        assert rel_err(dV2, ref_l) < 1e-8
        # both terms at once: linear in (g_lambda, g_phi)
        dV3 = gpu_vec(np.zeros(nV))
        dd.dd_potential_gradient(es.ctx, gpu_vec(phi), lam, 2.5, gpu_vec(gphi), dV3, rtol=1e-11)
        assert rel_err(host(dV3), 2.5 * ref_lam + ref_l) < 1e-8


def test_gradient_full_size_oracle_and_finite_differences():
    """The differentiable workload at full size (L = 256, h = 1/32, 253,921 unknowns):
    torch.autograd through the library against the oracle gradient, and against central
    differences of FP64 GPU eigen-solves (tolerances tightened so that the eigenvalue
    noise stays far below the step's signal)."""
    import torch
    from paper_2311_08757_gb300.autograd import ground_state, mass
    w = WORKLOADS["cfg5"]
    th, tt = theta_seed(w.seed)
    B = torch.from_numpy(theta8_qp_basis(w)).cuda()
    V0 = torch.from_numpy(sample_cell_qp(w)).cuda()
    with make_solver(w) as es:
        lam_t, phi_t = ground_state(torch.from_numpy(tt).cuda() @ B, es, **TIGHT)
        phi_t = phi_t.detach()

        def objective(theta, grad_on=True):
            V = theta @ B
            lam, phi = ground_state(V, es, **TIGHT)
            e = phi - phi_t
            return lam, (e * mass(e, es)).sum()

        theta = torch.from_numpy(th).cuda().requires_grad_(True)
        lam, loss = objective(theta)
        g_lam, = torch.autograd.grad(lam, theta, retain_graph=True)
        g_loss, = torch.autograd.grad(loss, theta)
        assert torch.allclose(theta.detach() @ B, V0, rtol=0, atol=1e-12)
        # oracle gradient at full size
        P, lam_o, phi_o = _oracle_state(w)
        assert abs(lam.item() - lam_o) <= 1e-10 * abs(lam_o)
        _, _, phi_to = _oracle_state(w.with_(params={"theta": tt}))
        Bn = B.cpu().numpy()
        ref_lam = Bn @ grad.eigenvalue_gradient(P.g, phi_o)
        ref_loss = Bn @ grad.loss_gradient(P.g, P.A, P.M, lam_o, phi_o, 2.0 * (P.M @ (phi_o - phi_to)), sigma=P.sigma)
        assert rel_err(g_lam.cpu().numpy(), ref_lam) < 1e-8
        assert rel_err(g_loss.cpu().numpy(), ref_loss) < 1e-6
        # Richardson-extrapolated central differences (steps 2e-4 and 1e-4; the eigenvalue's
        # rounding floor, ~1e-13 relative, would dominate a 1e-6 step: see the design notes),
        # agreement measured on the gradient vector: max_j |fd_j - g_j| / max_j |g_j| <= 1e-6
        def central(j, eps):
            tp = theta.detach().clone()
            tm = theta.detach().clone()
            tp[j] += eps
            tm[j] -= eps
            with torch.no_grad():
                lp, fp = objective(tp)
                lm, fm = objective(tm)
            return (lp - lm).item() / (2 * eps), (fp - fm).item() / (2 * eps)

        fd = np.array([[(4 * a1 - a2) / 3 for a1, a2 in zip(central(j, 1e-4), central(j, 2e-4))]
                       for j in range(8)])
        gl, gf = g_lam.cpu().numpy(), g_loss.cpu().numpy()
        err_lam = np.abs(fd[:, 0] - gl).max() / np.abs(gl).max()
        err_loss = np.abs(fd[:, 1] - gf).max() / np.abs(gf).max()
        print(f"finite differences: lambda {err_lam:.2e}, loss {err_loss:.2e}")
        assert err_lam <= 1e-6
        assert err_loss <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_gradient_from_gpu_ground_state_default_tolerances(prec):
    """The backward pass straight after a ground state at the default tolerances (eta <= 1e-8):
    lambda carries the eigen-solve's error, so A - lambda M is slightly indefinite along phi;
    the projected adjoint PCG still converges, and the gradient agrees with the oracle's to
    the accuracy of the eigenvector itself."""
    w = WORKLOADS["cfg5_small"]
    P, lam_o, phi_o = _oracle_state(w)
    th, tt = theta_seed(5)
    _, _, phi_t = _oracle_state(w.with_(params={"theta": tt}))
    ref = grad.eigenvalue_gradient(P.g, phi_o) + grad.loss_gradient(
        P.g, P.A, P.M, lam_o, phi_o, 2.0 * (P.M @ (phi_o - phi_t)), sigma=P.sigma)
    with make_solver(w, precision=prec) as es:
        es.prepare()
        x = gpu_vec(np.ones(w.dofs))
        lam, *_ = dd.dd_inverse_iterate(es.ctx, x)
        g = gpu_vec(2.0 * (P.M @ (host(x) - phi_t)))
        dV = gpu_vec(np.zeros(ref.size))
        it = dd.dd_potential_gradient(es.ctx, x, lam, 1.0, g, dV)
        assert 0 < it < 200
        assert rel_err(host(dV), ref) < 1e-5
