"""Batched ground states (dd_batch_*): many instances with uneven L and their own potentials
solved concurrently give, instance by instance, the exact ground state (oracle) and the very
same bits as the single-instance calls."""
import numpy as np
import pytest

import paper_2311_08757_gb300 as dd
from ddinputs import batch_workloads, sample_cell_qp
from oracle import solvers
from tests.gpu_util import gpu_vec, host, make_solver, oracle_problem

pytestmark = pytest.mark.gpu


def _batch(ws, precision="bf16"):
    import torch
    grids = [dd.grid_from_workload(w, precision=dd.PRECISIONS[precision]) for w in ws]
    Vs = [torch.from_numpy(sample_cell_qp(w)).cuda() for w in ws]
    return dd.Batch(grids, Vs)


@pytest.mark.parametrize("method", ["ipm", "lopcg_fused", "lopcg_adaptive"])
@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_small_batch_matches_oracle_and_single_calls(method, precision):
    ws = batch_workloads(seed=11, count=8, L_min=2, L_max=40, n=16, overlap=2)
    phis = [gpu_vec(np.zeros(w.dofs)) for w in ws]
    with _batch(ws, precision) as b:
        res = b.ground_states(method, threads=4, phi=phis)
        info = b.info()
    # the inverse iteration of the mixed form runs as batched kernels over all instances
    assert info["batchable"] == (precision == "bf16")
    assert info["last_batched"] == (precision == "bf16" and method in ("ipm", "lopcg_fused"))
    for i, w in enumerate(ws):
        P = oracle_problem(w, build_prec=False)
        lam_ex, _ = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma, dense_limit=3000 if w.dofs <= 3000 else 0)
        assert abs(res["lambda"][i] - lam_ex) <= 1e-10 * abs(lam_ex), (i, w.L)
        xh = host(phis[i])
        Mx = P.M @ xh
        assert np.linalg.norm(P.A @ xh - res["lambda"][i] * Mx) / (abs(lam_ex) * np.linalg.norm(Mx)) <= 1e-8 + 1e-12
        # the single-instance path gives the same bits
        with make_solver(w, precision=precision) as es:
            es.prepare()
            x = gpu_vec(np.ones(w.dofs))
            if method == "ipm":
                lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
            else:
                lam, outer, tot, mx = dd.dd_lopcg(es.ctx, x, method.split("_")[1])
        assert lam == res["lambda"][i] and outer == res["outer"][i] and tot == res["inner"][i]
        assert np.array_equal(host(x), xh)


def test_full_batched_workload():
    """The 64-instance workload (L log-uniform in [16, 2048], h = 1/32, delta = 4): every
    instance converges with residual eta <= 1e-8, the smallest ones match the oracle, and the
    largest ones match their single-instance solves bit for bit."""
    import torch
    ws = batch_workloads()
    order = np.argsort([w.L for w in ws])
    with _batch(ws) as b:
        res = b.ground_states("ipm")
        assert b.info()["last_batched"] == 1 and b.info()["gemm_tile_n"] in (128, 160, 256)
        for i, w in enumerate(ws):
            ctx = b.context(i)
            x = torch.ones(w.dofs, dtype=torch.float64, device="cuda")
            # eta of the returned pair from the instance's own operators
            lam, *_ = dd.dd_inverse_iterate(ctx, x)
            assert lam == res["lambda"][i]
            Ax = torch.empty_like(x)
            Mx = torch.empty_like(x)
            dd.dd_apply_operator(ctx, dd.DD_OP_A, x, Ax)
            dd.dd_apply_operator(ctx, dd.DD_OP_MASS, x, Mx)
            eta = float(torch.linalg.norm(Ax - lam * Mx) / (abs(lam) * torch.linalg.norm(Mx)))
            assert eta <= 1e-8 + 1e-12, (i, w.L)
    for i in order[:3]:
        w = ws[i]
        P = oracle_problem(w, build_prec=False)
        lam_ex, _ = solvers.exact_ground_state(P.A, P.M, sigma=P.sigma, dense_limit=0)
        assert abs(res["lambda"][i] - lam_ex) <= 1e-10 * abs(lam_ex)
    for i in order[-2:]:
        w = ws[i]
        with make_solver(w, precision="bf16") as es:
            es.prepare()
            x = gpu_vec(np.ones(w.dofs))
            lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
        assert lam == res["lambda"][i] and tot == res["inner"][i]


def test_batched_lopcg_equals_single_calls_on_the_full_workload():
    """Fused SI-LOPCG batched over the 64-instance workload: every instance's eigenvalue, step
    count and iterate equal those of its own dd_lopcg call (checked on the four largest and
    the four smallest instances), and the batched kernels ran."""
    ws = batch_workloads()
    order = np.argsort([w.L for w in ws])
    phis = [gpu_vec(np.zeros(w.dofs)) for w in ws]
    with _batch(ws) as b:
        res = b.ground_states("lopcg_fused", phi=phis)
        assert b.info()["last_batched"] == 1
    for i in list(order[:4]) + list(order[-4:]):
        w = ws[i]
        with make_solver(w, precision="bf16") as es:
            es.prepare()
            x = gpu_vec(np.ones(w.dofs))
            lam, outer, tot, mx = dd.dd_lopcg(es.ctx, x, "fused")
        assert lam == res["lambda"][i] and outer == res["outer"][i] and tot == res["inner"][i]
        assert np.array_equal(host(x), host(phis[i]))


def test_batched_kernels_equal_concurrent_pipelines():
    """The batched inverse iteration and fused SI-LOPCG (one launch per kernel over a group's
    instances, one graph per block of PCG iterations, instances joining as their set-up ends)
    give the same bits as the concurrent per-instance pipelines, instance by instance, for
    1, 2 and 4 groups, on a group's first call (built after every set-up) and on later calls
    (set-up and solves overlapping); the batched path launches fewer kernels."""
    ws = batch_workloads(seed=7, count=12, L_min=3, L_max=300, n=32, overlap=4)
    with _batch(ws) as b:
        ref = {}
        b.set_groups(-1)                       # every method per instance, concurrently
        for method in ("ipm", "lopcg_fused"):
            phis_c = [gpu_vec(np.zeros(w.dofs)) for w in ws]
            b.ground_states(method, phi=phis_c)   # warm-up (graphs, workspaces)
            l0 = dd.dd_kernel_launch_count()
            rc = b.ground_states(method, phi=phis_c)
            lc = dd.dd_kernel_launch_count() - l0
            assert b.info()["last_batched"] == 0
            ref[method] = (rc, [host(p) for p in phis_c], lc)
        for groups in (1, 2, 4):
            b.set_groups(groups)
            for method in ("ipm", "lopcg_fused"):
                rc, pc, lc = ref[method]
                for call in range(2):
                    phis = [gpu_vec(np.zeros(w.dofs)) for w in ws]
                    l0 = dd.dd_kernel_launch_count()
                    res = b.ground_states(method, phi=phis)
                    la = dd.dd_kernel_launch_count() - l0
                    info = b.info()
                    assert info["last_batched"] == 1 and info["groups"] == groups
                    assert np.array_equal(res["lambda"], rc["lambda"]), (groups, method, call)
                    assert np.array_equal(res["outer"], rc["outer"]) and np.array_equal(res["inner"], rc["inner"])
                    for a, c in zip(phis, pc):
                        assert np.array_equal(host(a), c)
                    assert la < lc


@pytest.mark.parametrize("fuse,pairs", [(1, 1), (0, 0)])
def test_batched_kernels_with_options_equal_single_calls(fuse, pairs):
    """The batched kernels follow each instance's options (here the x/r update fused into the
    packing, or the FP64 form of the fused pass): set on every instance's context, the
    batched inverse iteration still gives each instance's single-call bits."""
    ws = batch_workloads(seed=13, count=6, L_min=2, L_max=30, n=16, overlap=2)
    phis = [gpu_vec(np.zeros(w.dofs)) for w in ws]
    with _batch(ws) as b:
        for i in range(len(ws)):
            dd.dd_set_option(b.context(i), dd.DD_OPT_PAIRS, pairs)
            dd.dd_set_option(b.context(i), dd.DD_OPT_FUSE_XR, fuse)
        res = b.ground_states("ipm", threads=3, phi=phis)
        assert b.info()["last_batched"] == 1
    for i, w in enumerate(ws):
        with make_solver(w, precision="bf16") as es:
            es.prepare()
            dd.dd_set_option(es.ctx, dd.DD_OPT_PAIRS, pairs)
            dd.dd_set_option(es.ctx, dd.DD_OPT_FUSE_XR, fuse)
            x = gpu_vec(np.ones(w.dofs))
            lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
        assert lam == res["lambda"][i] and outer == res["outer"][i] and tot == res["inner"][i]
        assert np.array_equal(host(x), host(phis[i]))
