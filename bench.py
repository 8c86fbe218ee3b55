#!/usr/bin/env python3
"""Time to the ground state on the periodic-potential box L = 2048, h = 1/32, delta = 4.

One step = everything that depends on the potential, on one GPU: upload V (already in
HBM) and rebuild the stencil tables, the cell eigenpair (sigma, psi), the local
factorisations / rounded local inverses and the coarse matrix, and the shifted inverse
iteration from x_0 = 1 to the stopping rule (eta <= 1e-8, relative change of the
Rayleigh quotient <= 1e-10), with every inner PCG solve at rTOL = 1e-8.  The context
(device buffers) is allocated once before the timed region.

Printed: one JSON line.  ``value`` is ground states per second of the whole job
(mixed precision: BF16 local inverses on the tensor cores inside flexible CG; the
plain FP64 method is timed beside it); ``e2e`` repeats the measurement through
``dd_eigenpair`` with host buffers (V in, phi out) and context set-up inside the timed
region; ``roofline`` is for the kernel class with the largest device time;
``cpu_baseline`` is the oracle on the host cores on a bounded sample.

``--impl reference`` times the oracle itself (the reference arm of this workload).
For N > 1 GPUs the ranks run independent replicas of the workload (the method has no
data exchange between independent eigenproblems); ``value`` counts all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time to ground state @1e-10 rel, mixed vs FP64 plain; PCG iters/s; % roofline"
UNIT = "ground states/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# FP64 FMA throughput measured on this machine's GB300 with a DFMA microbenchmark
# (8 independent chains per thread, 152 x 8 x 256 threads): 1.19 TFLOP/s.
FP64_TFLOPS = 1.19


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg2")
    ap.add_argument("--precision", default="bf16", choices=["bf16", "tf32"])
    ap.add_argument("--fp64-steps", type=int, default=None, help="timed steps of the plain FP64 method")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-lopcg", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--coarse-solve", default="auto", choices=["auto", "cr", "dense"])
    ap.add_argument("--cpu-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--setup-only", default=None, choices=["cfg2", "cfg3"],
                    help="time only the set-up stages (cell eigenpair, coarse build) of one workload")
    return ap.parse_args()


# ----------------------------------------------------------------------------------------
# oracle sample (runs in a child process with one BLAS thread)
# ----------------------------------------------------------------------------------------
def cpu_sample(workload: str, pcg_its: int = 3) -> dict:
    import numpy as np
    from ddinputs import WORKLOADS, potential
    from oracle import q1, solvers
    from oracle.dd import Decomposition, TwoLevelAS
    w = WORKLOADS[workload]
    g = q1.Grid.from_workload(w)
    V = potential(w)
    t0 = time.perf_counter()
    K, M, MV = q1.assemble_box(g, V)
    A = (K + MV).tocsr()
    sigma, psi = solvers.cell_eigenpair(g, V)
    As = (A - sigma * M).tocsr()
    P = TwoLevelAS(As, Decomposition(g), q1.periodic_extension(g, psi))
    t1 = time.perf_counter()
    x = np.ones(g.ndof)
    x /= np.sqrt(x @ (M @ x))
    b = M @ x
    t2 = time.perf_counter()
    _, it, _ = solvers.pcg(As, b, None, P, 1e-8, pcg_its)
    t3 = time.perf_counter()
    return {"setup_s": t1 - t0, "pcg_s_per_iter": (t3 - t2) / max(it, 1), "pcg_iters_run": it,
            "sigma": sigma}


def run_cpu_sample(workload: str) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", workload],
                         capture_output=True, text=True, env=env, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


# ----------------------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------------------
def load_peaks() -> tuple[dict, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return dict(FALLBACK_PEAKS), "fallback"


def max_over_ranks(value: float, device) -> float:
    """The largest `value` over the ranks of the default process group (the value itself
    without one): every rank's timed region must end before the job's does."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return value
    t = torch.tensor([value], device=device, dtype=torch.float64)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds


class ClockSampler:
    """nvidia-smi sampling (every 50 ms) of SM clocks and throttle reasons.  `start` returns
    once the first sample has arrived, so the sampler is running before the timed region
    opens; `stop(t0, t1)` keeps the samples taken between two `time.perf_counter` marks (the
    first one after t0 when the region is shorter than the interval)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []   # (perf_counter at arrival, csv line)

    def start(self, wait_s: float = 5.0):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except FileNotFoundError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()
        t_end = time.perf_counter() + wait_s
        while not self.lines and time.perf_counter() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    @staticmethod
    def summarise(lines) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}

    def stop(self, t0: float = None, t1: float = None) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        if t1 is not None:   # one more interval so that a sample taken inside the region arrives
            time.sleep(2 * self.INTERVAL_MS / 1e3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=5)
        rows = list(self.lines)
        if t0 is not None and t1 is not None:
            inside = [ln for ts, ln in rows if t0 <= ts <= t1]
            if not inside:
                inside = [ln for ts, ln in rows if ts >= t0][:1]
            rows = inside
        else:
            rows = [ln for _, ln in rows]
        return self.summarise(rows)


def kernel_model(w, info, ntype_counts, nloc_by_type, band, precision):
    """Algorithmic work per launch of each kernel class: (FP64 flops, tensor flops, bytes).

    Bytes count one pass over each vector the kernel must read or write (DOF = interior
    unknown, f = sum |N_i| / ndof); FP64 flops count 2 per FMA of the arithmetic the
    kernel must do.
    """
    ndof = info["ndof"]
    nloc_sum = sum(c * n for c, n in zip(ntype_counts, nloc_by_type))
    f = nloc_sum / ndof
    es = 2 if precision == "bf16" else 4
    gemm_flops = sum(2.0 * c * n * n for c, n in zip(ntype_counts, nloc_by_type))
    fp64_band = 0.0
    for c, n in zip(ntype_counts, nloc_by_type):
        b = min(band, n - 1)
        per_sweep = n * b - b * (b + 1) / 2
        fp64_band += c * 2 * 2 * per_sweep
    taps = 3 ** (w.p + 1)
    if w.p == 1:   # fused p update + stencil + (p, q)
        stencil = (2.0 * (taps + 2) * ndof, 0.0, 32.0 * ndof)
    else:
        stencil = (2.0 * (taps + 1) * ndof, 0.0, 16.0 * ndof)
    return {
        "stencil_Asigma": stencil,
        "p_update": (2.0 * ndof, 0.0, 24.0 * ndof),
        "xr_update": (6.0 * ndof, 0.0, 48.0 * ndof),
        "prolong_sum": (2.0 * (3.0 + f) * ndof, 0.0, (24.0 + 4.0 * f) * ndof),
        "pack_restrict": (2.0 * f * ndof, 0.0, (8.0 + es * f) * ndof),
        "local_gemm_tc": (0.0, gemm_flops, (es * f + 4.0 * f) * ndof),
        "local_solve_fp64": (fp64_band, 0.0, 16.0 * f * ndof),
    }


def roofline_entry(name, model, ms_total, nlaunch, peaks, peak_src, precision):
    """The binding roofline of one kernel class (the resource whose ideal time is longest)."""
    fp64, tens, byt = model
    avg_s = ms_total / nlaunch / 1e3
    t_alu = fp64 / (FP64_TFLOPS * 1e12)
    tpeak = peaks["bf16_tflops"] * (0.5 if precision == "tf32" else 1.0)
    t_ten = tens / (tpeak * 1e12)
    t_hbm = byt / (peaks["hbm_gbs"] * 1e9)
    bound = max((t_alu, "alu"), (t_ten, "tensor"), (t_hbm, "hbm"))[1]
    if bound == "alu":
        ent = {"bound": "alu", "achieved": fp64 / avg_s / 1e12, "peak": FP64_TFLOPS, "unit": "TFLOP/s",
               "peak_source": "FP64 FMA microbenchmark on this GB300: 8 independent FMA chains per thread, "
                              "152 x 8 blocks of 256 threads"}
    elif bound == "tensor":
        ent = {"bound": "tensor", "achieved": tens / avg_s / 1e12, "peak": tpeak, "unit": "TFLOP/s",
               "peak_source": peak_src + (" (bf16 x 1/2 for tf32)" if precision == "tf32" else "")}
    else:
        ent = {"bound": "hbm", "achieved": byt / avg_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "peak_source": peak_src}
    ent["frac"] = ent["achieved"] / ent["peak"]
    ent["kernel"] = name
    ent["avg_launch_us"] = avg_s * 1e6
    ent["launches"] = nlaunch
    ent["hbm_gbs_algorithmic"] = byt / avg_s / 1e9
    ent["traffic"] = TRAFFIC.get(name)
    return ent


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the current kernels
# from one ncu capture of this workload (profiles/top_kernels_cfg2_bench.md,
# profiles/local_solve_fp64_cfg2.md); a kernel changed since its capture is left out.
TRAFFIC = {
    "stencil_Asigma": (33.651 + 0.615) * 1e6,
    "prolong_sum": (44.916 + 0.131) * 1e6,
    "xr_update": (67.133 + 0.625) * 1e6,
    "pack_restrict": (16.874 + 0.000) * 1e6,
    "local_gemm_tc": (15.096 + 0.000) * 1e6,
    "local_solve_fp64": (18.789 + 0.022) * 1e6,
}


# ----------------------------------------------------------------------------------------
# reference arm: the oracle as it stands
# ----------------------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from ddinputs import WORKLOADS
    w = WORKLOADS[args.workload]
    times = []
    samples = []
    for i in range(args.warmup + args.steps):
        s = run_cpu_sample(args.workload)
        samples.append(s)
    # extrapolation to a full ground state: the plain method's inner iterations on this
    # workload (outer x inner, measured by the FP64 GPU run of the same algorithm)
    inner_total = REF_INNER_ITERS.get(args.workload)
    for s in samples[args.warmup:]:
        times.append(s["setup_s"] + s["pcg_s_per_iter"] * inner_total)
    t = sum(times) / len(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": 1.0 / t, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: p=1, L={w.L}, h=1/{w.n}, delta={w.overlap}, "
                                 f"dofs={w.dofs}, V=4-term cosine (seed {w.seed})",
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": 1.0 / t, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"per step: oracle set-up + 3 PCG iterations; extrapolated with "
                                   f"{inner_total} inner iterations per ground state"},
        "e2e": {"value": 1.0 / t, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# total inner PCG iterations of one ground state with the plain FP64 method, used to
# extrapolate oracle samples (filled from the GPU run of the same algorithm)
REF_INNER_ITERS = {"cfg2": 330, "cfg1": 106, "cfg2_small": 250}


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------
def setup_only(args, dd, dev, reps=3):
    """Times the two set-up stages of one ground state on their own: the cell eigen-solve
    (shift and cell eigenfunction) and the coarse build (local factors or inverses and the
    coarse matrix).  One untimed pass, then `reps` timed ones with CUDA events."""
    import torch
    from ddinputs import WORKLOADS, sample_cell_qp
    w = WORKLOADS[args.setup_only]
    V = torch.from_numpy(sample_cell_qp(w)).to(dev)
    es = dd.Eigensolver(dd.grid_from_workload(w, precision=dd.PRECISIONS[args.precision]), V)
    stream = torch.cuda.current_stream(dev)
    t_cell, t_coarse = [], []
    for i in range(reps + 1):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        e[0].record(stream)
        dd.dd_set_potential(es.ctx, V)
        sigma = dd.dd_cell_eigenpair(es.ctx)
        e[1].record(stream)
        dd.dd_coarse_build(es.ctx)
        e[2].record(stream)
        torch.cuda.synchronize()
        if i:
            t_cell.append(e[0].elapsed_time(e[1]))
            t_coarse.append(e[1].elapsed_time(e[2]))
    es.close()
    return {"mode": "setup_only", "workload": args.setup_only, "dofs": w.dofs, "precision": args.precision,
            "sigma": sigma, "ms_cell_eigenpair": t_cell, "ms_coarse_build": t_coarse}


def main():
    args = parse()
    if args.cpu_sample:
        print(json.dumps(cpu_sample(args.cpu_sample)))
        return
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch
    import paper_2311_08757_gb300 as dd
    from ddinputs import WORKLOADS, sample_cell_qp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    if not os.path.exists(dd.lib_path()):
        raise RuntimeError("libddeig.so is not built (run __graft_entry__.build())")
    if args.setup_only:
        if rank == 0:
            print(json.dumps(setup_only(args, dd, dev)))
        return

    w = WORKLOADS[args.workload]
    V_host = sample_cell_qp(w)
    V = torch.from_numpy(V_host).to(dev)
    ones = torch.ones(w.dofs, dtype=torch.float64, device=dev)
    x = torch.empty_like(ones)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    def make(prec):
        es = dd.Eigensolver(dd.grid_from_workload(w, precision=dd.PRECISIONS[prec]), V)
        dd.dd_set_option(es.ctx, dd.DD_OPT_COARSE_SOLVE, {"auto": 0, "cr": 1, "dense": 2}[args.coarse_solve])
        return es

    def step(es):
        dd.dd_set_potential(es.ctx, V)
        sigma = dd.dd_cell_eigenpair(es.ctx)
        dd.dd_coarse_build(es.ctx)
        x.copy_(ones)
        lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
        return lam, sigma, outer, tot

    def step_lopcg(es, inner):
        dd.dd_set_potential(es.ctx, V)
        sigma = dd.dd_cell_eigenpair(es.ctx)
        dd.dd_coarse_build(es.ctx)
        x.copy_(ones)
        lam, outer, tot, mx = dd.dd_lopcg(es.ctx, x, inner)
        return lam, sigma, outer, tot

    def timed(es, nsteps, count_launches=False, fn=None):
        stream = torch.cuda.current_stream()
        per = []
        res = None
        l0 = dd.dd_kernel_launch_count()
        for _ in range(nsteps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = step(es) if fn is None else fn(es)
            e1.record(stream)
            torch.cuda.synchronize()
            per.append(e0.elapsed_time(e1))
        l1 = dd.dd_kernel_launch_count()
        flushes = nsteps  # flush kernels are torch's, not counted by the library
        return per, res, (l1 - l0)

    mixed = make(args.precision)
    for _ in range(args.warmup):
        step(mixed)

    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    per, res, launches = timed(mixed, args.steps)
    torch.cuda.synchronize()
    barrier()
    t_wall1 = time.perf_counter()
    t_wall = t_wall1 - t_wall0
    clk = clocks.stop(t_wall0, t_wall1)
    lam, sigma, outer, inner_tot = res
    step_ms = sum(per) / len(per)
    step_ms = max_over_ranks(step_ms, dev)
    value = whole_job_rate(1.0, world, step_ms / 1e3)

    # plain FP64 method, same workload
    fp64_steps = args.fp64_steps if args.fp64_steps is not None else max(1, args.steps // 2)
    plain = make("fp64")
    step(plain)
    per64, res64, _ = timed(plain, fp64_steps)
    fp64_ms = sum(per64) / len(per64)

    # SI-LOPCG (Algorithm 1) with the three inner strategies of Sec. 4.3, same workload and
    # stop rule, mixed and plain forms
    lopcg = {}
    if not args.no_lopcg:
        for form, es_f in (("mixed", mixed), ("fp64_plain", plain)):
            for inner in ("fixed", "adaptive", "fused"):
                if form == "fp64_plain" and inner == "fixed":
                    continue
                fn = (lambda e, m=inner: step_lopcg(e, m))
                fn(es_f)
                perl, resl, _ = timed(es_f, max(1, min(3, args.steps)), fn=fn)
                lopcg[f"{form}_{inner}"] = {"ms": sum(perl) / len(perl), "lambda": resl[0], "outer_iters": resl[2],
                                            "inner_iters_total": resl[3]}

    # differentiable workload (L = 256, 8-mode cosine potential): forward ground state and the
    # backward pass (Hellmann-Feynman reduction + adjoint PCG) of lambda and of the
    # eigenvector loss ||phi - phi_target||_M^2
    grad_line = None
    if not args.no_grad:
        from ddinputs import theta_seed, theta8_qp_basis
        w5 = WORKLOADS["cfg5"]
        th5, tt5 = theta_seed(w5.seed)
        B5 = torch.from_numpy(theta8_qp_basis(w5)).to(dev)
        es5 = dd.Eigensolver(dd.grid_from_workload(w5, precision=dd.PRECISIONS[args.precision]),
                             torch.from_numpy(tt5).to(dev) @ B5)
        es5.prepare()
        phi5t = torch.ones(w5.dofs, dtype=torch.float64, device=dev)
        dd.dd_inverse_iterate(es5.ctx, phi5t)
        V5 = (torch.from_numpy(th5).to(dev) @ B5).contiguous()
        x5 = torch.empty(w5.dofs, dtype=torch.float64, device=dev)
        g5 = torch.empty(w5.dofs, dtype=torch.float64, device=dev)
        dV5 = torch.empty_like(V5)
        fw, bw, its = [], [], 0
        for rep in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dd.dd_set_potential(es5.ctx, V5)
            dd.dd_cell_eigenpair(es5.ctx)
            dd.dd_coarse_build(es5.ctx)
            x5.fill_(1.0)
            lam5 = dd.dd_inverse_iterate(es5.ctx, x5)[0]
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            dd.dd_apply_operator(es5.ctx, dd.DD_OP_MASS, (x5 - phi5t).contiguous(), g5)
            g5.mul_(2.0)
            its = dd.dd_potential_gradient(es5.ctx, x5, lam5, 1.0, g5, dV5)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            if rep > 0:
                fw.append(t1 - t0)
                bw.append(t2 - t1)
        es5.close()
        grad_line = {"workload": "cfg5: p=1, L=256, h=1/32, delta=4, V = sum_j theta_j cos(2 pi j x)(1+0.3y), "
                                 f"theta ~ N(0,25) seed {w5.seed}",
                     "forward_ms": 1e3 * sum(fw) / len(fw), "backward_ms": 1e3 * sum(bw) / len(bw),
                     "adjoint_pcg_iters": its, "lambda": lam5}

    # batched workload: 64 instances, L log-uniform in [16, 2048], own potentials; all
    # pipelines (cell eigenpair, coarse build, inverse iteration) concurrent on the GPU
    batch_line = None
    if not args.no_batch:
        from ddinputs import batch_workloads
        wb = batch_workloads()
        grids_b = [dd.grid_from_workload(wi, precision=dd.PRECISIONS[args.precision]) for wi in wb]
        Vb = [torch.from_numpy(sample_cell_qp(wi)).to(dev) for wi in wb]
        with dd.Batch(grids_b, Vb) as bt:
            runs = {}
            for label, method, threads in (("concurrent_ipm", "ipm", 0), ("concurrent_lopcg_fused", "lopcg_fused", 0),
                                           ("one_thread_ipm", "ipm", 1)):
                bt.ground_states(method, threads=threads)          # warm-up (graphs, workspaces)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rb = bt.ground_states(method, threads=threads)
                torch.cuda.synchronize()
                tb = time.perf_counter() - t0
                runs[label] = {"seconds": tb, "eigenpairs_per_s": len(wb) / tb,
                               "instance_seconds_min_median_max": [float(rb["seconds"].min()),
                                                                   float(np.median(rb["seconds"])),
                                                                   float(rb["seconds"].max())],
                               "inner_iters_total": int(rb["inner"].sum())}
        batch_line = {"workload": f"cfg4: {len(wb)} instances, p=1, h=1/32, delta=4, L log-uniform in [16, 2048] "
                                  f"(sum of unknowns {sum(wi.dofs for wi in wb)}), own 4-term cosine potentials "
                                  "(seed 4242)", **runs}

    # the d = 3 workload (p = 2, L = 64, h = 1/16, delta = 2, Gaussian wells; 15.7M unknowns,
    # 4096 subdomains of 9 types): mixed form, same step as the headline
    d3_line = None
    if not args.no_3d:
        w3 = WORKLOADS["cfg3"]
        V3 = torch.from_numpy(sample_cell_qp(w3)).to(dev)
        es3 = dd.Eigensolver(dd.grid_from_workload(w3, precision=dd.PRECISIONS[args.precision]), V3)
        x3 = torch.empty(w3.dofs, dtype=torch.float64, device=dev)

        def step3():
            dd.dd_set_potential(es3.ctx, V3)
            dd.dd_cell_eigenpair(es3.ctx)
            dd.dd_coarse_build(es3.ctx)
            x3.fill_(1.0)
            return dd.dd_inverse_iterate(es3.ctx, x3)

        step3()
        torch.cuda.synchronize()
        ts3 = []
        for _ in range(2):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            r3 = step3()
            e1.record()
            torch.cuda.synchronize()
            ts3.append(e0.elapsed_time(e1))
        d3_line = {"workload": f"cfg3: p=2, L=64, h=1/16, delta=2, dofs={w3.dofs}, 4096 subdomains, Gaussian-well "
                               "lattice", "precision": args.precision, "ms_per_ground_state": sum(ts3) / len(ts3),
                   "lambda": r3[0], "outer_iters": r3[1], "inner_iters_total": r3[2]}
        es3.close()

    # phase breakdown of one step (host timer around each synchronous call)
    def phases(es):
        out = {}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dd.dd_set_potential(es.ctx, V)
        t1 = time.perf_counter()
        dd.dd_cell_eigenpair(es.ctx)
        t2 = time.perf_counter()
        dd.dd_coarse_build(es.ctx)
        t3 = time.perf_counter()
        x.copy_(ones)
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        dd.dd_inverse_iterate(es.ctx, x)
        t5 = time.perf_counter()
        return {"set_potential": 1e3 * (t1 - t0), "cell_eigenpair": 1e3 * (t2 - t1),
                "coarse_build": 1e3 * (t3 - t2), "inverse_iterate": 1e3 * (t5 - t4)}

    breakdown = {"mixed": phases(mixed), "fp64_plain": phases(plain)}

    # per-kernel device times (CUDA events around every launch, one profiled step)
    dd.dd_set_option(mixed.ctx, dd.DD_OPT_TIMING, 1)
    dd.dd_reset_timings(mixed.ctx)
    step(mixed)
    kt = dd.dd_kernel_timings(mixed.ctx)
    dd.dd_set_option(mixed.ctx, dd.DD_OPT_TIMING, 0)
    dd.dd_set_option(plain.ctx, dd.DD_OPT_TIMING, 1)
    dd.dd_reset_timings(plain.ctx)
    step(plain)
    kt64 = dd.dd_kernel_timings(plain.ctx)
    dd.dd_set_option(plain.ctx, dd.DD_OPT_TIMING, 0)

    info = mixed.info
    peaks, peak_src = load_peaks()
    subs = []
    nloc_interior = (w.n + 2 * w.overlap - 1) * (w.ny - 1)
    nloc_edge = (w.n + w.overlap - 1) * (w.ny - 1)
    counts, nlocs = ([w.L - 2, 2], [nloc_interior, nloc_edge]) if w.p == 1 and w.L > 2 else ([1], [info["nloc_max"]])
    model = kernel_model(w, info, counts, nlocs, info["band_local"], args.precision)
    busy = {k: v for k, v in kt.items() if v[0] > 0}
    dom = max((k for k in busy if k in model), key=lambda k: busy[k][1])
    roofline = roofline_entry(dom, model[dom], busy[dom][1], busy[dom][0], peaks, peak_src, args.precision)
    others = {k: roofline_entry(k, model[k], v[1], v[0], peaks, peak_src, args.precision)
              for k, v in busy.items() if k in model and k != dom}
    kernel_table = {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in busy.items()}
    kernel_table64 = {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in kt64.items() if v[0] > 0}

    # end to end through the public C-ABI with HOST buffers: one context serves the stream of
    # potentials (dd_setup once); every step uploads V and x_0 from pinned host memory and
    # returns phi to host memory.  The one-shot dd_eigenpair (context set-up and teardown
    # inside) is reported beside it.
    e2e = None
    if not args.no_e2e:
        Vp = torch.from_numpy(V_host).pin_memory()
        x0 = torch.ones(w.dofs, dtype=torch.float64).pin_memory()
        phi = torch.empty(w.dofs, dtype=torch.float64).pin_memory()
        es_h = make(args.precision)

        def host_step():
            dd.dd_set_potential(es_h.ctx, Vp)
            dd.dd_cell_eigenpair(es_h.ctx)
            dd.dd_coarse_build(es_h.ctx)
            phi.copy_(x0)
            return dd.dd_inverse_iterate(es_h.ctx, phi)

        for _ in range(2):
            host_step()
        ts = []
        for _ in range(max(1, args.steps)):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lam_h = host_step()[0]
            ts.append(time.perf_counter() - t0)
        te = sum(ts) / len(ts)
        es_h.close()
        g = dd.grid_from_workload(w, precision=dd.PRECISIONS[args.precision])
        dd.dd_eigenpair(g, Vp, phi_out=phi)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dd.dd_eigenpair(g, Vp, phi_out=phi)
        t_cold = time.perf_counter() - t0
        te = max_over_ranks(te, dev)
        e2e = {"value": whole_job_rate(1.0, world, te), "unit": UNIT, "h2d_bytes_per_step": int(Vp.numel() * 8 + x0.numel() * 8),
               "d2h_bytes_per_step": int(phi.numel() * 8), "ms_per_step": te * 1e3,
               "path": "dd_set_potential + dd_cell_eigenpair + dd_coarse_build + dd_inverse_iterate, host buffers",
               "lambda": lam_h,
               "one_shot_dd_eigenpair_ms": t_cold * 1e3}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            s = run_cpu_sample(args.workload)
            t_cpu = s["setup_s"] + s["pcg_s_per_iter"] * res64[3]
            cpu = {"value": 1.0 / t_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": (f"oracle set-up of the same workload ({s['setup_s']:.1f} s: assembly, cell "
                              f"eigenpair, {w.L ** w.p} local factorisations, coarse factorisation) + "
                              f"{s['pcg_iters_run']} PCG iterations ({s['pcg_s_per_iter']:.3f} s each); "
                              f"time to ground state extrapolated with the {res64[3]} inner iterations "
                              f"the plain FP64 method needs"),
                   "est_time_to_ground_state_s": t_cpu}
        except Exception as e:  # noqa: BLE001
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (local inverses %s)" % args.precision, "data": "synthetic",
            "config": {"workload": f"{args.workload}: p=1, L={w.L}, ell=1, h=1/{w.n}, delta={w.overlap}, "
                                   f"dofs={w.dofs}, {w.L ** w.p} subdomains, V=4-term cosine (seed {w.seed})",
                       "precision": args.precision, "l2": "flushed between steps (256 MB write)",
                       "local_gemm_tile": f"128x{dd.dd_query(mixed.ctx)['gemm_tile_n']}",
                       "parallelism": f"replicas x{world}"},
            "time_to_ground_state_ms": {"mixed": step_ms, "fp64_plain": fp64_ms,
                                        "speedup_mixed_vs_fp64": fp64_ms / step_ms},
            "lambda": lam, "sigma": sigma, "outer_iters": outer, "inner_iters_total": inner_tot,
            "fp64_plain": {"lambda": res64[0], "outer_iters": res64[2], "inner_iters_total": res64[3]},
            "pcg_iters_per_s": inner_tot / (step_ms / 1e3),
            "si_lopcg_time_to_ground_state": lopcg,
            "differentiable": grad_line,
            "batched": batch_line,
            "d3": d3_line,
            "roofline": roofline,
            "roofline_other_kernels": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv)
                                           for kk, vv in v.items() if kk in ("bound", "achieved", "peak", "unit",
                                                                             "frac", "avg_launch_us")}
                                       for k, v in others.items()},
            "breakdown_ms": breakdown,
            "kernels_mixed": kernel_table, "kernels_fp64": kernel_table64,
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "wall_s_timed_region": t_wall,
        }
        print(json.dumps(line))
    mixed.close()
    plain.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
