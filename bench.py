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
ALU_PEAK_SOURCE = ("dd_alu_peak_test, measured in this run: 8 independent FMA chains per thread, 8 blocks of 256 "
                   "threads per SM, fastest of 5 launches")


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
    ap.add_argument("--no-sweeps", action="store_true")
    ap.add_argument("--coarse-solve", default="auto", choices=["auto", "cr", "dense"])
    ap.add_argument("--cpu-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--setup-only", default=None, choices=["cfg2", "cfg3"],
                    help="time only the set-up stages (cell eigenpair, coarse build) of one workload")
    ap.add_argument("--profile-region", default=None, choices=["cfg2", "cfg3"],
                    help="set up one workload, then run --pcg-iters PCG iterations (eager launches) between "
                         "cudaProfilerStart/Stop, for `ncu --profile-from-start off`")
    ap.add_argument("--pcg-iters", type=int, default=2)
    ap.add_argument("--gemm-tile", type=int, default=0, choices=[0, 128, 160, 256],
                    help="--profile-region: the local GEMM's N tile (0: the set-up autotuner's choice, which "
                         "under ncu sees serialised launches)")
    ap.add_argument("--one-shot-breakdown", action="store_true",
                    help="time dd_setup, dd_cell_eigenpair, dd_coarse_build, dd_inverse_iterate and dd_destroy "
                         "of fresh contexts on the headline workload")
    return ap.parse_args()


# ----------------------------------------------------------------------------------------
# the oracle's full ground state (runs in a child process with one BLAS thread)
# ----------------------------------------------------------------------------------------
def cpu_ground_state(workload: str) -> dict:
    """One complete ground state by the oracle as it stands: assembly, cell eigenpair, the
    decomposition with one banded Cholesky factor per subdomain and the dense coarse factor,
    then the shifted inverse iteration with its own PCG (same stop rules as the GPU)."""
    import numpy as np
    from ddinputs import WORKLOADS, potential
    from oracle import q1, solvers
    w = WORKLOADS[workload]
    t0 = time.perf_counter()
    g = q1.Grid.from_workload(w)
    P = solvers.Problem(g, potential(w))
    t1 = time.perf_counter()
    lam, x, k, inner, info = P.ground_state()
    t2 = time.perf_counter()
    return {"setup_s": t1 - t0, "solve_s": t2 - t1, "total_s": t2 - t0, "outer": int(k),
            "inner_total": int(np.sum(inner)), "lambda": float(lam), "sigma": float(P.sigma)}


def cpu_child_env() -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    return env


def start_cpu_ground_state(workload: str) -> subprocess.Popen:
    return subprocess.Popen([sys.executable, os.path.abspath(__file__), "--cpu-sample", workload],
                            stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=cpu_child_env())


def finish_cpu_ground_state(proc: subprocess.Popen, timeout: float = 900.0) -> dict:
    out, err = proc.communicate(timeout=timeout)
    if proc.returncode != 0:
        raise RuntimeError(err[-2000:])
    return json.loads(out.strip().splitlines()[-1])


def cpu_baseline_entry(s: dict, w) -> dict:
    return {"value": 1.0 / s["total_s"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"one full ground state of the same workload by the oracle (numpy/scipy FP64, one BLAS "
                       f"thread): set-up {s['setup_s']:.1f} s (assembly, cell eigenpair, {w.L ** w.p} banded local "
                       f"factorisations, coarse factorisation) + inverse iteration {s['solve_s']:.1f} s "
                       f"({s['outer']} outer steps, {s['inner_total']} PCG iterations of its own)"),
            "setup_s": s["setup_s"], "solve_s": s["solve_s"], "outer_iters": s["outer"],
            "inner_iters_total": s["inner_total"], "lambda": s["lambda"]}


def workload_label(w) -> str:
    if w.p == 1:
        return (f"{w.name}: p=1, L={w.L}, ell=1, h=1/{w.n}, delta={w.overlap}, dofs={w.dofs}, {w.L ** w.p} "
                f"subdomains, V=4-term cosine (seed {w.seed})")
    return f"{w.name}: p=2, L={w.L}, ell=1, h=1/{w.n}, delta={w.overlap}, dofs={w.dofs}, {w.L ** w.p} subdomains"


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
    """Algorithmic work per launch of each kernel class: FP64 flops, FP32 flops, tensor flops
    and bytes (2 flops per FMA; bytes = one pass over each vector the kernel must read or
    write; DOF = interior unknown, f = sum |N_i| / ndof).  Work a kernel does in FP32 is
    counted against the FP32 pipe, FP64 work against the FP64 pipe."""
    ndof = info["ndof"]
    nloc_sum = sum(c * n for c, n in zip(ntype_counts, nloc_by_type))
    f = nloc_sum / ndof
    mixed = precision in ("bf16", "tf32")
    es = 2 if precision == "bf16" else 4
    gemm_flops = sum(2.0 * c * n * n for c, n in zip(ntype_counts, nloc_by_type))
    fp64_band = 0.0
    for c, n in zip(ntype_counts, nloc_by_type):
        b = min(band, n - 1)
        per_sweep = n * b - b * (b + 1) / 2
        fp64_band += c * 2 * 2 * per_sweep
    taps = 3 ** (w.p + 1)
    # the p update also makes the previous iteration's x += alpha p (DD_OPT_X_LAG, the default):
    # x read and written, one FMA
    if w.p == 1 and mixed:
        # fused p update + stencil + (p, q) with q = A_sigma p in float pairs (the default with
        # rounded local inverses): FP64 p update, x update, q = hi + lo and the (p, q) FMA
        # (7 flops); per tap one error-free product and sum with the cross terms (15 FP32 flops)
        stencil = (7.0 * ndof, 15.0 * taps * ndof, 0.0, 48.0 * ndof)
    elif w.p == 1:   # fused p update + x update + stencil + (p, q)
        stencil = (2.0 * (taps + 3) * ndof, 0.0, 0.0, 48.0 * ndof)
    elif mixed:
        # p = 2 in float pairs: the taps read the split p (8 B), the (p, q) FMA reads p (8 B),
        # q written (8 B); FP64: q = hi + lo and the (p, q) FMA (3 flops)
        stencil = (3.0 * ndof, 15.0 * taps * ndof, 0.0, 24.0 * ndof)
    else:
        stencil = (2.0 * (taps + 1) * ndof, 0.0, 0.0, 16.0 * ndof)
    # prolong-sum: per owner of a node one add of its local result and one FMA of the coarse
    # term (3 flops), then the (r, z) and (q, z) dots (4 FP64 flops); the mixed form forms the
    # node value in FP32 from FP32 local results
    if mixed:
        prolong = (4.0 * ndof, 3.0 * f * ndof, 0.0, (24.0 + 4.0 * f) * ndof)
    else:
        prolong = ((4.0 + 3.0 * f) * ndof, 0.0, 0.0, (24.0 + 8.0 * f) * ndof)
    return {
        "stencil_Asigma": stencil,
        # p = 2 in float pairs: the split p is written beside p
        "p_update": (4.0 * ndof, 0.0, 0.0, (48.0 if (mixed and w.p == 2) else 40.0) * ndof),
        # r -= alpha q and (r, r); x is updated by the next p update
        "xr_update": (4.0 * ndof, 0.0, 0.0, 24.0 * ndof),
        "prolong_sum": prolong,
        "pack_restrict": (2.0 * f * ndof, 0.0, 0.0, (8.0 + es * f) * ndof),
        "local_gemm_tc": (0.0, 0.0, gemm_flops, (es * f + 4.0 * f) * ndof),
        "local_solve_fp64": (fp64_band, 0.0, 0.0, 16.0 * f * ndof),
    }


def roofline_entry(name, model, ms_total, nlaunch, peaks, peak_src, precision, alu):
    """The binding roofline of one kernel class: the resource (FP64 pipe, FP32 pipe, tensor
    pipe, HBM) whose ideal time for the kernel's algorithmic work is longest."""
    fp64, fp32, tens, byt = model
    avg_s = ms_total / nlaunch / 1e3
    tpeak = peaks["bf16_tflops"] * (0.5 if precision == "tf32" else 1.0)
    times = [(fp64 / (alu["fp64_tflops"] * 1e12), "fp64"), (fp32 / (alu["fp32_tflops"] * 1e12), "fp32"),
             (tens / (tpeak * 1e12), "tensor"), (byt / (peaks["hbm_gbs"] * 1e9), "hbm")]
    bound = max(times)[1]
    if bound in ("fp64", "fp32"):
        work = fp64 if bound == "fp64" else fp32
        ent = {"bound": "alu", "pipe": bound, "achieved": work / avg_s / 1e12, "peak": alu[bound + "_tflops"],
               "unit": "TFLOP/s", "peak_source": ALU_PEAK_SOURCE}
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
    ent["hbm_frac_algorithmic"] = byt / avg_s / 1e9 / peaks["hbm_gbs"]
    ent["traffic"] = TRAFFIC.get(name)
    return ent


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the current kernels
# at the L = 2048, h = 1/32 workload, from one ncu capture of each; a kernel changed since its
# capture is left out.
TRAFFIC = {
    "stencil_Asigma": (50.447 + 1.114) * 1e6,   # an iteration k >= 1 pass (it also updates x)
    "xr_update": (33.576 + 0.000) * 1e6,
    "pack_restrict": (16.87 + 0.000) * 1e6,
    "local_gemm_tc": (15.103 + 0.000) * 1e6,
    "prolong_sum": (45.93 + 0.147) * 1e6,
    "local_solve_fp64": (18.789 + 0.022) * 1e6,
}


# ----------------------------------------------------------------------------------------
# reference arm: the oracle as it stands
# ----------------------------------------------------------------------------------------
def run_reference(args):
    """The oracle as it stands, on the host cores: one complete ground state of the headline
    workload, timed whole (about a minute on one core).  One step is timed whatever --steps
    asks for, so that ms_per_step x steps is the measured time; `requested` records the
    flags."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from ddinputs import WORKLOADS
    w = WORKLOADS[args.workload]
    t0 = time.perf_counter()
    s = finish_cpu_ground_state(start_cpu_ground_state(args.workload), timeout=1800)
    wall = time.perf_counter() - t0
    t = s["total_s"]
    line = {
        "impl": "reference", "metric": METRIC, "value": 1.0 / t, "unit": UNIT, "n_gpus": args.gpus,
        "steps": 1, "warmup": 0, "requested": {"steps": args.steps, "warmup": args.warmup},
        "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_label(w), "precision": "fp64 (plain method)", "l2": "n/a (CPU)"},
        "cpu_baseline": cpu_baseline_entry(s, w),
        "e2e": {"value": 1.0 / t, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "time_to_ground_state_ms": {"setup": 1e3 * s["setup_s"], "solve": 1e3 * s["solve_s"]},
        "wall_s": wall,
    }
    print(json.dumps(line))


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


def profile_region(args, dd, dev):
    """Set-up outside the profiled range, then `--pcg-iters` PCG iterations on b = M 1 with
    eager launches (no graph) inside cudaProfilerStart/Stop."""
    import torch
    from ddinputs import WORKLOADS, sample_cell_qp
    w = WORKLOADS[args.profile_region]
    V = torch.from_numpy(sample_cell_qp(w)).to(dev)
    with dd.Eigensolver(dd.grid_from_workload(w, precision=dd.PRECISIONS[args.precision]), V) as es:
        es.prepare()
        dd.dd_set_option(es.ctx, dd.DD_OPT_USE_GRAPH, 0)
        dd.dd_set_option(es.ctx, dd.DD_OPT_CHECK_EVERY, 1)
        if args.gemm_tile:
            dd.dd_set_option(es.ctx, dd.DD_OPT_GEMM_TILE_N, args.gemm_tile)
        ones = torch.ones(w.dofs, dtype=torch.float64, device=dev)
        b = torch.empty_like(ones)
        dd.dd_apply_operator(es.ctx, dd.DD_OP_MASS, ones, b)
        x = torch.zeros_like(ones)
        dd.dd_pcg_solve(es.ctx, b, x, 1e-8, 1, allow_maxit=True)   # untimed warm pass
        x.zero_()
        torch.cuda.synchronize()
        l0 = dd.dd_kernel_launch_count()
        torch.cuda.profiler.start()
        its, rel = dd.dd_pcg_solve(es.ctx, b, x, 1e-8, args.pcg_iters, allow_maxit=True)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        l1 = dd.dd_kernel_launch_count()
    return {"mode": "profile_region", "workload": args.profile_region, "dofs": w.dofs, "precision": args.precision,
            "pcg_iters": its, "relres": rel, "library_launches": l1 - l0, "gemm_tile": args.gemm_tile}


def one_shot_breakdown(args, dd, dev, reps=3, precision=None):
    """Host wall time of each call of a fresh context (dd_setup ... dd_destroy) on the headline
    workload, device buffers; every call synchronises before it returns, so the host clock
    around it is its time.  The first of reps + 1 passes is untimed."""
    import torch
    from ddinputs import WORKLOADS, sample_cell_qp
    precision = precision or args.precision
    w = WORKLOADS[args.workload]
    V = torch.from_numpy(sample_cell_qp(w)).to(dev)
    x = torch.empty(w.dofs, dtype=torch.float64, device=dev)
    grid = dd.grid_from_workload(w, precision=dd.PRECISIONS[precision])
    rows = []
    for i in range(reps + 1):
        torch.cuda.synchronize()
        t = [time.perf_counter()]
        ctx = dd.dd_setup(grid, V)
        t.append(time.perf_counter())
        dd.dd_cell_eigenpair(ctx)
        t.append(time.perf_counter())
        dd.dd_coarse_build(ctx)
        t.append(time.perf_counter())
        x.fill_(1.0)
        torch.cuda.synchronize()
        t.append(time.perf_counter())
        dd.dd_inverse_iterate(ctx, x)
        t.append(time.perf_counter())
        dd.dd_destroy(ctx)
        t.append(time.perf_counter())
        if i:
            rows.append([1e3 * (b - a) for a, b in zip(t[:-1], t[1:])])
    names = ["dd_setup", "cell_eigenpair", "coarse_build", "fill_x0", "inverse_iterate", "destroy"]
    med = {k: sorted(r[j] for r in rows)[len(rows) // 2] for j, k in enumerate(names)}
    return {"mode": "one_shot_breakdown", "workload": args.workload, "precision": precision,
            "ms": {k: [r[j] for r in rows] for j, k in enumerate(names)},
            "median_ms": med,
            "setup_ms": med["dd_setup"] + med["cell_eigenpair"] + med["coarse_build"],
            "solve_ms": med["inverse_iterate"],
            "total_ms": med["dd_setup"] + med["cell_eigenpair"] + med["coarse_build"] + med["inverse_iterate"]}


def sweeps(dd, dev, headline) -> dict:
    """The iteration-count sweeps of Sec. 4.1 and the L-independence of the eigen-solver's
    inner counts, on the GPU kernels (plain FP64 form unless noted):
      fig3    source problem a_sigma(u, v) = (1, v), printed potential of Sec. 4.1, h = 1/30,
              delta = 1, CG from 1 to rTOL = 1e-8: one-level M_AS1 / two-level M_AS2 counts;
      table1  the same with the distance partition of unity, h in {1/10, 1/20, 1/30} x delta in
              {1, 2, 3} (M_AS1 up to L = 256, M_AS2 up to L = 2048);
      eigen_L inverse iteration on the headline potential (h = 1/32, delta = 4), FP64 and mixed:
              outer steps, inner PCG iterations (total and per outer step), time;
      gmres_ras2  the headline ground state with GMRES + M_RAS2^{-1} as the inner solver (Sec. 2.2,
              Sec. 4.2) beside CG + M_AS2^{-1}."""
    import numpy as np
    import torch
    from ddinputs import WORKLOADS, Workload, sample_cell_qp

    def solver(w, precision="fp64", coarse=1, pu=0):
        V = torch.from_numpy(sample_cell_qp(w)).to(dev)
        es = dd.Eigensolver(dd.grid_from_workload(w, precision=dd.PRECISIONS[precision], coarse=coarse,
                                                  pu_kind=pu), V)
        es.prepare()
        return es

    def count(L, n, delta, coarse, pu):
        w = Workload("e1", p=1, L=L, n=n, overlap=delta, kind="sin4")
        with solver(w, coarse=coarse, pu=pu) as es:
            b = torch.full((w.dofs,), (1.0 / n) ** 2, dtype=torch.float64, device=dev)
            x = torch.ones(w.dofs, dtype=torch.float64, device=dev)
            its, rel = dd.dd_pcg_solve(es.ctx, b, x, 1e-8, 20000)
        return its

    Ls = [2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048]
    fig3 = {"h": "1/30", "delta": 1, "pu": "equal", "L": Ls,
            "as1": [count(L, 30, 1, 0, 0) for L in Ls], "as2": [count(L, 30, 1, 1, 0) for L in Ls]}
    t1L = [16, 256, 2048]
    table1 = {"pu": "distance", "L": t1L, "cases": []}
    for n in (10, 20, 30):
        for delta in (1, 2, 3):
            table1["cases"].append({"h": f"1/{n}", "delta": delta,
                                    "as1": [count(L, n, delta, 0, 1) if L <= 256 else None for L in t1L],
                                    "as2": [count(L, n, delta, 1, 1) for L in t1L]})
    eigen = {"h": "1/32", "delta": 4, "potential": "4-term cosine (seed 2311)", "L": [2, 8, 32, 128, 512, 2048],
             "fp64": [], "mixed": []}
    for L in eigen["L"]:
        w = WORKLOADS["cfg2"].with_(name=f"cfg2_l{L}", L=L)
        for label, prec in (("fp64", "fp64"), ("mixed", "bf16")):
            with solver(w, prec) as es:
                x = torch.ones(w.dofs, dtype=torch.float64, device=dev)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
                ms = 1e3 * (time.perf_counter() - t0)
            eigen[label].append({"outer": outer, "inner_total": tot, "inner_max": mx,
                                 "inner_per_outer": tot / max(outer, 1), "ms": ms})
    w = WORKLOADS["cfg2"]
    gm = {"restart": 30}
    for label, prec in (("fp64", "fp64"), ("mixed", "bf16")):
        with solver(w, prec) as es:
            dd.dd_set_option(es.ctx, dd.DD_OPT_KRYLOV, 1)
            dd.dd_set_option(es.ctx, dd.DD_OPT_PRECOND, 1)
            dd.dd_set_option(es.ctx, dd.DD_OPT_RESTART, gm["restart"])
            x = torch.ones(w.dofs, dtype=torch.float64, device=dev)
            dd.dd_inverse_iterate(es.ctx, x)          # warm-up (GMRES workspace)
            x.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lam, outer, tot, mx = dd.dd_inverse_iterate(es.ctx, x)
            ms = 1e3 * (time.perf_counter() - t0)
        gm[label] = {"lambda": lam, "outer": outer, "inner_total": tot, "inner_max": mx,
                     "inverse_iterate_ms": ms}
    gm["cg_as2_inverse_iterate_ms"] = headline
    return {"fig3": fig3, "table1": table1, "eigen_L": eigen, "gmres_ras2": gm}


def main():
    args = parse()
    if args.cpu_sample:
        print(json.dumps(cpu_ground_state(args.cpu_sample)))
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
    if args.profile_region:
        if rank == 0:
            print(json.dumps(profile_region(args, dd, dev)))
        return
    if args.one_shot_breakdown:
        if rank == 0:
            print(json.dumps(one_shot_breakdown(args, dd, dev)))
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

    # the oracle's full ground state on one host core, in a child process beside the GPU work
    # that follows (started after the headline and end-to-end regions, so that neither shares
    # the host with it)
    cpu_proc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_proc = start_cpu_ground_state(args.workload)

    # measured FP64 / FP32 FMA throughput: the roofline denominators of the ALU-bound kernels
    alu = {"fp64_tflops": dd.dd_alu_peak_test(0, 5), "fp32_tflops": dd.dd_alu_peak_test(1, 5),
           "source": ALU_PEAK_SOURCE}
    peaks, peak_src = load_peaks()

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

            def timed_call(label, method, groups, threads=0, warm=1):
                bt.set_groups(groups)
                for _ in range(warm):
                    bt.ground_states(method, threads=threads)          # warm-up (graphs, workspaces)
                torch.cuda.synchronize()
                l0 = dd.dd_kernel_launch_count()
                t0 = time.perf_counter()
                rb = bt.ground_states(method, threads=threads)
                torch.cuda.synchronize()
                tb = time.perf_counter() - t0
                info = bt.info()
                runs[label] = {"seconds": tb, "eigenpairs_per_s": len(wb) / tb,
                               "instance_seconds_min_median_max": [float(rb["seconds"].min()),
                                                                   float(np.median(rb["seconds"])),
                                                                   float(rb["seconds"].max())],
                               "inner_iters_total": int(rb["inner"].sum()),
                               "kernel_launches": dd.dd_kernel_launch_count() - l0,
                               "batched_kernels": bool(info["last_batched"]),
                               "groups": info["groups"] if info["last_batched"] else None,
                               "grouped_gemm_tile": f"128x{info['gemm_tile_n']}" if info["last_batched"] else None,
                               "setup_phase_s": info["setup_seconds"]}
                return runs[label]

            # batched kernels: every group count timed, then the library's own choice (it tries
            # each count on successive calls and keeps the fastest)
            runs["batched_ipm_by_groups"] = {str(G): timed_call("tmp", "ipm", G)["seconds"] for G in (1, 2, 4, 8)}
            bt.set_groups(0)
            for _ in range(8):
                bt.ground_states("ipm")
            timed_call("batched_ipm", "ipm", 0, warm=0)
            for _ in range(8):
                bt.ground_states("lopcg_fused")
            timed_call("batched_lopcg_fused", "lopcg_fused", 0, warm=0)
            # the same methods as concurrent per-instance pipelines, and one thread
            timed_call("concurrent_ipm", "ipm", -1)
            timed_call("concurrent_lopcg_fused", "lopcg_fused", -1)
            timed_call("one_thread_ipm", "ipm", -1, threads=1)
            runs.pop("tmp", None)
        batch_line = {"workload": f"cfg4: {len(wb)} instances, p=1, h=1/32, delta=4, L log-uniform in [16, 2048] "
                                  f"(sum of unknowns {sum(wi.dofs for wi in wb)}), own 4-term cosine potentials "
                                  "(seed 4242), mixed (bf16 local inverses)", **runs}

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
        # per-kernel device times of one profiled ground state (CUDA events around every
        # launch) and each kernel class against its binding roofline
        dd.dd_set_option(es3.ctx, dd.DD_OPT_TIMING, 1)
        dd.dd_reset_timings(es3.ctx)
        step3()
        kt3 = {k: v for k, v in dd.dd_kernel_timings(es3.ctx).items() if v[0] > 0}
        dd.dd_set_option(es3.ctx, dd.DD_OPT_TIMING, 0)
        i3 = es3.info
        wi, we = w3.n + 2 * w3.overlap - 1, w3.n + w3.overlap - 1
        cnt3 = [(w3.L - 2) ** 2, 4 * (w3.L - 2), 4]
        nl3 = [wi * wi * (w3.ny - 1), wi * we * (w3.ny - 1), we * we * (w3.ny - 1)]
        m3 = kernel_model(w3, i3, cnt3, nl3, i3["band_local"], args.precision)
        d3_line["kernels"] = {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in kt3.items()}
        d3_line["roofline"] = {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv)
                                   for kk, vv in roofline_entry(k, m3[k], v[1], v[0], peaks, peak_src, args.precision,
                                                                alu).items()
                                   if kk in ("bound", "pipe", "achieved", "peak", "unit", "frac", "avg_launch_us",
                                             "launches", "hbm_frac_algorithmic")}
                               for k, v in kt3.items() if k in m3}
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

    sweep_line = None
    if not args.no_sweeps:
        sweep_line = sweeps(dd, dev, {"fp64": breakdown["fp64_plain"]["inverse_iterate"],
                                      "mixed": breakdown["mixed"]["inverse_iterate"]})

    # time to the ground state from dd_setup (a fresh context each time), split into set-up
    # (dd_setup, cell eigenpair, coarse build) and solve (inverse iteration)
    from_setup = {}
    for label, prec in (("mixed", args.precision), ("fp64_plain", "fp64")):
        ob = one_shot_breakdown(args, dd, dev, reps=3, precision=prec)
        from_setup[label] = {"setup_ms": ob["setup_ms"], "solve_ms": ob["solve_ms"], "total_ms": ob["total_ms"],
                             "destroy_ms": ob["median_ms"]["destroy"],
                             "phases_ms": {k: round(v, 3) for k, v in ob["median_ms"].items()}}

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
    subs = []
    nloc_interior = (w.n + 2 * w.overlap - 1) * (w.ny - 1)
    nloc_edge = (w.n + w.overlap - 1) * (w.ny - 1)
    counts, nlocs = ([w.L - 2, 2], [nloc_interior, nloc_edge]) if w.p == 1 and w.L > 2 else ([1], [info["nloc_max"]])
    model = kernel_model(w, info, counts, nlocs, info["band_local"], args.precision)
    busy = {k: v for k, v in kt.items() if v[0] > 0}
    dom = max((k for k in busy if k in model), key=lambda k: busy[k][1])
    roofline = roofline_entry(dom, model[dom], busy[dom][1], busy[dom][0], peaks, peak_src, args.precision, alu)
    others = {k: roofline_entry(k, model[k], v[1], v[0], peaks, peak_src, args.precision, alu)
              for k, v in busy.items() if k in model and k != dom}
    kernel_table = {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in busy.items()}
    kernel_table64 = {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in kt64.items() if v[0] > 0}

    cpu = None
    if cpu_proc is not None:
        try:
            cpu = cpu_baseline_entry(finish_cpu_ground_state(cpu_proc), w)
        except Exception as e:  # noqa: BLE001
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic",
            "dtype": "f64 (local inverses %s%s)" % (args.precision, "; inner-solve A_sigma p in float pairs"
                                                    if args.precision in ("bf16", "tf32") and w.p == 1 else ""),
            "config": {"workload": workload_label(w),
                       "precision": args.precision, "l2": "flushed between steps (256 MB write)",
                       "local_gemm_tile": f"128x{dd.dd_query(mixed.ctx)['gemm_tile_n']}",
                       "parallelism": f"replicas x{world}"},
            "time_to_ground_state_ms": {"mixed": step_ms, "fp64_plain": fp64_ms,
                                        "speedup_mixed_vs_fp64": fp64_ms / step_ms,
                                        "from_dd_setup": from_setup},
            "alu_peaks": alu,
            "lambda": lam, "sigma": sigma, "outer_iters": outer, "inner_iters_total": inner_tot,
            "fp64_plain": {"lambda": res64[0], "outer_iters": res64[2], "inner_iters_total": res64[3]},
            "pcg_iters_per_s": inner_tot / (step_ms / 1e3),
            "si_lopcg_time_to_ground_state": lopcg,
            "differentiable": grad_line,
            "batched": batch_line,
            "d3": d3_line,
            "sweeps": sweep_line,
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
