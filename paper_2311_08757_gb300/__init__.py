"""Python binding of ``libddeig`` (ctypes; argument marshalling only).

Every function here has the name and argument order of the C entry point in
``include/ddeig.h`` and forwards to it; all arithmetic runs in the library's CUDA
kernels.  Vector arguments may be CUDA tensors (device pointers are passed through)
or host arrays (numpy arrays or CPU tensors, staged by the library).  A failing call
raises :class:`DDError` carrying the status code and the library's message.

The library is built in-tree by ``__graft_entry__.build()`` (or
``python -m paper_2311_08757_gb300._build``); importing this package does not load
it, the first call does, and fails loudly if it is missing.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_longlong, c_size_t, c_void_p

from . import _build

DD_OK, DD_EINVAL, DD_ESTATE, DD_ENOMEM, DD_ECUDA, DD_ENAN, DD_ENOTSPD, DD_EMAXIT, DD_ETIMEOUT, \
    DD_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
DD_PREC_FP64, DD_PREC_TF32, DD_PREC_BF16, DD_PREC_FP8 = 0, 1, 2, 3
DD_PU_EQUAL, DD_PU_DISTANCE = 0, 1
DD_OP_ASIGMA, DD_OP_MASS, DD_OP_A = 0, 1, 2
DD_OPT_CHECK_EVERY, DD_OPT_USE_GRAPH, DD_OPT_FLEXIBLE, DD_OPT_TIMING, DD_OPT_LOCAL_RHS = 0, 1, 2, 3, 4
DD_OPT_KRYLOV, DD_OPT_PRECOND, DD_OPT_RESTART, DD_OPT_GEMM_TILE_N, DD_OPT_COARSE_SOLVE = 5, 6, 7, 8, 9
DD_OPT_FUSED_PQ, DD_OPT_PROLONG_TABLES, DD_OPT_PAIRS, DD_OPT_PDL, DD_OPT_FUSE_XR, DD_OPT_TILED3 = 10, 11, 12, 13, 14, 15
DD_OPT_X_LAG = 16
PRECISIONS = {"fp64": DD_PREC_FP64, "tf32": DD_PREC_TF32, "bf16": DD_PREC_BF16, "fp8": DD_PREC_FP8}
DD_INNER_FIXED, DD_INNER_ADAPTIVE, DD_INNER_FUSED = 0, 1, 2
INNER_MODES = {"fixed": DD_INNER_FIXED, "adaptive": DD_INNER_ADAPTIVE, "fused": DD_INNER_FUSED}


class dd_grid(ctypes.Structure):
    _fields_ = [("p", c_int), ("q", c_int), ("L", c_int), ("ell", c_double), ("n", c_int),
                ("overlap", c_int), ("quad_pts", c_int), ("pu_kind", c_int), ("precision", c_int),
                ("coarse", c_int)]


class dd_info(ctypes.Structure):
    _fields_ = [("ndof", c_longlong), ("ncell", c_longlong), ("nsub", c_int), ("ntypes", c_int),
                ("nloc_max", c_int), ("kpad", c_int), ("band_local", c_int), ("sigma", c_double),
                ("cell_iters", c_int), ("stage", c_int), ("device_bytes", c_longlong), ("gemm_tile_n", c_int),
                ("reserved_", c_int)]


class DDError(RuntimeError):
    def __init__(self, code: int, message: str):
        self.code = code
        super().__init__(f"{status_string(code)}: {message}")


_lib = None

_SIGS = {
    "dd_setup": (c_int, [POINTER(dd_grid), c_void_p, c_size_t, c_void_p, POINTER(c_void_p)]),
    "dd_cell_eigenpair": (c_int, [c_void_p, POINTER(c_double), c_void_p]),
    "dd_coarse_build": (c_int, [c_void_p]),
    "dd_pcg_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, POINTER(c_int), POINTER(c_double)]),
    "dd_inverse_iterate": (c_int, [c_void_p, c_void_p, c_double, c_double, c_int, c_double, POINTER(c_double),
                                   POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "dd_potential_gradient": (c_int, [c_void_p, c_void_p, c_double, c_double, c_void_p, c_double, c_void_p,
                                      c_size_t, POINTER(c_int)]),
    "dd_gmres_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, POINTER(c_int), POINTER(c_double)]),
    "dd_batch_create": (c_int, [POINTER(dd_grid), POINTER(c_void_p), POINTER(c_size_t), c_int, c_void_p,
                                POINTER(c_void_p)]),
    "dd_batch_ground_states": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dd_batch_size": (c_int, [c_void_p]),
    "dd_batch_info": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int),
                              POINTER(c_double), POINTER(c_double)]),
    "dd_batch_set_groups": (c_int, [c_void_p, c_int]),
    "dd_batch_context": (c_void_p, [c_void_p, c_int]),
    "dd_batch_destroy": (None, [c_void_p]),
    "dd_lopcg": (c_int, [c_void_p, c_void_p, c_int, c_double, c_double, c_int, c_double, POINTER(c_double),
                         POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "dd_eigenpair": (c_int, [POINTER(dd_grid), c_void_p, c_size_t, c_void_p, POINTER(c_double), c_void_p,
                             POINTER(c_double)]),
    "dd_destroy": (None, [c_void_p]),
    "dd_status_string": (c_char_p, [c_int]),
    "dd_last_error": (c_char_p, [c_void_p]),
    "dd_query": (c_int, [c_void_p, POINTER(dd_info)]),
    "dd_apply_operator": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "dd_apply_asigma_pairs": (c_int, [c_void_p, c_void_p, c_void_p]),
    "dd_apply_preconditioner": (c_int, [c_void_p, c_void_p, c_void_p]),
    "dd_coarse_matrix": (c_int, [c_void_p, c_void_p]),
    "dd_set_option": (c_int, [c_void_p, c_int, c_int]),
    "dd_kernel_timings": (c_int, [c_void_p, POINTER(c_int), POINTER(c_char_p), POINTER(c_longlong),
                                  POINTER(c_double)]),
    "dd_reset_timings": (c_int, [c_void_p]),
    "dd_tc_gemm_test": (c_int, [c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "dd_convert_test": (c_int, [c_int, c_longlong, c_void_p, c_void_p]),
    "dd_set_potential": (c_int, [c_void_p, c_void_p, c_size_t]),
    "dd_kernel_launch_count": (c_longlong, []),
    "dd_tc_gemm_noalloc": (c_int, [c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dd_alu_peak_test": (c_int, [c_int, c_int, POINTER(c_double)]),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load ``libddeig.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().dd_status_string(code).decode()


def _check(code: int, ctx=None, allow=()):
    if code != DD_OK and code not in allow:
        msg = lib().dd_last_error(ctx).decode()
        raise DDError(code, msg)
    return code


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (contiguous float64), or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return c_void_p(a.data_ptr())
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return c_void_p(stream)
    return c_void_p(stream.cuda_stream)


def make_grid(p=1, L=1, n=16, ell=1.0, overlap=1, quad_pts=2, pu_kind=DD_PU_EQUAL, precision=DD_PREC_FP64,
              coarse=1) -> dd_grid:
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    return dd_grid(p=p, q=1, L=L, ell=ell, n=n, overlap=overlap, quad_pts=quad_pts, pu_kind=pu_kind,
                   precision=precision, coarse=coarse)


def grid_from_workload(w, precision=DD_PREC_FP64, coarse=1, pu_kind=DD_PU_EQUAL) -> dd_grid:
    return make_grid(p=w.p, L=w.L, n=w.n, ell=w.ell, overlap=w.overlap, quad_pts=w.quad_pts,
                     pu_kind=pu_kind, precision=precision, coarse=coarse)


# ---- entry points (names of include/ddeig.h) ------------------------------------------

def dd_setup(grid: dd_grid, V_cell_qp, stream=None) -> c_void_p:
    ctx = c_void_p()
    n = V_cell_qp.numel() if hasattr(V_cell_qp, "numel") else V_cell_qp.size
    _check(lib().dd_setup(byref(grid), _ptr(V_cell_qp), n, _stream_ptr(stream), byref(ctx)))
    return ctx


def dd_set_potential(ctx, V_cell_qp) -> None:
    n = V_cell_qp.numel() if hasattr(V_cell_qp, "numel") else V_cell_qp.size
    _check(lib().dd_set_potential(ctx, _ptr(V_cell_qp), n), ctx)


def dd_kernel_launch_count() -> int:
    return int(lib().dd_kernel_launch_count())


def dd_cell_eigenpair(ctx, psi_cell_out=None) -> float:
    s = c_double()
    _check(lib().dd_cell_eigenpair(ctx, byref(s), _ptr(psi_cell_out)), ctx)
    return s.value


def dd_coarse_build(ctx) -> None:
    _check(lib().dd_coarse_build(ctx), ctx)


def dd_pcg_solve(ctx, b, x, rtol=1e-8, maxit=10000, allow_maxit=False):
    it, rel = c_int(), c_double()
    _check(lib().dd_pcg_solve(ctx, _ptr(b), _ptr(x), rtol, maxit, byref(it), byref(rel)), ctx,
           allow=(DD_EMAXIT,) if allow_maxit else ())
    return it.value, rel.value


def dd_gmres_solve(ctx, b, x, rtol=1e-8, maxit=10000):
    it, rel = c_int(), c_double()
    _check(lib().dd_gmres_solve(ctx, _ptr(b), _ptr(x), rtol, maxit, byref(it), byref(rel)), ctx)
    return it.value, rel.value


def dd_inverse_iterate(ctx, x, tol_res=1e-8, tol_lam=1e-10, maxit_outer=100, rtol_inner=1e-8):
    lam, outer, tot, mx = c_double(), c_int(), c_int(), c_int()
    _check(lib().dd_inverse_iterate(ctx, _ptr(x), tol_res, tol_lam, maxit_outer, rtol_inner, byref(lam),
                                    byref(outer), byref(tot), byref(mx)), ctx)
    return lam.value, outer.value, tot.value, mx.value


def dd_lopcg(ctx, x, inner="fused", tol_res=1e-8, tol_lam=1e-10, maxit_outer=1000, rtol_inner=1e-8):
    """SI-LOPCG (Algorithm 1); ``inner`` is "fixed", "adaptive" or "fused" (or its code)."""
    mode = INNER_MODES[inner] if isinstance(inner, str) else int(inner)
    lam, outer, tot, mx = c_double(), c_int(), c_int(), c_int()
    _check(lib().dd_lopcg(ctx, _ptr(x), mode, tol_res, tol_lam, maxit_outer, rtol_inner, byref(lam), byref(outer),
                          byref(tot), byref(mx)), ctx)
    return lam.value, outer.value, tot.value, mx.value


def dd_potential_gradient(ctx, phi, lam, g_lambda, g_phi, dV, rtol=1e-10) -> int:
    """dV = g_lambda d(lambda)/dV_cell_qp + dl/dV_cell_qp (adjoint term when g_phi is given);
    returns the adjoint PCG iteration count."""
    it = c_int()
    n = dV.numel() if hasattr(dV, "numel") else dV.size
    _check(lib().dd_potential_gradient(ctx, _ptr(phi), float(lam), float(g_lambda), _ptr(g_phi), rtol, _ptr(dV), n,
                                       byref(it)), ctx)
    return it.value


def dd_eigenpair(grid: dd_grid, V_cell_qp, stream=None, phi_out=None):
    lam, sig = c_double(), c_double()
    n = V_cell_qp.numel() if hasattr(V_cell_qp, "numel") else V_cell_qp.size
    _check(lib().dd_eigenpair(byref(grid), _ptr(V_cell_qp), n, _stream_ptr(stream), byref(lam), _ptr(phi_out),
                              byref(sig)))
    return lam.value, sig.value


def dd_destroy(ctx) -> None:
    if ctx:
        lib().dd_destroy(ctx)


def dd_query(ctx) -> dict:
    info = dd_info()
    _check(lib().dd_query(ctx, byref(info)), ctx)
    return {k: getattr(info, k) for k, _ in dd_info._fields_}


def dd_apply_operator(ctx, op: int, x, y) -> None:
    _check(lib().dd_apply_operator(ctx, op, _ptr(x), _ptr(y)), ctx)


def dd_apply_asigma_pairs(ctx, x, y) -> None:
    """y = A_sigma x by the float-pair pass of the PCG iteration (see the header)."""
    _check(lib().dd_apply_asigma_pairs(ctx, _ptr(x), _ptr(y)), ctx)


def dd_apply_preconditioner(ctx, r, z) -> None:
    _check(lib().dd_apply_preconditioner(ctx, _ptr(r), _ptr(z)), ctx)


def dd_coarse_matrix(ctx, A0_host) -> None:
    _check(lib().dd_coarse_matrix(ctx, _ptr(A0_host)), ctx)


def dd_set_option(ctx, option: int, value: int) -> None:
    _check(lib().dd_set_option(ctx, option, value), ctx)


def dd_kernel_timings(ctx) -> dict:
    cnt = c_int()
    _check(lib().dd_kernel_timings(ctx, byref(cnt), None, None, None), ctx)
    n = cnt.value
    names = (c_char_p * n)()
    launches = (c_longlong * n)()
    ms = (c_double * n)()
    _check(lib().dd_kernel_timings(ctx, byref(cnt), names, launches, ms), ctx)
    return {names[k].decode(): (launches[k], ms[k]) for k in range(n)}


def dd_reset_timings(ctx) -> None:
    _check(lib().dd_reset_timings(ctx), ctx)


def _require(cond: bool, msg: str) -> None:
    if not cond:
        raise ValueError(msg)


def dd_tc_gemm_test(precision: int, A, B, D) -> int:
    """D[n][m] = sum_k A[m][k] B[n][k] (host float32 arrays) through the tensor-core kernel."""
    import numpy as np
    for name, a in (("A", A), ("B", B), ("D", D)):
        _require(isinstance(a, np.ndarray) and a.dtype == np.float32 and a.ndim == 2 and a.flags["C_CONTIGUOUS"],
                 f"{name} must be a C-contiguous 2-D float32 numpy array")
    M, K = A.shape
    N = B.shape[0]
    _require(B.shape == (N, K), f"B must be N x K = {N} x {K}, got {B.shape}")
    _require(D.shape == (N, M), f"D must be N x M = {N} x {M}, got {D.shape}")
    return _check(lib().dd_tc_gemm_test(precision, M, N, K, _ptr(A), _ptr(B), _ptr(D)))


def dd_convert_test(kind: int, x):
    """Device precision conversions on a host array: kind 0 float64 -> BF16 bits (uint16),
    1 float64 -> TF32 (float32), 2 float32 -> float64."""
    import numpy as np
    x = np.ascontiguousarray(x, dtype=np.float32 if kind == 2 else np.float64)
    out = np.zeros(x.size, dtype={0: np.uint16, 1: np.float32, 2: np.float64}[kind])
    _check(lib().dd_convert_test(kind, x.size, _ptr(x), _ptr(out)))
    return out


def dd_alu_peak_test(kind: int, reps: int = 5) -> float:
    """Measured FMA throughput of the GPU (TFLOP/s): kind 0 FP64, kind 1 FP32."""
    t = c_double()
    _check(lib().dd_alu_peak_test(kind, reps, byref(t)))
    return t.value


def dd_tc_gemm_noalloc(precision: int, A_dev, B_dev, D_dev, stream=None) -> int:
    """Allocation-free tensor-core product D[n][m] = sum_k A[m][k] B[n][k] on device tensors
    (A: M x K, B: N x K, BF16 or FP32/TF32, K a multiple of 64; D: N x M float32).  For callers
    that must not allocate device memory; its scratch is fixed static device memory shared by
    all calls, so overlapping calls race.  Not to be called while its stream is being captured
    into a CUDA graph: every call synchronises the stream and copies its tile list from host
    memory.  Shapes, types and devices are checked here before the library is called."""
    import torch
    _require(precision in (DD_PREC_BF16, DD_PREC_TF32), "precision must be DD_PREC_BF16 or DD_PREC_TF32")
    want = torch.bfloat16 if precision == DD_PREC_BF16 else torch.float32
    for name, a, dt in (("A", A_dev, want), ("B", B_dev, want), ("D", D_dev, torch.float32)):
        _require(isinstance(a, torch.Tensor) and a.dim() == 2 and a.is_contiguous(),
                 f"{name} must be a contiguous 2-D torch tensor")
        _require(a.dtype == dt, f"{name} must be {dt}, got {a.dtype}")
        _require(a.is_cuda, f"{name} must be in device memory")
        _require(a.device.index == torch.cuda.current_device(), f"{name} must be on the current device")
    M, K = A_dev.shape
    N = B_dev.shape[0]
    _require(tuple(B_dev.shape) == (N, K), f"B must be N x K = {N} x {K}, got {tuple(B_dev.shape)}")
    _require(tuple(D_dev.shape) == (N, M), f"D must be N x M = {N} x {M}, got {tuple(D_dev.shape)}")
    return _check(lib().dd_tc_gemm_noalloc(precision, M, N, K, _ptr(A_dev), _ptr(B_dev), _ptr(D_dev),
                                           _stream_ptr(stream)))


class Eigensolver:
    """Owns a context: set-up, cell eigenpair, coarse build; ``ground_state`` runs
    the inverse iteration.  Thin convenience over the entry points above."""

    def __init__(self, grid: dd_grid, V_cell_qp, stream=None):
        self.ctx = dd_setup(grid, V_cell_qp, stream)
        self.grid = grid

    def close(self):
        if self.ctx:
            dd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def info(self) -> dict:
        return dd_query(self.ctx)

    def prepare(self):
        sigma = dd_cell_eigenpair(self.ctx)
        dd_coarse_build(self.ctx)
        return sigma

    def ground_state(self, x, **kw):
        return dd_inverse_iterate(self.ctx, x, **kw)

    def ground_state_lopcg(self, x, inner="fused", **kw):
        return dd_lopcg(self.ctx, x, inner, **kw)


DD_BATCH_IPM, DD_BATCH_LOPCG_FUSED, DD_BATCH_LOPCG_ADAPTIVE, DD_BATCH_IPM_CONCURRENT = 0, 1, 2, 3
BATCH_METHODS = {"ipm": DD_BATCH_IPM, "lopcg_fused": DD_BATCH_LOPCG_FUSED, "lopcg_adaptive": DD_BATCH_LOPCG_ADAPTIVE,
                 "ipm_concurrent": DD_BATCH_IPM_CONCURRENT}


class Batch:
    """Many independent ground-state problems solved concurrently (dd_batch_*)."""

    def __init__(self, grids, potentials, stream=None):
        import numpy as np
        n = len(grids)
        self._grids = (dd_grid * n)(*grids)
        self._V = list(potentials)               # keep the buffers alive during set-up
        ptrs = (c_void_p * n)(*[_ptr(v).value for v in self._V])
        sizes = (c_size_t * n)(*[(v.numel() if hasattr(v, "numel") else v.size) for v in self._V])
        h = c_void_p()
        code = lib().dd_batch_create(self._grids, ptrs, sizes, n, _stream_ptr(stream), byref(h))
        if code != DD_OK:
            raise DDError(code, lib().dd_last_error(None).decode())
        self.handle = h
        self.count = n
        self._np = np

    def context(self, i):
        return c_void_p(lib().dd_batch_context(self.handle, i))

    def ground_states(self, method="ipm", threads=0, phi=None):
        """Returns dict of per-instance arrays (lambda, outer, inner, seconds); phi: optional list
        of output buffers (host or device), one per instance."""
        np = self._np
        n = self.count
        lam = np.zeros(n)
        outer = np.zeros(n, dtype=np.int32)
        inner = np.zeros(n, dtype=np.int32)
        sec = np.zeros(n)
        phis = (c_void_p * n)(*[(_ptr(p).value if p is not None else None) for p in phi]) if phi is not None else None
        code = lib().dd_batch_ground_states(self.handle, BATCH_METHODS[method] if isinstance(method, str) else method,
                                            threads, c_void_p(lam.ctypes.data), phis,
                                            c_void_p(outer.ctypes.data), c_void_p(inner.ctypes.data),
                                            c_void_p(sec.ctypes.data))
        if code != DD_OK:
            raise DDError(code, "batched ground states failed")
        return {"lambda": lam, "outer": outer, "inner": inner, "seconds": sec}

    def info(self) -> dict:
        """dd_batch_info: batchable, last_batched, gemm_tile_n, groups, setup_seconds, total_seconds."""
        v = [c_int() for _ in range(4)] + [c_double(), c_double()]
        _check(lib().dd_batch_info(self.handle, *[byref(x) for x in v]))
        return dict(zip(("batchable", "last_batched", "gemm_tile_n", "groups", "setup_seconds",
                         "total_seconds"), (x.value for x in v)))

    def set_groups(self, groups: int) -> None:
        """dd_batch_set_groups: instances split into this many batched groups (0: chosen by timing)."""
        _check(lib().dd_batch_set_groups(self.handle, groups))

    def close(self):
        if getattr(self, "handle", None):
            lib().dd_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
