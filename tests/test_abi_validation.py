"""Argument checking at the C ABI, which needs no GPU: every entry point below rejects a bad
argument with DD_EINVAL (and, for dd_setup, a message) before it touches the device, as
include/ddeig.h states.  A valid problem on a machine without a GPU fails with DD_ECUDA."""
import ctypes
import os

import numpy as np
import pytest

import paper_2311_08757_gb300 as dd
from paper_2311_08757_gb300 import _build


@pytest.fixture(scope="module", autouse=True)
def built():
    if not os.path.exists(dd.lib_path()):
        _build.build()


def _v(g):
    """A cell potential of the size dd_setup expects for grid g (n^p ny Q^(p+1) values)."""
    ny = int(round(g.ell * g.n))
    return np.ones(ny * g.n ** g.p * g.quad_pts ** (g.p + 1))


def _setup_fails(g, V=None, match=None):
    with pytest.raises(dd.DDError) as e:
        dd.dd_setup(g, _v(g) if V is None else V)
    assert e.value.code == dd.DD_EINVAL
    if match:
        assert match in str(e.value)


@pytest.mark.parametrize("field,value,match", [
    ("p", 0, "p must be 1 or 2"),
    ("p", 3, "p must be 1 or 2"),
    ("q", 2, "q must be 1"),
    ("L", 0, "L must be >= 1"),
    ("n", 2, "n must be >= 3"),
    ("ell", 1.03, "ell * n must be an integer"),
    ("overlap", 0, "overlap"),
    ("overlap", 8, "overlap"),            # 2 overlap >= n = 16
    ("quad_pts", 0, "quad_pts"),
    ("quad_pts", 5, "quad_pts"),
    ("pu_kind", 7, "pu_kind"),
    ("precision", 9, "precision"),
    ("coarse", 2, "coarse"),
])
def test_setup_rejects_each_bad_grid_field(field, value, match):
    g = dd.make_grid(p=1, L=4, n=16, overlap=2)
    setattr(g, field, value)
    V = _v(dd.make_grid(p=1, L=4, n=16, overlap=2)) if field in ("p", "ell", "quad_pts", "n") else None
    _setup_fails(g, V, match)


def test_setup_rejects_wrong_potential_size_and_huge_grids():
    g = dd.make_grid(p=1, L=4, n=16, overlap=2)
    _setup_fails(g, _v(g)[:-1], "nV does not match")
    big = dd.make_grid(p=2, L=10000, n=16, overlap=2)   # (160001)^2 columns x 16 slots > 2^31
    _setup_fails(big, None, "grid too large")


def test_setup_rejects_null_arguments():
    L = dd.lib()
    g = dd.make_grid(p=1, L=4, n=16, overlap=2)
    ctx = ctypes.c_void_p()
    assert L.dd_setup(ctypes.byref(g), None, 0, None, ctypes.byref(ctx)) == dd.DD_EINVAL
    V = _v(g)
    assert L.dd_setup(None, V.ctypes.data_as(ctypes.c_void_p), V.size, None, ctypes.byref(ctx)) == dd.DD_EINVAL
    assert not ctx.value


def test_one_shot_eigenpair_validates_like_setup():
    g = dd.make_grid(p=1, L=4, n=16, overlap=0)
    V = _v(g)
    lam = ctypes.c_double()
    rc = dd.lib().dd_eigenpair(ctypes.byref(g), V.ctypes.data_as(ctypes.c_void_p), V.size, None,
                               ctypes.byref(lam), None, None)
    assert rc == dd.DD_EINVAL


def test_status_strings():
    names = {dd.DD_OK: "DD_OK", dd.DD_EINVAL: "DD_EINVAL", dd.DD_ESTATE: "DD_ESTATE",
             dd.DD_ENOMEM: "DD_ENOMEM", dd.DD_ECUDA: "DD_ECUDA", dd.DD_ENAN: "DD_ENAN",
             dd.DD_ENOTSPD: "DD_ENOTSPD", dd.DD_EMAXIT: "DD_EMAXIT", dd.DD_ETIMEOUT: "DD_ETIMEOUT"}
    for code, name in names.items():
        assert dd.status_string(code) == name
    assert dd.status_string(12345) == "DD_UNKNOWN"


def test_options_need_a_context():
    assert dd.lib().dd_set_option(None, dd.DD_OPT_CHECK_EVERY, 8) == dd.DD_EINVAL


def test_operator_entry_points_need_a_context_and_buffers():
    L = dd.lib()
    buf = (ctypes.c_double * 4)()
    out = (ctypes.c_double * 4)()
    assert L.dd_apply_asigma_pairs(None, buf, out) == dd.DD_EINVAL
    assert L.dd_apply_asigma_pairs(None, None, out) == dd.DD_EINVAL
    assert L.dd_apply_operator(None, dd.DD_OP_ASIGMA, buf, out) == dd.DD_EINVAL


def test_self_test_entry_points_check_arguments_first():
    L = dd.lib()
    buf = (ctypes.c_double * 4)()
    out = (ctypes.c_double * 4)()
    assert L.dd_convert_test(3, 4, buf, out) == dd.DD_EINVAL     # no such conversion
    assert L.dd_convert_test(0, 0, buf, out) == dd.DD_EINVAL     # empty
    assert L.dd_convert_test(0, 4, None, out) == dd.DD_EINVAL
    t = ctypes.c_double()
    assert L.dd_alu_peak_test(2, 3, ctypes.byref(t)) == dd.DD_EINVAL     # no such pipe
    assert L.dd_alu_peak_test(0, 0, ctypes.byref(t)) == dd.DD_EINVAL     # no timed launch
    assert L.dd_alu_peak_test(1, 3, None) == dd.DD_EINVAL
    p = ctypes.c_void_p(16)   # never dereferenced: the checks come first
    f = ctypes.cast(p, ctypes.POINTER(ctypes.c_float))
    assert L.dd_tc_gemm_noalloc(dd.DD_PREC_FP64, 128, 128, 128, p, p, f, None) == dd.DD_EINVAL
    assert L.dd_tc_gemm_noalloc(dd.DD_PREC_BF16, 128, 128, 65, p, p, f, None) == dd.DD_EINVAL
    assert L.dd_tc_gemm_noalloc(dd.DD_PREC_BF16, 128, 128, 128, None, p, f, None) == dd.DD_EINVAL
    assert L.dd_tc_gemm_noalloc(dd.DD_PREC_BF16, 1 << 20, 1 << 20, 128, p, p, f, None) == dd.DD_EINVAL
    # sizes near INT_MAX: the tile count must not wrap around to a small or negative number
    imax = 2 ** 31 - 1
    assert L.dd_tc_gemm_noalloc(dd.DD_PREC_BF16, imax, imax, 128, p, p, f, None) == dd.DD_EINVAL
    assert L.dd_tc_gemm_noalloc(dd.DD_PREC_BF16, imax, 1, 128, p, p, f, None) == dd.DD_EINVAL
    assert L.dd_tc_gemm_noalloc(dd.DD_PREC_TF32, 1, imax, 128, p, p, f, None) == dd.DD_EINVAL
    assert L.dd_tc_gemm_test(dd.DD_PREC_BF16, imax, 8, 64, p, p, p) == dd.DD_EINVAL
    assert L.dd_tc_gemm_test(dd.DD_PREC_BF16, 8, 8, imax, p, p, p) == dd.DD_EINVAL


def test_gemm_wrappers_check_shapes_and_types_first():
    """The binding's tensor-core wrappers reject mismatched operands before the library is
    called: a wrong shape, type or device would make the kernel read or write out of bounds."""
    import numpy as np
    import torch
    A = np.zeros((128, 64), np.float32)
    with pytest.raises(ValueError):
        dd.dd_tc_gemm_test(dd.DD_PREC_BF16, A, np.zeros((8, 32), np.float32), np.zeros((8, 128), np.float32))
    with pytest.raises(ValueError):
        dd.dd_tc_gemm_test(dd.DD_PREC_BF16, A, np.zeros((8, 64), np.float32), np.zeros((8, 64), np.float32))
    with pytest.raises(ValueError):
        dd.dd_tc_gemm_test(dd.DD_PREC_BF16, A, np.zeros((8, 64), np.float64), np.zeros((8, 128), np.float32))
    At = torch.zeros(128, 64, dtype=torch.bfloat16)
    Bt = torch.zeros(8, 64, dtype=torch.bfloat16)
    Dt = torch.zeros(8, 128, dtype=torch.float32)
    with pytest.raises(ValueError):          # host tensors: the entry point takes device memory
        dd.dd_tc_gemm_noalloc(dd.DD_PREC_BF16, At, Bt, Dt)
    with pytest.raises(ValueError):          # precision without an allocation-free form
        dd.dd_tc_gemm_noalloc(dd.DD_PREC_FP8, At, Bt, Dt)


def test_no_cpu_fallback_without_a_gpu():
    """A valid problem on a machine without a GPU fails with DD_ECUDA: the library has no
    host path to fall back on."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from ddinputs import WORKLOADS, sample_cell_qp
    w = WORKLOADS["cfg1"]
    with pytest.raises(dd.DDError) as e:
        dd.dd_setup(dd.grid_from_workload(w), sample_cell_qp(w))
    assert e.value.code == dd.DD_ECUDA
    with pytest.raises(dd.DDError) as e:
        dd.dd_eigenpair(dd.grid_from_workload(w), sample_cell_qp(w))
    assert e.value.code == dd.DD_ECUDA
