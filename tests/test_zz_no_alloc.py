"""Allocation-free tensor-core product against the allocating entry point.

dd_tc_gemm_noalloc serves callers that cannot allocate device memory where they need
the product (a server whose device memory sits in an arena reserved at start-up, or a
latency-critical path where cudaMalloc/cudaFree would synchronise the device).  It
must give the same result as dd_tc_gemm_test, which allocates its own buffers and runs
the same kernel.  Small integer operands make both products exact, so the two must
agree bit for bit; each case runs two calls in a row because the calls share one
static scratch array that keeps the previous call's contents.
"""
import ctypes

import numpy as np
import pytest

import paper_2311_08757_gb300 as dd

pytestmark = pytest.mark.gpu


def _operands(M, N, K, seed):
    rng = np.random.default_rng(seed)
    A = rng.integers(-8, 9, size=(M, K)).astype(np.float32)
    B = rng.integers(-8, 9, size=(N, K)).astype(np.float32)
    return A, B


@pytest.mark.parametrize("prec", [dd.DD_PREC_BF16, dd.DD_PREC_TF32])
def test_noalloc_matches_allocating_entry_point(prec):
    import torch
    dt = torch.bfloat16 if prec == dd.DD_PREC_BF16 else torch.float32
    for call, (M, N, K) in enumerate([(300, 700, 192), (1209, 517, 1216)]):
        A, B = _operands(M, N, K, seed=100 + call)
        ref = np.zeros((N, M), dtype=np.float32)
        dd.dd_tc_gemm_test(prec, A, B, ref)
        Ad = torch.from_numpy(A).to("cuda").to(dt).contiguous()
        Bd = torch.from_numpy(B).to("cuda").to(dt).contiguous()
        for _ in range(2):
            D = torch.full((N, M), float("nan"), dtype=torch.float32, device="cuda")
            dd.dd_tc_gemm_noalloc(prec, Ad, Bd, D)
            torch.cuda.synchronize()
            assert np.array_equal(D.cpu().numpy(), ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    A = torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda")
    D = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
    f = dd.lib().dd_tc_gemm_noalloc
    # 65 x 64 output tiles exceed the 4096 tiles of the fixed scratch
    rc = f(dd.DD_PREC_BF16, 128 * 65, 256 * 64, 64, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(A.data_ptr()),
           ctypes.c_void_p(D.data_ptr()), None)
    assert rc == dd.DD_EINVAL
    rc = f(dd.DD_PREC_BF16, 128, 128, 100, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(A.data_ptr()),
           ctypes.c_void_p(D.data_ptr()), None)
    assert rc == dd.DD_EINVAL
