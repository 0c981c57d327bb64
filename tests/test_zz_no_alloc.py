"""GPU test of wp_wprod_noalloc, the w-product entry point for callers that
cannot allocate device memory (plain C hosts without a device allocator, or
plug-ins whose host application owns every device allocation).  It must give
the same result as wp_wprod, which takes a caller-allocated workspace, on
consecutive calls that reuse the library's one scratch array: both run the
same kernels on the same workspace layout, so the results must agree bit for
bit (a partial read of a previous call's leftovers would show up here).  The
first result is also checked against the FP64 oracle at the product
tolerance, and requests that do not fit in the array must be refused.

This file is named so that pytest collects it last."""

import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_08228_gb300 import capi, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the product tolerance used by the other parity tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2601_08228_gb300 import build
    build.build()
    capi.lib()


def _call_noalloc(A, B, C, n1, n2, n4, p, L, prec):
    """Call the entry point directly through the C ABI."""
    return capi.lib().wp_wprod_noalloc(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                       ctypes.c_void_p(C.data_ptr()), n1, n2, n4, p, L, 0, 0,
                                       capi.PREC[prec], capi._stream())


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_noalloc_matches_wprod_on_consecutive_calls(prec):
    cases = [(32, 32, 32, 16, 2, 0), (48, 40, 24, 24, 3, 1)]   # n1, n2, n4, p, L, seed
    for i, (n1, n2, n4, p, L, seed) in enumerate(cases):   # two calls in a row, different shapes and data
        A_h, B_h = synth.plain_pair(n1, n2, n4, p, seed=seed, dtype=np.float32)
        A, B = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
        C = torch.empty((p, n1, n4), dtype=torch.float32, device="cuda")
        assert _call_noalloc(A, B, C, n1, n2, n4, p, L, prec) == capi.WP_OK
        ref = capi.wp_wprod(A, B, L, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(C, ref)
        if i == 0:
            C64 = C.cpu().numpy().astype(np.float64)
            assert O.rel_fro(C64, O.wprod(A_h.astype(np.float64), B_h.astype(np.float64), L)) <= TOL
    # the same shape twice in a row: the second call must not see the first's data
    A_h, B_h = synth.plain_pair(32, 32, 32, 16, seed=7, dtype=np.float32)
    A, B = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
    C = torch.empty((16, 32, 32), dtype=torch.float32, device="cuda")
    assert _call_noalloc(A, B, C, 32, 32, 32, 16, 2, prec) == capi.WP_OK
    ref = capi.wp_wprod(A, B, 2, prec=prec)
    torch.cuda.synchronize()
    assert torch.equal(C, ref)
    assert capi.wp_get_device_error() == capi.WP_OK


def test_noalloc_rejects_oversized_requests():
    A = torch.zeros((192, 256, 256), device="cuda")
    C = torch.empty_like(A)
    status = _call_noalloc(A, A, C, 256, 256, 256, 192, 3, "fp32")
    assert status == capi.WP_ERR_WORKSPACE   # the request needs more than the scratch array
