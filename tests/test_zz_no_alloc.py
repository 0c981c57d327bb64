"""GPU test of wp_wprod_noalloc, the w-product entry point for callers that
cannot allocate device memory (plain C hosts without a device allocator, or
plug-ins whose host application owns every device allocation).  It must give
the same result as wp_wprod, which takes a caller-allocated workspace, on
consecutive calls that reuse the library's one scratch array, and must
refuse requests that do not fit in that array.

This file is named so that pytest collects it last."""

import ctypes

import numpy as np
import pytest
import torch

from paper_2601_08228_gb300 import capi, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the product tolerance used by the other parity tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2601_08228_gb300 import build
    build.build()
    capi.lib()


def _rel(x, ref):
    x, ref = x.double(), ref.double()
    return float(torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref))


def _call_noalloc(A, B, C, n1, n2, n4, p, L, prec):
    """Call the entry point directly through the C ABI."""
    return capi.lib().wp_wprod_noalloc(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                       ctypes.c_void_p(C.data_ptr()), n1, n2, n4, p, L, 0, 0,
                                       capi.PREC[prec], capi._stream())


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_noalloc_matches_wprod_on_consecutive_calls(prec):
    cases = [(32, 32, 32, 16, 2, 0), (48, 40, 24, 24, 3, 1)]   # n1, n2, n4, p, L, seed
    for n1, n2, n4, p, L, seed in cases:     # two calls in a row, different shapes and data
        A_h, B_h = synth.plain_pair(n1, n2, n4, p, seed=seed, dtype=np.float32)
        A, B = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
        C = torch.empty((p, n1, n4), dtype=torch.float32, device="cuda")
        assert _call_noalloc(A, B, C, n1, n2, n4, p, L, prec) == 0
        ref = capi.wp_wprod(A, B, L, prec=prec)
        torch.cuda.synchronize()
        assert _rel(C, ref) <= TOL
    # the same shape twice in a row: the second call must not see the first's data
    A_h, B_h = synth.plain_pair(32, 32, 32, 16, seed=7, dtype=np.float32)
    A, B = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
    C = torch.empty((16, 32, 32), dtype=torch.float32, device="cuda")
    assert _call_noalloc(A, B, C, 32, 32, 32, 16, 2, prec) == 0
    torch.cuda.synchronize()
    assert _rel(C, capi.wp_wprod(A, B, 2, prec=prec)) <= TOL
    assert capi.wp_get_device_error() == 0


def test_noalloc_rejects_oversized_requests():
    A = torch.zeros((192, 256, 256), device="cuda")
    C = torch.empty_like(A)
    status = _call_noalloc(A, A, C, 256, 256, 256, 192, 3, "fp32")
    assert status == 7   # WP_ERR_WORKSPACE: the request needs more than the scratch array
