"""GPU parity of wp_wprod_host (host buffers; chunks of whole tube groups
copied in, multiplied and copied back on overlapping streams): the result is
bit-identical to wp_wprod on device copies of the same tensors and within
the precision's bar of the FP64 oracle, for chunks that split the slices
unevenly, a single chunk, pageable host memory and the benchmark shape."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_08228_gb300 import capi, synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x3": 1e-5, "bf16": 1e-2}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2601_08228_gb300 import build
    build.build()
    capi.lib()


def rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(size=shape).astype(np.float32)


@pytest.mark.parametrize("p,n1,n2,n4,L,chunk,prec,pinned", [
    (40, 33, 20, 17, 2, 12, "fp32", True),      # 4 chunks, the last one short (4 slices)
    (64, 64, 48, 80, 3, 16, "bf16x3", True),    # fused tensor-core path per chunk
    (24, 9, 7, 5, 3, 0, "bf16", True),          # default chunk (one tube group each)
    (16, 32, 32, 32, 4, 16, "fp32", False),     # one chunk, pageable host memory
    (8, 5, 6, 7, 0, 3, "bf16x3", True),         # L = 0: chunks of any size
])
def test_wprod_host_matches_device_call_and_oracle(p, n1, n2, n4, L, chunk, prec, pinned):
    A, B = rand((p, n1, n2), 31), rand((p, n2, n4), 32)
    Ah, Bh = torch.from_numpy(A), torch.from_numpy(B)
    if pinned:
        Ah, Bh = Ah.pin_memory(), Bh.pin_memory()
    C = capi.wp_wprod_host(Ah, Bh, L, prec=prec, chunk_slices=chunk)
    torch.cuda.synchronize()
    Cd = capi.wp_wprod(Ah.cuda(), Bh.cuda(), L, prec=prec)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(C.numpy(), Cd.cpu().numpy())
    assert O.rel_fro(C.numpy().astype(np.float64), O.wprod(A.astype(np.float64), B.astype(np.float64), L)) <= TOL[prec]
    assert capi.wp_get_device_error() == 0


def test_wprod_host_benchmark_shape_sampled():
    """256 x 256 x 192, L = 3, BF16x3 (the benchmark's end-to-end call): four
    sampled tube groups against the oracle, all of C against the device call."""
    A = synth.hsi_cube(256, 256, 192, seed=0, dtype=np.float32)
    B = synth.hsi_cube(256, 256, 192, seed=1, dtype=np.float32)
    Ah, Bh = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
    C = capi.wp_wprod_host(Ah, Bh, 3, prec="bf16x3")
    torch.cuda.synchronize()
    Cd = capi.wp_wprod(Ah.cuda(), Bh.cuda(), 3, prec="bf16x3")
    np.testing.assert_array_equal(C.numpy(), Cd.cpu().numpy())
    for g in (0, 7, 13, 23):
        s = slice(8 * g, 8 * g + 8)
        ref = O.wprod(A[s].astype(np.float64), B[s].astype(np.float64), 3)
        assert O.rel_fro(C.numpy()[s].astype(np.float64), ref) <= 1e-5


def test_wprod_host_rejects_device_tensors():
    with pytest.raises(ValueError):
        capi.wp_wprod_host(torch.zeros((8, 4, 4), device="cuda"), torch.zeros((8, 4, 4)), 3)
