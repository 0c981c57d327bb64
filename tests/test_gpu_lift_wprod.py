"""GPU parity: lifting transforms, FP32 face-products, w-product and its
backward, through the C ABI, against the FP64 oracle on the same seeded
inputs.  Tolerances: transforms 1e-6 relative Frobenius (a few FP32 roundings
per level); products and gradients 1e-5 (the stated product bar); the
worked example is bit-exact (dyadic rationals)."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_08228_gb300 import capi, synth
from tests import _golden

pytestmark = pytest.mark.gpu

TOL_LIFT = 1e-6
TOL_PROD = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2601_08228_gb300 import build
    build.build()
    capi.lib()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def rand(shape, seed):
    return np.random.default_rng(seed).uniform(-1, 1, size=shape).astype(np.float32)


LIFT_SHAPES = [
    (16, 32, 32, 2),     # 128-bit path
    (24, 17, 5, 3),      # ragged plane (85 elements): scalar path, m = 3
    (96, 6, 10, 5),      # L = 5: 64-bit path
    (64, 3, 7, 6),       # shared-memory path
    (384, 9, 33, 7),     # shared-memory path, m = 3, ragged plane
    (1024, 4, 8, 10),    # deepest supported level
    (7, 3, 4, 0),        # L = 0: identity
    (2, 1, 1, 1),        # single element
    (256, 64, 64, 4),    # several grid-stride rounds
]


@pytest.mark.parametrize("p,n1,n2,L", LIFT_SHAPES)
def test_lift_forward_inverse_adjoints(p, n1, n2, L):
    x = rand((p, n1, n2), p + L)
    xd = dev(x)
    assert O.rel_fro(host(capi.wp_lift_forward(xd, L)), O.lift(x, L)) <= TOL_LIFT
    assert O.rel_fro(host(capi.wp_lift_inverse(xd, L)), O.ilift(x, L)) <= TOL_LIFT
    assert O.rel_fro(host(capi.wp_lift_adjoint(xd, L)), O.lift_adjoint(x, L)) <= TOL_LIFT
    assert O.rel_fro(host(capi.wp_lift_adjoint(xd, L, of_inverse=True)), O.ilift_adjoint(x, L)) <= TOL_LIFT
    # perfect reconstruction on the GPU (Lemma 2.1), FP32 round trip
    assert O.rel_fro(host(capi.wp_lift_inverse(capi.wp_lift_forward(xd, L), L)), x) <= TOL_LIFT


def test_lift_example_2_2_bit_exact():
    ex = _golden.load("example_2_2.txt")
    for T in ("A", "B"):
        y = host(capi.wp_lift_forward(dev(ex[T]), 2))
        np.testing.assert_array_equal(y, O.lift(ex[T], 2))
        np.testing.assert_array_equal(y[0:1], ex[T + "_s2"])


def test_wprod_example_2_2_bit_exact():
    ex = _golden.load("example_2_2.txt")
    C = host(capi.wp_wprod(dev(ex["A"]), dev(ex["B"]), 2))
    np.testing.assert_array_equal(C, ex["C"])


def test_wprod_plain_32x32x16():
    """The plain case: A, B 32x32x16 iid U[-1, 1] from seed 0, L = 2."""
    A, B = synth.plain_pair(32, 32, 32, 16, seed=0)
    C = host(capi.wp_wprod(dev(A), dev(B), 2))
    assert O.rel_fro(C, O.wprod(A, B, 2)) <= TOL_PROD


PROD_CASES = [
    # p, n1, n2, n4, L
    (24, 33, 17, 45, 3),
    (64, 130, 129, 131, 4),   # several 128-wide tiles plus ragged tails
    (8, 1, 1, 1, 3),
    (12, 5, 300, 7, 2),       # long K
    (6, 20, 9, 11, 0),        # L = 0: plain batched product
    (96, 16, 24, 8, 5),
]


@pytest.mark.parametrize("p,n1,n2,n4,L", PROD_CASES)
@pytest.mark.parametrize("tA,tB", [(False, False), (True, False), (False, True), (True, True)])
def test_wprod_fp32_parity(p, n1, n2, n4, L, tA, tB):
    A = rand((p, n2, n1) if tA else (p, n1, n2), 1)
    B = rand((p, n4, n2) if tB else (p, n2, n4), 2)
    C = host(capi.wp_wprod(dev(A), dev(B), L, transA=tA, transB=tB))
    assert O.rel_fro(C, O.wprod(A, B, L, transA=tA, transB=tB)) <= TOL_PROD


def test_facewise_fp32_parity():
    Ah, Bh = rand((10, 70, 33), 3), rand((10, 33, 90), 4)
    C = host(capi.wp_facewise(dev(Ah), dev(Bh)))
    assert O.rel_fro(C, O.facewise(Ah, Bh)) <= TOL_PROD


@pytest.mark.parametrize("p,n1,n2,n4,L", [(8, 16, 16, 16, 3), (24, 33, 17, 45, 3), (64, 40, 70, 20, 4)])
def test_backward_fp32_parity(p, n1, n2, n4, L):
    A, B, G = rand((p, n1, n2), 5), rand((p, n2, n4), 6), rand((p, n1, n4), 7)
    dA, dB = capi.wp_wprod_backward(dev(A), dev(B), dev(G), L)
    rA, rB = O.wprod_grad(A, B, G, L)
    assert O.rel_fro(host(dA), rA) <= TOL_PROD
    assert O.rel_fro(host(dB), rB) <= TOL_PROD
    dA2, none = capi.wp_wprod_backward(dev(A), dev(B), dev(G), L, need_dB=False)
    assert none is None and O.rel_fro(host(dA2), rA) <= TOL_PROD


def test_backward_fd_crop_16x16x8():
    """Central finite differences (FP64, oracle forward) against the GPU
    gradient on a 16x16x8 crop, L = 3."""
    p, n, L = 8, 16, 3
    A, B, G = rand((p, n, n), 8), rand((p, n, n), 9), rand((p, n, n), 10)
    dA, dB = capi.wp_wprod_backward(dev(A), dev(B), dev(G), L)
    dA, dB = host(dA), host(dB)
    rng = np.random.default_rng(11)
    f = lambda a, b: float(np.sum(G * O.wprod(a, b, L)))
    for _ in range(3):
        EA, EB = rng.standard_normal(A.shape), rng.standard_normal(B.shape)
        h = 1e-3
        fd = (f(A + h * EA, B + h * EB) - f(A - h * EA, B - h * EB)) / (2 * h)
        an = np.sum(dA * EA) + np.sum(dB * EB)
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd))


def test_error_codes_on_device_args():
    x = torch.zeros((12, 4, 4), device="cuda")
    with pytest.raises(capi.WPError) as e:
        capi.wp_lift_forward(x, 3)
    assert e.value.status == 3
    with pytest.raises(capi.WPError) as e:
        capi.wp_lift_forward(x, 2, out=x)
    assert e.value.status == 11
    buf = torch.zeros(12 * 16 + 1, device="cuda")
    st = capi.lib().wp_lift_forward(capi._ptr(buf[1:]), capi._ptr(x), 4, 4, 12, 2, capi._stream())
    assert st == 6
    with pytest.raises(capi.WPError) as e:
        capi.wp_wprod(torch.zeros((8, 0, 3), device="cuda"), torch.zeros((8, 3, 2), device="cuda"), 3)
    assert e.value.status == 2
    assert capi.wp_get_device_error() == 0


@pytest.mark.parametrize("n1,n2,n4,p,L", [(256, 256, 256, 192, 3)])
def test_wprod_full_size_sampled(n1, n2, n4, p, L):
    """Full-size 256x256x192 (L = 3) product in the launch configuration the
    benchmark times; 16 sampled output rows x 16 columns against the oracle
    (the transform acts per tube, so C[:, rows][:, :, cols] = A[:, rows, :] *w B[:, :, cols])."""
    A = synth.hsi_cube(n1, n2, p, seed=0, dtype=np.float32)
    B = synth.hsi_cube(n2, n4, p, seed=1, dtype=np.float32)
    C = host(capi.wp_wprod(dev(A), dev(B), L))
    rng = np.random.default_rng(12)
    rows = np.sort(rng.choice(n1, 16, replace=False))
    cols = np.sort(rng.choice(n4, 16, replace=False))
    ref = O.wprod(A[:, rows, :], B[:, :, cols], L)
    assert O.rel_fro(C[:, rows][:, :, cols], ref) <= TOL_PROD
