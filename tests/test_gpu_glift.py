"""GPU parity of the general-operator lifting (Eq. 2-3 with arbitrary
predict / update operators, Example 2.1, Remark 3.1) against the FP64 oracle
(oracle.glifting): the four transforms, the w-product and its backward.
Tolerances: transforms 1e-6 relative Frobenius (a few FP32 roundings per
level), products 1e-5 (FP32 and BF16x3 face-products), gradients 1e-5."""

import numpy as np
import pytest
import torch

from oracle import glifting as GL
import oracle as O
from paper_2601_08228_gb300 import capi

pytestmark = pytest.mark.gpu


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


CUBIC = ((-2, (-0.0625, 0.5625, 0.5625, -0.0625)), (0, (0.25, 0.25)))
OPS = {"haar": GL.HAAR, "interp": GL.INTERP, "cdf53": GL.CDF53, "cubic": CUBIC}


@pytest.mark.parametrize("name", list(OPS))
@pytest.mark.parametrize("p,n1,n2,L", [(16, 5, 7, 2), (48, 33, 3, 3), (192, 16, 20, 3), (64, 1, 1, 4), (800, 4, 9, 5)])
def test_glift_four_transforms(name, p, n1, n2, L):
    ops = OPS[name]
    levels = [ops] * L
    try:
        GL._check_ops(levels, L, p)
    except ValueError:
        pytest.skip("stencil wider than a level")
    X = rand((p, n1, n2), p + L)
    Xd = dev(X)
    refs = {"forward": GL.glift(X, L, levels), "inverse": GL.iglift(X, L, levels),
            "adjoint": GL.glift_adjoint(X, L, levels), "inverse_adjoint": GL.iglift_adjoint(X, L, levels)}
    for op, ref in refs.items():
        Y = host(capi.wp_glift(Xd, L, levels, op=op))
        assert O.rel_fro(Y, ref) <= 1e-6, (op, O.rel_fro(Y, ref))
    assert capi.wp_get_device_error() == 0


def test_glift_haar_equals_lift_bit_for_bit():
    X = dev(rand((64, 17, 9), 3))
    for L in (1, 3, 5):
        a = capi.wp_glift(X, L, [GL.HAAR] * L)
        b = capi.wp_lift_forward(X, L)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


def test_glift_mixed_levels_round_trip():
    levels = [GL.CDF53, CUBIC, GL.INTERP, GL.HAAR]
    X = rand((128, 40, 13), 4)
    Y = capi.wp_glift(dev(X), 4, levels)
    Z = host(capi.wp_glift(Y, 4, levels, op="inverse"))
    assert O.rel_fro(Z, X) <= 1e-6
    assert O.rel_fro(host(Y), GL.glift(X, 4, levels)) <= 1e-6


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16x3", 1e-5)])
def test_gwprod_and_backward(prec, tol):
    levels = [GL.CDF53, GL.INTERP, CUBIC]
    p, n1, n2, n4, L = 64, 40, 36, 28, 3
    A, B, G = rand((p, n1, n2), 5), rand((p, n2, n4), 6), rand((p, n1, n4), 7)
    C = host(capi.wp_gwprod(dev(A), dev(B), L, levels, prec=prec))
    assert O.rel_fro(C, GL.gwprod(A, B, L, levels)) <= tol
    dA, dB = capi.wp_gwprod_backward(dev(A), dev(B), dev(G), L, levels, prec=prec)
    rA, rB = GL.gwprod_grad(A, B, G, L, levels)
    assert O.rel_fro(host(dA), rA) <= tol
    assert O.rel_fro(host(dB), rB) <= tol
    assert capi.wp_get_device_error() == 0


def test_glift_host_validation():
    X = torch.zeros((8, 4, 4), device="cuda")
    with pytest.raises(capi.WPError) as e:
        capi.wp_glift(X, 3, [GL.CDF53] * 3)          # level 3 half length 1: stencil too wide
    assert e.value.status == capi.WP_ERR_SHAPE
    with pytest.raises(capi.WPError) as e:
        capi.wp_glift(torch.zeros((1024, 2, 2), device="cuda"), 1, [GL.HAAR])
    assert e.value.status == capi.WP_ERR_UNSUPPORTED
