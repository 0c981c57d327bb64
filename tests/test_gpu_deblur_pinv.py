"""GPU parity of the two-sided pseudo-inverse deblurring X = A_V^+ *w B *w
(A_H^T)^+ (Sec. IV-C) through the C ABI, against the FP64 oracle."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_08228_gb300 import capi, synth

pytestmark = pytest.mark.gpu
EPS32 = 1.1920929e-7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2601_08228_gb300 import build
    build.build()
    capi.lib()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


@pytest.mark.parametrize("p,n1,n2,L,b", [(8, 24, 16, 2, 4), (12, 40, 33, 2, 5), (16, 64, 48, 4, 6)])
@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_deblur_pinv_paper_blur(p, n1, n2, L, b, prec):
    """The paper's linear blur operators; B an arbitrary cube.  Both sides cut
    singular values at max(n) * eps32 relative; two refinement steps."""
    AV = synth.linear_blur_operator(n1, p, b=b, dtype=np.float32)
    AH = synth.linear_blur_operator(n2, p, b=b, dtype=np.float32)
    B = synth.hsi_cube(n1, n2, p, rank=4, seed=7, dtype=np.float32)
    X = capi.wp_deblur_pinv(dev(AV), dev(AH), dev(B), L, refine_iters=2, prec=prec).cpu().numpy()
    ref = O.deblur_pinv(AV, AH, B, L, rtol=max(n1, n2) * EPS32)
    kap = np.linalg.cond(AV[0].astype(np.float64)) + np.linalg.cond(AH[0].astype(np.float64))
    err = O.rel_fro(X, ref)
    print(f"deblur_pinv {p}x{n1}x{n2} L={L} b={b} {prec}: {err:.2e} (kappa sum {kap:.1e})")
    assert err <= max(1e-4, 8 * kap * EPS32), err
    assert capi.wp_get_device_error() == 0


def test_deblur_pinv_recovers_with_invertible_operators():
    """Operators whose every wavelet slice is I + a small perturbation
    (condition numbers near 1.5; non-symmetric, so the transposed second
    product is exercised): B = A_V *w X *w A_H^T is deblurred back to X."""
    rng = np.random.default_rng(3)
    p, n1, n2, L = 8, 48, 40, 3
    AV = O.ilift(np.eye(n1) + 0.2 * rng.standard_normal((p, n1, n1)) / np.sqrt(n1), L)
    AH = O.ilift(np.eye(n2) + 0.2 * rng.standard_normal((p, n2, n2)) / np.sqrt(n2), L)
    X0 = rng.standard_normal((p, n1, n2))
    B = O.wprod(O.wprod(AV, X0, L), O.transpose(AH), L)
    X = capi.wp_deblur_pinv(dev(AV), dev(AH), dev(B), L, refine_iters=1).cpu().numpy()
    assert O.rel_fro(X, X0) <= 1e-5


@pytest.mark.parametrize("n1,n2", [(217, 128), (128, 217)])
def test_deblur_pinv_wide_blur_singular_detail_slices(n1, n2):
    """The benchmark's blur width (b = 10) on a 217-pixel side: the spatial
    operator has condition number ~2e4 and its detail slices are singular, so
    the cut-off decides which singular values are kept.  Every singular value
    down to the cut-off must be resolved; a Jacobi that leaves small columns
    unrotated fails this by orders of magnitude."""
    p, L, b = 8, 2, 10
    AV = synth.linear_blur_operator(n1, p, b=b, dtype=np.float32)
    AH = synth.linear_blur_operator(n2, p, b=b, dtype=np.float32)
    B = synth.hsi_cube(n1, n2, p, rank=4, seed=11, dtype=np.float32)
    X = capi.wp_deblur_pinv(dev(AV), dev(AH), dev(B), L, refine_iters=2).cpu().numpy()
    ref = O.deblur_pinv(AV, AH, B, L, rtol=max(n1, n2) * EPS32)
    kap = np.linalg.cond(AV[0].astype(np.float64)) + np.linalg.cond(AH[0].astype(np.float64))
    err = O.rel_fro(X, ref)
    print(f"deblur_pinv {p}x{n1}x{n2} L={L} b={b}: {err:.2e} (kappa sum {kap:.1e})")
    assert err <= 8 * kap * EPS32, err
    assert capi.wp_get_device_error() == 0


def test_wpinv_wide_blur_operator():
    """wp_wpinv alone on the b = 10 blur of a 217-pixel side (cut-off
    217 eps32 relative), against the oracle on the same FP32 input."""
    p, n, L, b = 8, 217, 2, 10
    A = synth.linear_blur_operator(n, p, b=b, dtype=np.float32)
    X = capi.wp_wpinv(dev(A), L, rtol=n * EPS32, refine_iters=2).cpu().numpy()
    ref = O.wpinv(A, L, rtol=n * EPS32)
    kap = np.linalg.cond(A[0].astype(np.float64))
    err = O.rel_fro(X, ref)
    print(f"wpinv {p}x{n}x{n} L={L} b={b}: {err:.2e} (kappa {kap:.1e})")
    assert err <= 8 * kap * EPS32, err
    assert capi.wp_get_device_error() == 0
