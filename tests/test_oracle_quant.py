"""Pins for the oracle's FP8 (E4M3) emulation (CPU only).

The rounding is checked against the format's value table built here from
its bit fields, and against PyTorch's float8_e4m3fn conversion; the per-slice
scaling against its invariants (the largest code is 448, power-of-two scale
invariance, all-zero slices); the product against the exact FP64 product
within the E4M3 error level.
"""

import numpy as np
import pytest
import torch

import oracle as O
from oracle import quant as Q


def _table():
    """All finite non-negative E4M3 values from (exponent, mantissa) fields."""
    vals = []
    for e in range(16):
        for f in range(8):
            if e == 15 and f == 7:
                continue                      # NaN pattern
            vals.append(2.0 ** -6 * (f / 8) if e == 0 else 2.0 ** (e - 7) * (1 + f / 8))
    return np.array(sorted(set(vals)))


def test_table_values_are_fixed_points():
    t = _table()
    assert len(t) == 127 and t[-1] == 448.0 and t[1] == 2.0 ** -9
    np.testing.assert_array_equal(Q.e4m3_round(t), t)
    np.testing.assert_array_equal(Q.e4m3_round(-t), -t)


def test_midpoints_round_to_even_mantissa():
    t = _table()
    mid = 0.5 * (t[:-1] + t[1:])
    got = Q.e4m3_round(mid)
    # the neighbour whose code (index in the table) is even has the even mantissa
    idx = np.arange(len(t) - 1)
    want = np.where(idx % 2 == 0, t[:-1], t[1:])
    np.testing.assert_array_equal(got, want)
    # just off the midpoint: the nearer neighbour
    np.testing.assert_array_equal(Q.e4m3_round(mid * (1 - 1e-9)), t[:-1])
    np.testing.assert_array_equal(Q.e4m3_round(mid * (1 + 1e-9)), t[1:])


def test_saturation():
    np.testing.assert_array_equal(Q.e4m3_round([449.0, 480.0, 1e30, -500.0]), [448.0, 448.0, 448.0, -448.0])


def test_matches_torch_float8_e4m3fn():
    rng = np.random.default_rng(5)
    x = np.sign(rng.standard_normal(200000)) * 10.0 ** rng.uniform(-4, np.log10(440.0), 200000)
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(Q.e4m3_round(x), ref)


def test_slice_scales_and_codes():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((5, 7, 9)).astype(np.float32)
    X[3] = 0.0
    q, s = Q.quantize(X)
    for k in (0, 1, 2, 4):
        assert np.abs(q[k]).max() == 448.0
    assert s[3] == 1.0 and not q[3].any()
    # a power-of-two rescaling of a slice changes its scale, not its codes
    X2 = X.copy()
    X2[1] *= np.float32(2.0 ** 5)
    q2, s2 = Q.quantize(X2)
    np.testing.assert_array_equal(q2, q)
    assert s2[1] == s[1] * 2.0 ** 5


def test_float32_lift_is_single_rounding():
    """lift(x, L, float32) on integer data is exact (no rounding happens), and
    on random data within float32 rounding of the FP64 lift."""
    rng = np.random.default_rng(7)
    xi = rng.integers(-1000, 1000, size=(16, 3, 4)).astype(np.float64)
    np.testing.assert_array_equal(O.lift(xi, 4, np.float32), O.lift(xi, 4))
    x = rng.standard_normal((32, 5, 6))
    np.testing.assert_allclose(O.lift(x.astype(np.float32), 3, np.float32), O.lift(x, 3), rtol=0, atol=2e-6)


@pytest.mark.parametrize("L", [0, 2, 3])
def test_wprod_fp8_within_e4m3_error(L):
    rng = np.random.default_rng(8)
    A = rng.uniform(-1, 1, (8, 24, 40)).astype(np.float32)
    B = rng.uniform(-1, 1, (8, 40, 16)).astype(np.float32)
    C = O.wprod_fp8(A, B, L)
    err = O.rel_fro(C, O.wprod(A, B, L))
    # 3 mantissa bits: unit roundoff 2^-4 per operand, averaged over 40 terms
    assert 1e-3 < err < 0.08, err
    if L == 0:
        np.testing.assert_array_equal(C, O.facewise_fp8(A, B))


def test_per_slice_scales_keep_small_slices():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((4, 16, 16)).astype(np.float32) * np.float32(1e-3)
    A[0] *= np.float32(1e6)
    B = rng.standard_normal((4, 16, 16)).astype(np.float32)
    C, ref = O.facewise_fp8(A, B), O.facewise(A, B)
    for k in range(4):
        assert O.rel_fro(C[k], ref[k]) < 0.08
