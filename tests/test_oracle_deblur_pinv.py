"""Pins for the oracle's two-sided pseudo-inverse deblurring (Sec. IV-C) and
the linear blur operators it is run with (CPU only)."""

import numpy as np
import pytest

import oracle as O
from paper_2601_08228_gb300 import synth


def test_linear_blur_operator_as_printed():
    """c(k) = (b - k) / (3 b) for 0 <= k < b: c(0) = 1/3, c(b - 1) = 1/(3b),
    zero beyond; symmetric Toeplitz; interior rows sum to 10/3 at b = 10."""
    A = synth.linear_blur_operator(40, 3, b=10)
    T = A[0]
    assert np.array_equal(A[0], A[2]) and np.array_equal(T, T.T)
    assert T[5, 5] == pytest.approx(1 / 3, abs=0) and T[0, 9] == pytest.approx(1 / 30, abs=1e-16)
    assert T[0, 10] == 0.0 and T[12, 30] == 0.0
    assert T[20].sum() == pytest.approx(10 / 3, rel=1e-15)


def test_pinv_of_transpose_is_transpose_of_pinv():
    A = np.random.default_rng(1).standard_normal((8, 5, 7))
    np.testing.assert_allclose(O.wpinv(O.transpose(A), 2), O.transpose(O.wpinv(A, 2)), rtol=0, atol=1e-12)


def test_exact_recovery_with_invertible_operators():
    """B = A_V *w X *w A_H^T with invertible operators: the reconstruction
    returns X (Def. 2.4: A *w A^dagger is the identity tensor then)."""
    rng = np.random.default_rng(2)
    p, n1, n2, L = 8, 12, 9, 3
    AV = np.eye(n1) + 0.2 * rng.standard_normal((p, n1, n1)) / np.sqrt(n1)
    AH = np.eye(n2) + 0.2 * rng.standard_normal((p, n2, n2)) / np.sqrt(n2)
    X = rng.standard_normal((p, n1, n2))
    B = O.wprod(O.wprod(AV, X, L), O.transpose(AH), L)
    np.testing.assert_allclose(O.deblur_pinv(AV, AH, B, L), X, rtol=0, atol=1e-10)


def test_recovery_through_the_paper_blur():
    """The paper's blur operators at a small size (full rank).  They are
    constant across bands, so their detail slices are zero and the blurred
    data keep only the s_L part of X: the reconstruction is X with its
    detail slices removed, within the conditioning of the blur."""
    p, n1, n2, L = 8, 24, 16, 2
    AV = synth.linear_blur_operator(n1, p, b=4)
    AH = synth.linear_blur_operator(n2, p, b=4)
    X = synth.hsi_cube(n1, n2, p, rank=3, seed=5)
    B = O.wprod(O.wprod(AV, X, L), O.transpose(AH), L)
    Xh = O.lift(X, L)
    Xh[p >> L:] = 0.0
    expect = O.ilift(Xh, L)
    kap = np.linalg.cond(AV[0]) * np.linalg.cond(AH[0])
    got = O.deblur_pinv(AV, AH, B, L)
    assert O.rel_fro(got, expect) <= 100 * kap * np.finfo(float).eps
    assert O.rel_fro(got, X) > 1e-4          # the details are really gone


def test_band_constant_operator_has_zero_detail_pinv():
    """A band-constant operator has exactly zero detail slices, and so has its
    w-pseudo-inverse: only the s_L slices carry the reconstruction."""
    p, n, L = 16, 10, 2
    AV = synth.linear_blur_operator(n, p, b=3)
    Ph = O.lift(O.wpinv(AV, L), L)
    assert not Ph[p >> L:].any()
    np.testing.assert_allclose(Ph[0], np.linalg.pinv(AV[0]), rtol=0, atol=1e-12)
