"""Pins of the oracle's error metrics (Sec. IV-A): PSNR against values worked
out by hand, and the relative Frobenius error against its definition on
arrays whose norms are known exactly.  The planted variants (MPP squared, a
natural logarithm, a sum in place of the mean) each fail a hand value."""

import math

import numpy as np
import pytest

import oracle as O
from oracle import metrics as M


def test_psnr_hand_values():
    # every element off by 0.1: mean squared error 0.01, so 10 log10(1 / 0.01) = 20 dB
    x = np.zeros((4, 5, 6))
    y = np.full((4, 5, 6), 0.1)
    assert O.psnr(x, y) == pytest.approx(20.0, abs=1e-12)
    # peak value 2 (MPP, not MPP^2): 10 log10(2 / 0.01) = 10 (2 + log10 2)
    assert O.psnr(x, y, mpp=2.0) == pytest.approx(20.0 + 10.0 * math.log10(2.0), abs=1e-12)
    # one element off by 1 in 100: MSE 0.01, 20 dB again (the mean is over all elements)
    a = np.zeros(100)
    b = np.zeros(100)
    b[37] = 1.0
    assert O.psnr(a, b) == pytest.approx(20.0, abs=1e-12)
    # symmetric in its arguments, independent of the array shape
    assert O.psnr(b, a) == O.psnr(a, b)
    assert O.psnr(a.reshape(10, 10), b.reshape(10, 10)) == O.psnr(a, b)


def test_psnr_identical_is_inf():
    x = np.random.default_rng(0).uniform(size=(3, 7, 5))
    assert O.psnr(x, x.copy()) == float("inf")


def _psnr_mpp_squared(x1, x2, mpp=1.0):
    err = float(np.sum((np.asarray(x1, float) - np.asarray(x2, float)) ** 2))
    return 10.0 * np.log10(np.size(x1) * mpp * mpp / err)


def _psnr_natural_log(x1, x2, mpp=1.0):
    err = float(np.sum((np.asarray(x1, float) - np.asarray(x2, float)) ** 2))
    return 10.0 * np.log(np.size(x1) * mpp / err)


def _psnr_sum_not_mean(x1, x2, mpp=1.0):
    err = float(np.sum((np.asarray(x1, float) - np.asarray(x2, float)) ** 2))
    return 10.0 * np.log10(mpp / err)


@pytest.mark.parametrize("bad", [_psnr_mpp_squared, _psnr_natural_log, _psnr_sum_not_mean])
def test_planted_psnr_mistakes_fail(monkeypatch, bad):
    monkeypatch.setattr(M, "psnr", bad)
    x = np.zeros((4, 5, 6))
    y = np.full((4, 5, 6), 0.1)
    hand = (20.0, 20.0 + 10.0 * math.log10(2.0))
    got = (M.psnr(x, y), M.psnr(x, y, mpp=2.0))
    assert any(abs(g - h) > 1e-6 for g, h in zip(got, hand))


def test_rel_fro_hand_values():
    ref = np.array([[3.0, 0.0], [0.0, 4.0]])      # ||ref||_F = 5
    x = ref + np.array([[0.0, 0.6], [0.8, 0.0]])  # ||x - ref||_F = 1
    assert O.rel_fro(x, ref) == pytest.approx(0.2, abs=1e-15)
    assert O.rel_fro(ref, ref) == 0.0
    # a zero reference falls back to the absolute error
    assert O.rel_fro(np.array([3.0, 4.0]), np.zeros(2)) == pytest.approx(5.0, abs=1e-15)
