"""Pins for the oracle's lifting transform (CPU only).

Each pin ties the oracle to something other than itself: the paper's worked
Example 2.2, the dense level-matrix construction of Eq. (2), Lemma 2.1
(perfect reconstruction), Lemma 2.2 (linearity), closed forms (weighted
Parseval identity, constant tubes), and the adjoint definition.  The
`test_planted_*` cases show that plausible mistakes fail these pins.
"""

import numpy as np
import pytest

import oracle as O
from oracle import lifting as LF
from tests import _golden

EX = _golden.load("example_2_2.txt")

SHAPES = [(16, 3, 5, 2), (24, 2, 7, 3), (8, 4, 4, 3), (12, 3, 3, 2), (96, 2, 3, 5), (6, 2, 2, 1), (5, 2, 3, 0)]


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_example_2_2_forward_levels():
    """Example 2.2: level-1 and level-2 coefficients of A and B, exactly."""
    for T in ("A", "B"):
        y1 = O.lift(EX[T], 1)
        np.testing.assert_array_equal(y1[:2], EX[T + "_s1"])
        np.testing.assert_array_equal(y1[2:], EX[T + "_d1"])
        y2 = O.lift(EX[T], 2)
        np.testing.assert_array_equal(y2[0:1], EX[T + "_s2"])
        np.testing.assert_array_equal(y2[1:2], EX[T + "_d2"])
        np.testing.assert_array_equal(y2[2:4], EX[T + "_d1"])


def test_example_2_2_inverse_levels():
    """Example 2.2: inverse of (C_s2, C_d2) is C_s1; inverse of all is C."""
    cs1 = O.ilift(np.concatenate([EX["C_s2"], EX["C_d2"]]), 1)
    np.testing.assert_array_equal(cs1, EX["C_s1"])
    C = O.ilift(np.concatenate([EX["C_s2"], EX["C_d2"], EX["C_d1"]]), 2)
    np.testing.assert_array_equal(C, EX["C"])


@pytest.mark.parametrize("p,n1,n2,L", SHAPES)
def test_perfect_reconstruction(p, n1, n2, L):
    """Lemma 2.1: W^{-1}(W(f)) = f, to 1e-13 relative in float64."""
    x = _rand((p, n1, n2), p * 31 + L)
    assert O.rel_fro(O.ilift(O.lift(x, L), L), x) <= 1e-13
    assert O.rel_fro(O.lift(O.ilift(x, L), L), x) <= 1e-13


@pytest.mark.parametrize("p,n1,n2,L", SHAPES)
def test_linearity(p, n1, n2, L):
    """Lemma 2.2."""
    f, g = _rand((p, n1, n2), 1), _rand((p, n1, n2), 2)
    a, b = 0.7, -1.9
    lhs = O.lift(a * f + b * g, L)
    rhs = a * O.lift(f, L) + b * O.lift(g, L)
    assert O.rel_fro(lhs, rhs) <= 1e-14


@pytest.mark.parametrize("p,n1,n2,L", SHAPES)
def test_dense_matrix_matches_loop(p, n1, n2, L):
    """The loop form equals the p x p matrix assembled from Eq. (2)."""
    W = O.dense_lifting_matrix(p, L)
    x = _rand((p, n1, n2), 3)
    assert O.rel_fro(O.lift(x, L), np.einsum("kt,tij->kij", W, x)) <= 1e-14
    Winv = np.linalg.inv(W)
    assert O.rel_fro(O.ilift(x, L), np.einsum("kt,tij->kij", Winv, x)) <= 1e-13


def test_dense_matrix_example():
    """p = 4, L = 2: rows are s2, d2, d1(1), d1(2) per Algorithm 1."""
    W = O.dense_lifting_matrix(4, 2)
    expect = np.array([[0.25, 0.25, 0.25, 0.25],
                       [0.5, 0.5, -0.5, -0.5],
                       [1.0, -1.0, 0.0, 0.0],
                       [0.0, 0.0, 1.0, -1.0]])
    np.testing.assert_array_equal(W, expect)


@pytest.mark.parametrize("p,n1,n2,L", SHAPES)
def test_weighted_parseval(p, n1, n2, L):
    """Closed form: ||x||^2 = 2^L ||s_L||^2 + sum_j 2^(j-2) ||d_j||^2 (each
    level maps (a, b) to s = (a+b)/2, d = a-b, and a^2 + b^2 = 2 s^2 + d^2/2)."""
    x = _rand((p, n1, n2), 4)
    y = O.lift(x, L)
    s, details = O.split_mallat(y, L)
    total = (2.0 ** L) * np.sum(s ** 2)
    for idx, d in enumerate(details):
        j = L - idx
        total += 2.0 ** (j - 2) * np.sum(d ** 2)
    assert abs(total - np.sum(x ** 2)) <= 1e-12 * np.sum(x ** 2)


@pytest.mark.parametrize("p,L", [(16, 4), (24, 3), (96, 5), (8, 1)])
def test_constant_tubes_have_zero_details(p, L):
    """A tube constant along mode 3 has d_j = 0 exactly and s_L = the constant."""
    c = _rand((1, 3, 4), 5)
    x = np.broadcast_to(c, (p, 3, 4))
    y = O.lift(x, L)
    m = p >> L
    assert np.all(y[m:] == 0.0)
    np.testing.assert_array_equal(y[:m], np.broadcast_to(c, (m, 3, 4)))


def test_level_zero_is_identity():
    x = _rand((7, 2, 3), 6)
    np.testing.assert_array_equal(O.lift(x, 0), x)
    np.testing.assert_array_equal(O.ilift(x, 0), x)
    np.testing.assert_array_equal(O.lift_adjoint(x, 0), x)
    np.testing.assert_array_equal(O.ilift_adjoint(x, 0), x)


@pytest.mark.parametrize("p,n1,n2,L", SHAPES)
def test_adjoints_match_dense_transposes(p, n1, n2, L):
    """W^T and W^{-T} equal the transposes of the dense matrices."""
    W = O.dense_lifting_matrix(p, L)
    g = _rand((p, n1, n2), 7)
    assert O.rel_fro(O.lift_adjoint(g, L), np.einsum("tk,tij->kij", W, g)) <= 1e-14
    Winv = np.linalg.inv(W)
    assert O.rel_fro(O.ilift_adjoint(g, L), np.einsum("tk,tij->kij", Winv, g)) <= 1e-13


@pytest.mark.parametrize("p,n1,n2,L", SHAPES)
def test_adjoint_inner_products(p, n1, n2, L):
    """<W x, g> = <x, W^T g> and <W^{-1} x, g> = <x, W^{-T} g>."""
    x, g = _rand((p, n1, n2), 8), _rand((p, n1, n2), 9)
    assert abs(np.sum(O.lift(x, L) * g) - np.sum(x * O.lift_adjoint(g, L))) <= 1e-12 * np.sqrt(x.size)
    assert abs(np.sum(O.ilift(x, L) * g) - np.sum(x * O.ilift_adjoint(g, L))) <= 1e-12 * np.sqrt(x.size)


def test_transform_is_not_orthogonal():
    """Remark 2.1: W^T != W^{-1}; at p = 8, L = 3 they differ by 0.875."""
    W = O.dense_lifting_matrix(8, 3)
    diff = np.max(np.abs(W.T - np.linalg.inv(W)))
    assert abs(diff - 0.875) < 1e-12


def test_rejects_bad_levels():
    with pytest.raises(ValueError):
        O.lift(np.zeros((12, 1, 1)), 3)
    with pytest.raises(ValueError):
        O.lift(np.zeros((8, 1, 1)), -1)


# ---- planted mistakes: each must fail at least one pin above ----------------

def _pins_hold(lift_fn, ilift_fn):
    ok = True
    for T in ("A", "B"):
        y2 = lift_fn(EX[T], 2)
        ok &= np.array_equal(y2[0:1], EX[T + "_s2"]) and np.array_equal(y2[2:4], EX[T + "_d1"])
    ok &= np.array_equal(ilift_fn(np.concatenate([EX["C_s2"], EX["C_d2"], EX["C_d1"]]), 2), EX["C"])
    W = O.dense_lifting_matrix(24, 3)
    x = _rand((24, 2, 3), 10)
    ok &= O.rel_fro(lift_fn(x, 3), np.einsum("kt,tij->kij", W, x)) <= 1e-14
    ok &= O.rel_fro(ilift_fn(lift_fn(x, 3), 3), x) <= 1e-13
    return bool(ok)


def test_pins_accept_oracle():
    assert _pins_hold(O.lift, O.ilift)


def _lift_swapped_parity(x, L):
    s = np.asarray(x, dtype=np.float64)
    det = []
    for _ in range(L):
        d = s[1::2] - s[0::2]          # mistake: 0-based even minus odd
        s = s[0::2] + d / 2
        det.append(d)
    return np.concatenate([s] + det[::-1], axis=0)


def _lift_wrong_order(x, L):
    y = O.lift(x, L)
    s, det = O.split_mallat(y, L)
    return np.concatenate([s] + det[::-1], axis=0)  # mistake: d_1 before d_L


def _lift_dropped_update(x, L):
    s = np.asarray(x, dtype=np.float64)
    det = []
    for _ in range(L):
        d = s[0::2] - s[1::2]
        s = s[1::2]                    # mistake: update step omitted
        det.append(d)
    return np.concatenate([s] + det[::-1], axis=0)


def _ilift_wrong_sign(y, L):
    s, details = O.split_mallat(np.asarray(y, dtype=np.float64), L)
    for d in details:
        even = s + d / 2               # mistake: sign of the update undo
        odd = d + even
        out = np.empty((2 * s.shape[0],) + s.shape[1:])
        out[0::2], out[1::2] = odd, even
        s = out
    return s


@pytest.mark.parametrize("bad_lift,bad_ilift", [
    (_lift_swapped_parity, O.ilift),
    (_lift_wrong_order, O.ilift),
    (_lift_dropped_update, O.ilift),
    (O.lift, _ilift_wrong_sign),
])
def test_planted_mistakes_fail_pins(bad_lift, bad_ilift):
    assert not _pins_hold(bad_lift, bad_ilift)


def test_mallat_split_sizes():
    y = np.arange(24.0).reshape(24, 1, 1)
    s, det = LF.split_mallat(y, 3)
    assert s.shape[0] == 3 and [d.shape[0] for d in det] == [3, 6, 12]
