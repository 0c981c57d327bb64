"""Pins for the oracle's w-product, transpose, identity, inverse and trace
(CPU only).  Sources: Example 2.2, Def. 2.1-2.4, Thm 2.1-2.4, Def. 2.7 and
Lemma 2.5, plus brute force through the dense transform matrix.
"""

import numpy as np
import pytest

import oracle as O
from tests import _golden

EX = _golden.load("example_2_2.txt")


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_example_2_2_product():
    """Example 2.2: wavelet-domain face-products and the result C, exactly."""
    Ah, Bh = O.lift(EX["A"], 2), O.lift(EX["B"], 2)
    Ch = O.facewise(Ah, Bh)
    np.testing.assert_array_equal(Ch[0:1], EX["C_s2"])
    np.testing.assert_array_equal(Ch[1:2], EX["C_d2"])
    np.testing.assert_array_equal(Ch[2:4], EX["C_d1"])
    np.testing.assert_array_equal(O.wprod(EX["A"], EX["B"], 2), EX["C"])


@pytest.mark.parametrize("p,n1,n2,n4", [(5, 3, 4, 2), (8, 6, 1, 7)])
def test_level_zero_is_batched_matmul(p, n1, n2, n4):
    A, B = _rand((p, n1, n2), 1), _rand((p, n2, n4), 2)
    np.testing.assert_allclose(O.wprod(A, B, 0), np.matmul(A, B), rtol=0, atol=1e-13)


def _brute_force_wprod(A, B, L):
    """Explicit sums through the dense transform matrix: no slicing code."""
    p, n1, n2 = A.shape
    n4 = B.shape[2]
    W = O.dense_lifting_matrix(p, L)
    Winv = np.linalg.inv(W)
    C = np.zeros((p, n1, n4))
    for t in range(p):
        for i in range(n1):
            for l in range(n4):
                acc = 0.0
                for k in range(p):
                    inner = 0.0
                    for j in range(n2):
                        a = sum(W[k, u] * A[u, i, j] for u in range(p))
                        b = sum(W[k, u] * B[u, j, l] for u in range(p))
                        inner += a * b
                    acc += Winv[t, k] * inner
                C[t, i, l] = acc
    return C


@pytest.mark.parametrize("p,L,n1,n2,n4", [(4, 2, 2, 3, 2), (6, 1, 2, 2, 3), (8, 3, 1, 2, 2), (12, 2, 2, 1, 2)])
def test_brute_force_tiny(p, L, n1, n2, n4):
    A, B = _rand((p, n1, n2), 3), _rand((p, n2, n4), 4)
    assert O.rel_fro(O.wprod(A, B, L), _brute_force_wprod(A, B, L)) <= 1e-12


@pytest.mark.parametrize("p,L", [(8, 3), (24, 3), (12, 1)])
def test_associativity(p, L):
    """Thm 2.4."""
    A, B, C = _rand((p, 3, 4), 5), _rand((p, 4, 2), 6), _rand((p, 2, 5), 7)
    lhs = O.wprod(O.wprod(A, B, L), C, L)
    rhs = O.wprod(A, O.wprod(B, C, L), L)
    assert O.rel_fro(lhs, rhs) <= 1e-13


@pytest.mark.parametrize("p,L", [(8, 3), (24, 3)])
def test_transpose_invariance_and_reversal(p, L):
    """Thm 2.1 (W(A^T) = W(A)^T) and Thm 2.2 ((A *w B)^T = B^T *w A^T)."""
    A, B = _rand((p, 3, 4), 8), _rand((p, 4, 5), 9)
    np.testing.assert_array_equal(O.lift(O.transpose(A), L), O.transpose(O.lift(A, L)))
    np.testing.assert_array_equal(O.ilift(O.transpose(A), L), O.transpose(O.ilift(A, L)))
    lhs = O.transpose(O.wprod(A, B, L))
    rhs = O.wprod(O.transpose(B), O.transpose(A), L)
    assert O.rel_fro(lhs, rhs) <= 1e-14
    np.testing.assert_allclose(O.wprod(B, A, L, transA=True, transB=True), lhs, atol=1e-13)


@pytest.mark.parametrize("p,L", [(8, 3), (24, 3), (2, 1), (12, 2)])
def test_identity(p, L):
    """Def. 2.3: A *w I = I *w A = A."""
    A = _rand((p, 4, 4), 10)
    I = O.identity(4, p, L)
    assert O.rel_fro(O.wprod(A, I, L), A) <= 1e-14
    assert O.rel_fro(O.wprod(I, A, L), A) <= 1e-14


def test_identity_closed_form_level_one():
    """L = 1: the spatial identity alternates 1.5 I_n and 0.5 I_n (inverse of
    s = d = I_n: even = s - d/2, odd = d + even)."""
    I = O.identity(3, 4, 1)
    np.testing.assert_array_equal(I[0], 1.5 * np.eye(3))
    np.testing.assert_array_equal(I[1], 0.5 * np.eye(3))
    np.testing.assert_array_equal(I[2], 1.5 * np.eye(3))
    np.testing.assert_array_equal(I[3], 0.5 * np.eye(3))


def _winv(A, L):
    """Def. 2.4: facewise matrix inverse in the wavelet domain."""
    return O.ilift(np.linalg.inv(O.lift(A, L)), L)


@pytest.mark.parametrize("p,L", [(8, 3), (12, 2)])
def test_inverse_tensor(p, L):
    """Def. 2.4, Lemma 2.3 and Thm 2.3."""
    n = 4
    A = _rand((p, n, n), 11) + 3 * np.eye(n)
    B = _rand((p, n, n), 12) + 3 * np.eye(n)
    I = O.identity(n, p, L)
    Ai = _winv(A, L)
    assert O.rel_fro(O.wprod(A, Ai, L), I) <= 1e-12
    assert O.rel_fro(O.wprod(Ai, A, L), I) <= 1e-12
    assert O.rel_fro(_winv(Ai, L), A) <= 1e-12
    assert O.rel_fro(_winv(O.wprod(A, B, L), L), O.wprod(_winv(B, L), Ai, L)) <= 1e-11


@pytest.mark.parametrize("p,L", [(8, 3), (24, 3), (12, 2)])
def test_trace_closed_form(p, L):
    """Def. 2.7 with the tube-sum identity: every inverse level maps (s, d) to
    a pair summing to 2s, so Tr(A *w B) = 2^L sum_{k in s_L} Tr(A_k B_k)."""
    A, B = _rand((p, 5, 5), 13), _rand((p, 5, 5), 14)
    Ah, Bh = O.lift(A, L), O.lift(B, L)
    m = p >> L
    closed = 2 ** L * sum(np.trace(Ah[k] @ Bh[k]) for k in range(m))
    assert abs(O.trace(O.wprod(A, B, L)) - closed) <= 1e-11 * max(1.0, abs(closed))
    assert abs(O.trace(O.identity(5, p, L)) - 2 ** L * m * 5) <= 1e-12


@pytest.mark.parametrize("p,L", [(8, 3), (12, 2)])
def test_trace_properties(p, L):
    """Lemma 2.5, properties 1-4."""
    A, B = _rand((p, 4, 4), 15), _rand((p, 4, 4), 16)
    tr = O.trace
    assert abs(tr(A) - tr(O.transpose(A))) <= 1e-12
    assert abs(tr(2.0 * A - 3.0 * B) - (2.0 * tr(A) - 3.0 * tr(B))) <= 1e-12
    assert abs(tr(O.wprod(A, B, L)) - tr(O.wprod(B, A, L))) <= 1e-11
    assert abs(tr(O.wprod(O.transpose(A), B, L)) - tr(O.wprod(A, O.transpose(B), L))) <= 1e-11


def test_planted_wrong_facewise_pairing_fails():
    """Multiplying A_hat_k by B_hat_(k+1) (an index slip) breaks Example 2.2."""
    Ah, Bh = O.lift(EX["A"], 2), O.lift(EX["B"], 2)
    bad = O.ilift(O.facewise(Ah, np.roll(Bh, 1, axis=0)), 2)
    assert not np.array_equal(bad, EX["C"])


def test_planted_transposed_operand_fails():
    A, B = _rand((8, 3, 3), 17), _rand((8, 3, 3), 18)
    good = _brute_force_wprod(A, B, 3)
    assert O.rel_fro(O.wprod(A, B, 3, transB=True), good) > 1e-3
