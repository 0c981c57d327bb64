"""Pins of the general-operator lifting oracle (Sec. II-A Eq. 2-3, Example
2.1, Remark 3.1): the lazy-Haar operators give the Haar oracle bit for bit
(which Example 2.2 pins), perfect reconstruction (Lemma 2.1) for
interpolating and CDF-5/3-style operators, the level-by-level loops against
the dense block-matrix product, Example 2.1's structure (U = 0 keeps the
even samples; the interpolating predict annihilates linear signals away from
the ends), adjoints against brute-force linear probing, the w-product and its
gradient against definitions and finite differences, and planted mistakes."""

import numpy as np
import pytest

import oracle as O
from oracle import glifting as GL
from tests import _golden

RNG = np.random.default_rng(11)


def rand(shape, seed):
    return np.random.default_rng(seed).uniform(-1, 1, size=shape)


def haar_levels(L):
    return [GL.HAAR] * L


def test_haar_operators_equal_the_haar_oracle_bit_for_bit():
    ex = _golden.load("example_2_2.txt")
    A = ex["A"]
    p = A.shape[0]
    L = int(np.log2(p))
    assert np.array_equal(GL.glift(A, L, haar_levels(L)), O.lift(A, L))
    X = rand((24, 3, 5), 1)
    for L in (1, 2, 3):
        assert np.array_equal(GL.glift(X, L, haar_levels(L)), O.lift(X, L))
        assert np.array_equal(GL.iglift(O.lift(X, L), L, haar_levels(L)), O.ilift(O.lift(X, L), L))


@pytest.mark.parametrize("ops", [GL.INTERP, GL.CDF53, ((-2, (-0.0625, 0.5625, 0.5625, -0.0625)), (0, (0.25, 0.25)))])
@pytest.mark.parametrize("p,L", [(16, 1), (16, 2), (32, 3), (48, 2), (64, 3)])
def test_perfect_reconstruction(ops, p, L):
    X = rand((p, 4, 3), p + L)
    Y = GL.glift(X, L, [ops] * L)
    assert np.max(np.abs(GL.iglift(Y, L, [ops] * L) - X)) <= 1e-13 * np.max(np.abs(X))


def test_mixed_levels_reconstruct():
    levels = [GL.CDF53, GL.INTERP, GL.HAAR]
    X = rand((64, 2, 2), 5)
    assert np.max(np.abs(GL.iglift(GL.glift(X, 3, levels), 3, levels) - X)) <= 1e-13


@pytest.mark.parametrize("ops", [GL.HAAR, GL.INTERP, GL.CDF53])
def test_dense_matrix_equals_loops(ops):
    p, L = 32, 3
    levels = [ops] * L
    W = GL.dense(p, L, levels)
    X = rand((p, 3, 2), 3)
    assert np.allclose(np.einsum("ij,j...->i...", W, X), GL.glift(X, L, levels), atol=1e-14)
    Winv = np.linalg.inv(W)
    assert np.allclose(np.einsum("ij,j...->i...", Winv, GL.glift(X, L, levels)), X, atol=1e-13)


def test_example_2_1_structure():
    """U = 0: the smooth part of level 1 is the even samples themselves; the
    linear interpolating predict makes d vanish on a linear ramp except at
    the first sample, whose left neighbour comes from the boundary rule."""
    p = 16
    x = np.arange(p, dtype=np.float64)[:, None, None] * 0.75 + 2.0
    Y = GL.glift(x, 1, [GL.INTERP])
    s1, d1 = Y[: p // 2, 0, 0], Y[p // 2:, 0, 0]
    assert np.array_equal(s1, x[1::2, 0, 0])
    assert np.all(d1[1:] == 0.0) and d1[0] != 0.0
    # two levels: the level-2 input is again a ramp (every other sample)
    Y2 = GL.glift(x, 2, [GL.INTERP, GL.INTERP])
    d2 = Y2[p // 4: p // 2, 0, 0]
    assert np.all(d2[1:] == 0.0)
    # constant signals: zero details for every operator whose predict taps sum to 1
    c = np.full((32, 1, 1), 3.5)
    for ops in (GL.INTERP, GL.CDF53, GL.HAAR):
        Yc = GL.glift(c, 3, [ops] * 3)
        assert np.all(Yc[4:] == 0.0)


def test_boundary_rule_half_sample_symmetric():
    y = np.arange(5, dtype=np.float64)
    assert [GL._reflect(i, 5) for i in (-2, -1, 0, 4, 5, 6)] == [1, 0, 0, 4, 4, 3]
    M = GL.op_matrix((-1, (0.5, 0.5)), 5)
    assert np.allclose(M @ y, [0.0, 0.5, 1.5, 2.5, 3.5])


def _probe_matrix(fn, p):
    """The p x p matrix of a linear map along mode 3, by unit vectors."""
    cols = [fn(np.eye(p)[:, k].reshape(p, 1, 1))[:, 0, 0] for k in range(p)]
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("ops", [GL.INTERP, GL.CDF53])
def test_adjoints_against_probing(ops):
    p, L = 16, 2
    levels = [ops] * L
    W = _probe_matrix(lambda x: GL.glift(x, L, levels), p)
    Wi = _probe_matrix(lambda x: GL.iglift(x, L, levels), p)
    G = rand((p, 2, 3), 9)
    assert np.allclose(GL.glift_adjoint(G, L, levels), np.einsum("ij,j...->i...", W.T, G), atol=1e-13)
    assert np.allclose(GL.iglift_adjoint(G, L, levels), np.einsum("ij,j...->i...", Wi.T, G), atol=1e-12)
    # the transform is not orthogonal: W^T differs from W^{-1}
    assert np.max(np.abs(W.T - Wi)) > 0.1


def test_gwprod_definition_and_haar_case():
    A, B = rand((16, 4, 5), 1), rand((16, 5, 3), 2)
    assert np.allclose(GL.gwprod(A, B, 2, haar_levels(2)), O.wprod(A, B, 2), atol=1e-14)
    levels = [GL.CDF53, GL.INTERP]
    W = _probe_matrix(lambda x: GL.glift(x, 2, levels), 16)
    Ah = np.einsum("ij,j...->i...", W, A)
    Bh = np.einsum("ij,j...->i...", W, B)
    C = np.einsum("ij,j...->i...", np.linalg.inv(W), np.einsum("kij,kjl->kil", Ah, Bh))
    assert np.allclose(GL.gwprod(A, B, 2, levels), C, atol=1e-12)


def test_gwprod_grad_finite_differences():
    levels = [GL.CDF53, GL.CDF53]
    A, B, G = rand((8, 3, 4), 3), rand((8, 4, 2), 4), rand((8, 3, 2), 5)
    dA, dB = GL.gwprod_grad(A, B, G, 2, levels)
    f = lambda A_, B_: float(np.sum(G * GL.gwprod(A_, B_, 2, levels)))
    h = 1e-6
    for (X, dX, which) in ((A, dA, 0), (B, dB, 1)):
        for idx in [(0, 0, 0), (3, 1, 2), (7, 2, 1)]:
            idx = tuple(min(i, s - 1) for i, s in zip(idx, X.shape))
            Xp, Xm = X.copy(), X.copy()
            Xp[idx] += h
            Xm[idx] -= h
            fd = (f(Xp, B) - f(Xm, B)) / (2 * h) if which == 0 else (f(A, Xp) - f(A, Xm)) / (2 * h)
            assert abs(fd - dX[idx]) <= 1e-7 * max(1.0, abs(fd))


def test_planted_mistakes_fail(monkeypatch):
    levels = [GL.CDF53, GL.CDF53]
    A, B, G = rand((8, 3, 4), 3), rand((8, 4, 2), 4), rand((8, 3, 2), 5)
    ref_dA, _ = GL.gwprod_grad(A, B, G, 2, levels)
    # the inverse in place of the adjoint (orthogonality assumed) is wrong here
    monkeypatch.setattr(GL, "glift_adjoint", lambda X, L, lv: GL.iglift(X, L, lv))
    bad_dA, _ = GL.gwprod_grad(A, B, G, 2, levels)
    assert np.max(np.abs(bad_dA - ref_dA)) > 1e-3
    monkeypatch.undo()
    # periodic instead of symmetric extension changes the transform near the ends
    x = rand((16, 1, 1), 6)
    good = GL.glift(x, 1, [GL.CDF53])
    monkeypatch.setattr(GL, "_reflect", lambda i, n: i % n)
    assert np.max(np.abs(GL.glift(x, 1, [GL.CDF53]) - good)) > 1e-6


def test_stencil_wider_than_level_rejected():
    with pytest.raises(ValueError):
        GL.glift(np.zeros((8, 1, 1)), 3, [GL.CDF53] * 3)   # level 3 has half length 1
