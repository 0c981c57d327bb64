"""Pins for the oracle's gradient and deblurring objective (CPU only).

f(A, B) = <G, A *w B> is bilinear, so its gradient is pinned exactly by
linear probing (unit perturbations) and by central finite differences; the
closed forms dA = G *w B^T and dB = A^T *w G follow from W^T D W = I with D
the weighted-Parseval diagonal and are checked too.  Using the inverse
transform where the adjoint belongs (a plausible mistake, Remark 2.1) fails.
"""

import numpy as np
import pytest

import oracle as O
from oracle import grad as GR
from paper_2601_08228_gb300 import synth


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def _f(A, B, G, L):
    return float(np.sum(G * O.wprod(A, B, L)))


@pytest.mark.parametrize("p,L,n1,n2,n4", [(8, 3, 2, 3, 2), (6, 1, 2, 2, 2), (12, 2, 1, 2, 3)])
def test_grad_linear_probing(p, L, n1, n2, n4):
    """f is linear in A: dA[idx] = f(A + e_idx) - f(A) exactly (brute force)."""
    A, B, G = _rand((p, n1, n2), 1), _rand((p, n2, n4), 2), _rand((p, n1, n4), 3)
    dA, dB = O.wprod_grad(A, B, G, L)
    base = _f(A, B, G, L)
    for idx in np.ndindex(A.shape):
        E = np.zeros_like(A)
        E[idx] = 1.0
        assert abs((_f(A + E, B, G, L) - base) - dA[idx]) <= 1e-12
    for idx in np.ndindex(B.shape):
        E = np.zeros_like(B)
        E[idx] = 1.0
        assert abs((_f(A, B + E, G, L) - base) - dB[idx]) <= 1e-12


def test_grad_central_fd_16x16x8():
    """Central finite differences on a 16x16x8 crop, L = 3."""
    p, L, n = 8, 3, 16
    A, B, G = _rand((p, n, n), 4), _rand((p, n, n), 5), _rand((p, n, n), 6)
    dA, dB = O.wprod_grad(A, B, G, L)
    rng = np.random.default_rng(7)
    for _ in range(4):
        EA, EB = rng.standard_normal(A.shape), rng.standard_normal(B.shape)
        h = 1e-3
        fd = (_f(A + h * EA, B + h * EB, G, L) - _f(A - h * EA, B - h * EB, G, L)) / (2 * h)
        an = np.sum(dA * EA) + np.sum(dB * EB)
        assert abs(fd - an) <= 1e-8 * max(1.0, abs(an))


@pytest.mark.parametrize("p,L", [(8, 3), (24, 3), (12, 2)])
def test_grad_closed_forms(p, L):
    """dA = G *w B^T and dB = A^T *w G."""
    A, B, G = _rand((p, 4, 5), 8), _rand((p, 5, 3), 9), _rand((p, 4, 3), 10)
    dA, dB = O.wprod_grad(A, B, G, L)
    assert O.rel_fro(dA, O.wprod(G, B, L, transB=True)) <= 1e-13
    assert O.rel_fro(dB, O.wprod(A, G, L, transA=True)) <= 1e-13


@pytest.mark.parametrize("swap", ["W^T -> W^-1", "W^-T -> W"])
def test_planted_inverse_instead_of_adjoint_fails(monkeypatch, swap):
    """Substituting W^{-1} for W^T (or W for W^{-T}) on one side breaks the
    gradient.  (Swapping both at once happens to cancel: W^T = W^{-1} D^{-1}
    and W^{-T} = D W with D diagonal per wavelet slice, so the weights cancel
    in the bilinear face-product.)"""
    p, L, n = 8, 3, 2
    A, B, G = _rand((p, n, n), 11), _rand((p, n, n), 12), _rand((p, n, n), 13)
    if swap == "W^T -> W^-1":
        monkeypatch.setattr(GR, "lift_adjoint", O.ilift)
    else:
        monkeypatch.setattr(GR, "ilift_adjoint", O.lift)
    dA_bad, _ = GR.wprod_grad(A, B, G, L)
    monkeypatch.undo()
    dA, _ = O.wprod_grad(A, B, G, L)
    assert O.rel_fro(dA_bad, dA) > 1e-2


def test_both_sided_orthogonal_assumption_cancels(monkeypatch):
    """Documented quirk: W^{-1} for W^T together with W for W^{-T} gives the
    same gradient (see above)."""
    p, L, n = 8, 3, 2
    A, B, G = _rand((p, n, n), 11), _rand((p, n, n), 12), _rand((p, n, n), 13)
    monkeypatch.setattr(GR, "lift_adjoint", O.ilift)
    monkeypatch.setattr(GR, "ilift_adjoint", O.lift)
    dA_swapped, _ = GR.wprod_grad(A, B, G, L)
    monkeypatch.undo()
    dA, _ = O.wprod_grad(A, B, G, L)
    assert O.rel_fro(dA_swapped, dA) <= 1e-13


# ---- deblurring objective -----------------------------------------------------

def test_band_constant_blur_has_zero_details():
    """A band-constant K (the same matrix in every band) has exactly zero
    detail slices, so K *w X only sees X's s_L part."""
    K = synth.blur_operator(12, 16)
    y = O.lift(K, 4)
    assert np.all(y[1:] == 0.0)


def test_blur_adjoint_identity():
    """<K *w X, R> = <X, K^T *w R>."""
    p, L, n = 16, 4, 12
    K = synth.blur_operator(n, p)
    X, R = _rand((p, n, 5), 14), _rand((p, n, 5), 15)
    lhs = np.sum(O.wprod(K, X, L) * R)
    rhs = np.sum(X * O.wprod(K, R, L, transA=True))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_deblur_grad_fd_and_descent():
    p, L, n = 8, 3, 16
    K = synth.blur_operator(n, p)
    X0 = _rand((p, n, n), 16)
    Xt = synth.hsi_cube(n, n, p, rank=3, noise=0.0, seed=2)
    Y = O.wprod(K, Xt, L) + 0.01 * _rand((p, n, n), 3)
    lam = 1e-3
    g = O.deblur_grad(K, X0, Y, L, lam)
    E = _rand(X0.shape, 17)
    h = 1e-4
    fd = (O.deblur_loss(K, X0 + h * E, Y, L, lam) - O.deblur_loss(K, X0 - h * E, Y, L, lam)) / (2 * h)
    assert abs(fd - np.sum(g * E)) <= 1e-6 * abs(fd)
    # plain gradient descent with step 1/Lip decreases the loss monotonically
    # By the weighted Parseval identity ||K *w X|| <= ||T||_2 ||X|| <= ||X|| for a
    # band-constant K built from a normalised kernel, so 2 (1 + lam) bounds the
    # Lipschitz constant of the gradient; 2 (8 + lam) is a safe, smaller step.
    lip = 2 * (8.0 + lam)
    _X, losses = O.deblur_steps(K, X0, Y, L, lam, 1.0 / lip, 10)
    assert all(b <= a for a, b in zip(losses, losses[1:]))
