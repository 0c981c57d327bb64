"""Pins for the oracle's w-svd, sp-w-svd and Moore-Penrose inverse (CPU only).

Sources: Algorithm 2 and Thm 2.5 (w-svd), Sec. IV-B (sp-w-svd), Def. 2.6,
Thm 2.6, Remark 2.2 and Lemma 2.4 (pseudo-inverse).  Independent checks use
a different LAPACK routine (symmetric eigensolver), the weighted Parseval
identity and the Penrose equations.
"""

import numpy as np
import pytest

import oracle as O
from tests import _golden

REM = _golden.load("remark_2_2.txt")


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def _weighted_tail(Ah, L, r, slices):
    """Weighted Parseval sum of discarded squared singular values."""
    p = Ah.shape[0]
    total = 0.0
    for k in slices:
        sig = np.sqrt(np.clip(np.linalg.eigvalsh(Ah[k].T @ Ah[k] if Ah.shape[1] >= Ah.shape[2] else Ah[k] @ Ah[k].T), 0, None))[::-1]
        total += _weight(k, p, L) * np.sum(sig[r:] ** 2)
    return total


def _weight(k, p, L):
    m = p >> L
    if k < m:
        return 2.0 ** L
    for j in range(L, 0, -1):
        if k < (p >> (j - 1)):
            return 2.0 ** (j - 2)
    raise AssertionError


@pytest.mark.parametrize("p,L,n1,n2,r", [(24, 3, 10, 7, 3), (16, 2, 6, 9, 2), (8, 3, 5, 5, 4)])
def test_wsvd_truncation_error_identity(p, L, n1, n2, r):
    """||A - A^(r)||_F^2 equals the weighted tail 2^L sum_{s_L} + sum_j 2^(j-2)
    sum_{d_j} of discarded sigma^2 (singular values from eigvalsh)."""
    A = _rand((p, n1, n2), 1)
    err2 = np.sum((A - O.wsvd(A, L, r)) ** 2)
    tail = _weighted_tail(O.lift(A, L), L, r, range(p))
    assert abs(err2 - tail) <= 1e-10 * np.sum(A ** 2)


@pytest.mark.parametrize("p,L,n1,n2", [(24, 3, 6, 4), (8, 2, 3, 5)])
def test_wsvd_full_rank_is_exact(p, L, n1, n2):
    A = _rand((p, n1, n2), 2)
    assert O.rel_fro(O.wsvd(A, L, min(n1, n2)), A) <= 1e-13


@pytest.mark.parametrize("p,L,n1,n2,r", [(24, 3, 7, 6, 3), (8, 1, 4, 6, 2)])
def test_wsvd_factors_thm_2_5(p, L, n1, n2, r):
    """Thm 2.5: spatial factors give A^(r) = U *w Sigma *w V^T, and U, V have
    orthonormal columns facewise: U^T *w U = I_r (reading of Def. 2.5)."""
    A = _rand((p, n1, n2), 3)
    C, U, S, V = O.wsvd(A, L, r, return_factors=True, factors_in_wavelet_domain=False)
    Sig = np.zeros((p, r, r))
    for k in range(p):
        Sig[k] = np.diag(S[k])
    rec = O.wprod(O.wprod(U, Sig, L), V, L, transB=True)
    assert O.rel_fro(rec, C) <= 1e-13
    I = O.identity(r, p, L)
    assert O.rel_fro(O.wprod(U, U, L, transA=True), I) <= 1e-13
    assert O.rel_fro(O.wprod(V, V, L, transA=True), I) <= 1e-13


def test_wsvd_matches_eigh_reconstruction_tiny():
    """Rank-r truncation rebuilt from eigh of A_k^T A_k (a different LAPACK
    path): C_k = A_k V_r V_r^T."""
    p, L, n1, n2, r = 8, 3, 6, 4, 2
    A = _rand((p, n1, n2), 4)
    Ah = O.lift(A, L)
    Ch = np.empty((p, n1, n2))
    for k in range(p):
        w, V = np.linalg.eigh(Ah[k].T @ Ah[k])
        Vr = V[:, ::-1][:, :r]
        Ch[k] = Ah[k] @ Vr @ Vr.T
    assert O.rel_fro(O.wsvd(A, L, r), O.ilift(Ch, L)) <= 1e-11


@pytest.mark.parametrize("p,L,n1,n2,r", [(24, 3, 8, 6, 2), (96, 5, 5, 4, 3)])
def test_spwsvd_structure(p, L, n1, n2, r):
    """sp-w-svd: details d_j (j < L) are zero in the result's transform; the
    s_L and d_L slices equal w-svd's; its error is never below w-svd's."""
    A = _rand((p, n1, n2), 5)
    m = p >> L
    Csp, Cw = O.spwsvd(A, L, r), O.wsvd(A, L, r)
    ysp, yw = O.lift(Csp, L), O.lift(Cw, L)
    assert np.max(np.abs(ysp[2 * m:])) <= 1e-12
    assert O.rel_fro(ysp[:2 * m], yw[:2 * m]) <= 1e-12
    assert np.sum((A - Csp) ** 2) >= np.sum((A - Cw) ** 2) - 1e-12
    err2 = np.sum((A - Csp) ** 2)
    Ah = O.lift(A, L)
    tail = _weighted_tail(Ah, L, r, range(2 * m)) + sum(
        _weight(k, p, L) * np.sum(Ah[k] ** 2) for k in range(2 * m, p))
    assert abs(err2 - tail) <= 1e-10 * np.sum(A ** 2)


def test_wsvd_rejects_bad_rank():
    with pytest.raises(ValueError):
        O.wsvd(np.zeros((8, 3, 4)), 3, 4)
    with pytest.raises(ValueError):
        O.spwsvd(np.zeros((8, 3, 4)), 3, 0)


# ---- Moore-Penrose inverse --------------------------------------------------

def test_remark_2_2_counterexample():
    """Remark 2.2's printed values (two decimals)."""
    A, B = REM["A"], REM["B"]
    atol = 0.005
    yA, yB = O.lift(A, 1), O.lift(B, 1)
    np.testing.assert_allclose(yA[0:1], REM["A_s"], atol=atol)
    np.testing.assert_allclose(yA[1:2], REM["A_d"], atol=atol)
    np.testing.assert_allclose(yB[0:1], REM["B_s"], atol=atol)
    np.testing.assert_allclose(yB[1:2], REM["B_d"], atol=atol)
    AB = O.wprod(A, B, 1)
    yAB = O.lift(AB, 1)
    np.testing.assert_allclose(yAB[0:1], REM["AB_s"], atol=atol)
    np.testing.assert_allclose(yAB[1:2], REM["AB_d"], atol=atol)
    C = O.wpinv(AB, 1)
    yC = O.lift(C, 1)
    np.testing.assert_allclose(yC[0:1], REM["C_s"], atol=atol)
    np.testing.assert_allclose(yC[1:2], REM["C_d"], atol=atol)
    np.testing.assert_allclose(C, REM["C"], atol=atol)
    Ad, Bd = O.wpinv(A, 1), O.wpinv(B, 1)
    yAd, yBd = O.lift(Ad, 1), O.lift(Bd, 1)
    np.testing.assert_allclose(yAd[0:1], REM["Adag_s"], atol=atol)
    np.testing.assert_allclose(yAd[1:2], REM["Adag_d"], atol=atol)
    np.testing.assert_allclose(yBd[0:1], REM["Bdag_s"], atol=atol)
    np.testing.assert_allclose(yBd[1:2], REM["Bdag_d"], atol=atol)
    D = O.wprod(Bd, Ad, 1)
    yD = O.lift(D, 1)
    np.testing.assert_allclose(yD[0:1], REM["D_s"], atol=atol)
    np.testing.assert_allclose(yD[1:2], REM["D_d"], atol=atol)
    np.testing.assert_allclose(D, REM["D"], atol=atol)
    assert np.max(np.abs(C - D)) > 0.1


def _penrose_residuals(A, X, L):
    AX = O.wprod(A, X, L)
    XA = O.wprod(X, A, L)
    return (O.rel_fro(O.wprod(AX, A, L), A),
            O.rel_fro(O.wprod(XA, X, L), X),
            O.rel_fro(O.transpose(AX), AX),
            O.rel_fro(O.transpose(XA), XA))


@pytest.mark.parametrize("p,L,m,n,rank", [(8, 3, 5, 3, None), (24, 3, 4, 6, None), (12, 2, 6, 6, 2)])
def test_penrose_equations(p, L, m, n, rank):
    """Def. 2.6: the four Penrose equations hold for wpinv(A)."""
    if rank is None:
        A = _rand((p, m, n), 6)
    else:  # facewise rank-deficient in the wavelet domain
        Ah = np.einsum("kir,krj->kij", _rand((p, m, rank), 7), _rand((p, rank, n), 8))
        A = O.ilift(Ah, L)
    X = O.wpinv(A, L)
    assert X.shape == (p, n, m)
    for res in _penrose_residuals(A, X, L):
        assert res <= 1e-11


def test_pinv_of_invertible_is_inverse():
    """Def. 2.4 via Thm 2.6: A *w A^dagger = I for invertible A."""
    p, L, n = 8, 3, 4
    A = _rand((p, n, n), 9) + 3 * np.eye(n)
    assert O.rel_fro(O.wprod(A, O.wpinv(A, L), L), O.identity(n, p, L)) <= 1e-12


@pytest.mark.parametrize("p,L,m,n", [(8, 3, 5, 3), (12, 2, 3, 4)])
def test_mp_properties(p, L, m, n):
    """Lemma 2.4, properties 1-4."""
    A = _rand((p, m, n), 10)
    Ad = O.wpinv(A, L)
    assert O.rel_fro(O.wpinv(Ad, L), A) <= 1e-11
    assert O.rel_fro(O.wpinv(O.transpose(A), L), O.transpose(Ad)) <= 1e-11
    AAt = O.wprod(A, A, L, transB=True)
    assert O.rel_fro(O.wpinv(AAt, L), O.wprod(O.wpinv(O.transpose(A), L), Ad, L)) <= 1e-10
    assert O.rel_fro(Ad, O.wprod(A, O.wpinv(AAt, L), L, transA=True)) <= 1e-10


def test_pinv_zero_slice():
    X = O.wpinv(np.zeros((4, 3, 2)), 2)
    assert X.shape == (4, 2, 3) and np.all(X == 0)


def test_planted_pinv_without_transform_fails():
    """Taking the facewise pinv in the spatial domain (no lifting) breaks the
    Penrose equations under *w."""
    p, L = 8, 3
    A = _rand((p, 4, 3), 11)
    X = np.linalg.pinv(A)
    assert max(_penrose_residuals(A, X, L)) > 1e-3
