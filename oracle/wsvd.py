"""Truncated w-svd and sp-w-svd (test oracle).

Algorithm 2: transform A along mode 3, take the SVD of every wavelet-domain
frontal slice, keep the leading r singular triplets,
C_k = U_k[:, :r] Sigma_k[:r, :r] V_k[:, :r]^T, and transform back.  Thm 2.5
gives the spatial factors U = W^{-1}(U_k), Sigma = W^{-1}(Sigma_k),
V = W^{-1}(V_k) with A^(r) = U *w Sigma *w V^T.

sp-w-svd (Sec. IV-B, "Computational analysis") uses only the A_{s_L} and
A_{d_L} slices.  Reading taken: those 2m slices are truncated at rank r, every
d_j slice with j < L is set to zero before the inverse transform.

Per-slice SVD is numpy.linalg.svd (LAPACK gesdd), a library step.
"""

import numpy as np

from .lifting import lift, ilift, check_levels


def _check_rank(n1, n2, r):
    if r < 1 or r > min(n1, n2):
        raise ValueError(f"rank r={r} outside [1, min(n1, n2)={min(n1, n2)}]")


def _truncated(Ah, r, slices):
    p, n1, n2 = Ah.shape
    Ch = np.zeros_like(Ah)
    Uw = np.zeros((p, n1, r))
    Sw = np.zeros((p, r))
    Vw = np.zeros((p, n2, r))
    for k in slices:
        U, S, Vt = np.linalg.svd(Ah[k], full_matrices=False)
        Ch[k] = (U[:, :r] * S[:r]) @ Vt[:r]
        Uw[k] = U[:, :r]
        Sw[k] = S[:r]
        Vw[k] = Vt[:r].T
    return Ch, Uw, Sw, Vw


def wsvd(A, L, r, return_factors=False, factors_in_wavelet_domain=True):
    """Rank-r w-svd of A (p, n1, n2), Algorithm 2.

    Returns C = A^(r), and with return_factors also (U, S, V) of shapes
    (p, n1, r), (p, r), (p, n2, r): in the wavelet domain (Mallat order) by
    default, or mapped to the spatial domain with W^{-1} as in Thm 2.5.
    """
    A = np.asarray(A, dtype=np.float64)
    p, n1, n2 = A.shape
    check_levels(p, L)
    _check_rank(n1, n2, r)
    Ah = lift(A, L)
    Ch, Uw, Sw, Vw = _truncated(Ah, r, range(p))
    C = ilift(Ch, L)
    if not return_factors:
        return C
    if not factors_in_wavelet_domain:
        Uw, Sw, Vw = ilift(Uw, L), ilift(Sw, L), ilift(Vw, L)
    return C, Uw, Sw, Vw


def spwsvd(A, L, r, return_factors=False, factors_in_wavelet_domain=True):
    """Rank-r sp-w-svd: only the s_L and d_L slices (Mallat rows [0, 2m)) are
    kept and truncated; all finer details d_1..d_{L-1} are zeroed."""
    A = np.asarray(A, dtype=np.float64)
    p, n1, n2 = A.shape
    check_levels(p, L)
    _check_rank(n1, n2, r)
    m = p >> L
    Ah = lift(A, L)
    kept = range(min(2 * m, p))
    Ch, Uw, Sw, Vw = _truncated(Ah, r, kept)
    C = ilift(Ch, L)
    if not return_factors:
        return C
    if not factors_in_wavelet_domain:
        Uw, Sw, Vw = ilift(Uw, L), ilift(Sw, L), ilift(Vw, L)
    return C, Uw, Sw, Vw
