"""Face-product and w-product (test oracle).

Def. 2.1: A *w B = W_[L]^{-1}( W_[L](A) Delta W_[L](B) ), with Delta the
face-product: one independent matrix product per wavelet-domain frontal slice
(Algorithm 1, middle loop, which visits every d_j slice and the s_L slices).

Also the transpose (Def. 2.2), identity tensor (Def. 2.3) and trace
(Def. 2.7).  Tensors are slice-major (p, rows, cols).
"""

import numpy as np

from .lifting import lift, ilift, check_levels


def facewise(Ah, Bh):
    """Face-product Delta: C[k] = A[k] @ B[k] for every frontal slice k."""
    Ah = np.asarray(Ah, dtype=np.float64)
    Bh = np.asarray(Bh, dtype=np.float64)
    if Ah.ndim != 3 or Bh.ndim != 3 or Ah.shape[0] != Bh.shape[0] or Ah.shape[2] != Bh.shape[1]:
        raise ValueError(f"face-product shape mismatch {Ah.shape} x {Bh.shape}")
    C = np.empty((Ah.shape[0], Ah.shape[1], Bh.shape[2]))
    for k in range(Ah.shape[0]):
        C[k] = Ah[k] @ Bh[k]
    return C


def transpose(A):
    """Tensor transpose, Def. 2.2: A^T[i, j, :] = A[j, i, :]."""
    return np.ascontiguousarray(np.swapaxes(np.asarray(A, dtype=np.float64), 1, 2))


def wprod(A, B, L, transA=False, transB=False):
    """w-product op(A) *w op(B) following Algorithm 1 (Def. 2.1).

    transA / transB apply the tensor transpose of Def. 2.2 to the operand
    first.
    """
    A = transpose(A) if transA else np.asarray(A, dtype=np.float64)
    B = transpose(B) if transB else np.asarray(B, dtype=np.float64)
    check_levels(A.shape[0], L)
    if A.shape[0] != B.shape[0]:
        raise ValueError("A and B must have the same tube length p")
    return ilift(facewise(lift(A, L), lift(B, L)), L)


def identity(n, p, L):
    """Identity tensor of Def. 2.3: I_n in every wavelet-domain slice, mapped
    back to the spatial domain with the inverse transform."""
    check_levels(p, L)
    return ilift(np.broadcast_to(np.eye(n), (p, n, n)), L)


def trace(A):
    """Tensor trace of Def. 2.7: sum over k and i of A[i, i, k]."""
    A = np.asarray(A, dtype=np.float64)
    return float(sum(np.trace(A[k]) for k in range(A.shape[0])))
