"""Moore-Penrose inverse under the w-product (test oracle).

Def. 2.6 characterises A^dagger by the four Penrose equations under *w;
Thm 2.6 constructs it as V *w Sigma^dagger *w U^T from the facewise SVD of
Thm 2.5, i.e. the facewise matrix pseudo-inverse of every wavelet-domain
slice, mapped back with W^{-1}.

The paper does not state a cut-off for small singular values.  Reading taken:
per slice keep sigma_i > rtol * sigma_max with rtol = max(rows, cols) * eps
(eps of float64 here); an all-zero slice has an all-zero pseudo-inverse.
"""

import numpy as np

from .lifting import lift, ilift, check_levels


def wpinv(A, L, rtol=None):
    """Return A^dagger of A (p, m, n) as an array (p, n, m)."""
    A = np.asarray(A, dtype=np.float64)
    p, m, n = A.shape
    check_levels(p, L)
    if rtol is None or rtol < 0:
        rtol = max(m, n) * np.finfo(np.float64).eps
    Ah = lift(A, L)
    Xh = np.zeros((p, n, m))
    for k in range(p):
        U, S, Vt = np.linalg.svd(Ah[k], full_matrices=False)
        if S.size == 0 or S[0] == 0.0:
            continue
        keep = S > rtol * S[0]
        Xh[k] = (Vt[keep].T / S[keep]) @ U[:, keep].T
    return ilift(Xh, L)
