"""The lifting transform as an explicit p x p matrix (test oracle).

An independent formulation of W_[L] used to cross-check the loop form in
`lifting.py`.  It is assembled from Eq. (2): at level j the transform acts on
the first l = p / 2^(j-1) coefficients (the current smooth part s_{j-1}) as

    W_j = [[I, U_j], [0, I]] . [[I, 0], [-P_j, I]]   applied to [even; odd]

with P_j = I and U_j = I/2 (the lazy choice after Example 2.1), and leaves the
detail coefficients already produced untouched.  "even" and "odd" follow the
1-based convention that Algorithm 1 and Example 2.2 fix: even = positions
2, 4, ..., odd = positions 1, 3, ....  The level output [s_j; d_j] lands in
front of the older details, which yields the Mallat order of Eq. (1).

W_[L] = M_L ... M_1 with M_j = blockdiag(W_j S_j, I) and S_j the split
permutation.  No code is shared with `lifting.py`.
"""

import numpy as np


def _level_matrix(p, ell):
    half = ell // 2
    # S_j: f -> [even; odd] with 1-based parity (0-based rows 1,3,.. then 0,2,..)
    S = np.zeros((ell, ell))
    for k in range(half):
        S[k, 2 * k + 1] = 1.0          # even_(k+1) = f_(2k+2) (1-based)
        S[half + k, 2 * k] = 1.0       # odd_(k+1)  = f_(2k+1) (1-based)
    I = np.eye(half)
    Z = np.zeros((half, half))
    P = I                              # predict operator P_j = I
    U = 0.5 * I                        # update operator  U_j = I/2
    upd = np.block([[I, U], [Z, I]])
    pred = np.block([[I, Z], [-P, I]])
    Wj = upd @ pred @ S                # [s_j; d_j] from s_{j-1}
    M = np.eye(p)
    M[:ell, :ell] = Wj
    return M


def dense_lifting_matrix(p, L):
    """Return the p x p matrix of W_[L] in Mallat output order."""
    if L < 0 or p % (1 << L) != 0:
        raise ValueError("p must be a multiple of 2^L")
    W = np.eye(p)
    for j in range(1, L + 1):
        ell = p >> (j - 1)
        W = _level_matrix(p, ell) @ W
    return W
