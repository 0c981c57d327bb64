"""Lazy-Haar lifting along mode 3 (test oracle; see the package docstring).

Sec. II-A defines the second-generation wavelet transform W_[L] = W_L ... W_1,
each level W_j being a predict step (d = odd - P even) followed by an update
step (s = even + U d), Eq. (1)-(2).  The w-product uses the "lazy" choice
P_j = I, U_j = I/2 (text after Example 2.1).  Algorithm 1's forward loop pins
the parity convention with 1-based indices inside each tube:

    d_j[k] = s_{j-1}[2k-1] - s_{j-1}[2k]
    s_j[k] = s_{j-1}[2k]   + d_j[k] / 2

and its inverse loop undoes it coarsest level first (Eq. 3):

    s_{j-1}[2k]   = s_j[k] - d_j[k] / 2
    s_{j-1}[2k-1] = d_j[k] + s_{j-1}[2k]

In 0-based NumPy slicing, 1-based position 2k-1 is index 2k-2 (x[0::2]) and
position 2k is index 2k-1 (x[1::2]).

The coefficients are stored in the Mallat order of Eq. (1):
[s_L (m) | d_L (m) | d_{L-1} (2m) | ... | d_1 (p/2)], p = 2^L m, so d_j
occupies rows [p/2^j, p/2^(j-1)).

The transform is not orthogonal (Remark 2.1), so the adjoints W^T and W^{-T}
(needed by the backward pass) are separate operators.  They are written here
level by level as the transposes of the 2x2 level maps:
    forward level:  [s; d] = [[1/2, 1/2], [1, -1]] [a; b],   a = odd, b = even
    W^T level:      g_a = g_s/2 + g_d,  g_b = g_s/2 - g_d
    inverse level:  [a; b] = [[1, 1/2], [1, -1/2]] [s; d]
    W^{-T} level:   g_s = g_a + g_b,    g_d = (g_a - g_b)/2
"""

import numpy as np


def check_levels(p, L):
    """Validate p = 2^L m with L >= 0 and m >= 1 (Sec. II-A, first paragraph)."""
    if L < 0:
        raise ValueError("L must be >= 0")
    if p < 1 or p % (1 << L) != 0:
        raise ValueError(f"p={p} is not a positive multiple of 2^L={1 << L}")


def split_mallat(y, L):
    """Return (s_L, [d_L, d_{L-1}, ..., d_1]) as views into the Mallat array y."""
    p = y.shape[0]
    check_levels(p, L)
    m = p >> L
    details = [y[(p >> j):(p >> (j - 1))] for j in range(L, 0, -1)]
    return y[:m], details


def lift(x, L, dtype=np.float64):
    """Forward transform W_[L] along axis 0 (Algorithm 1 forward loop, Eq. 1).

    x: array (p, ...) with p = 2^L m.  Returns the Mallat-ordered coefficients,
    same shape, in `dtype` (float64; float32 only for the FP8 emulation, which
    needs the single-precision coefficients that a float32 implementation of
    the same two steps produces: d rounded once, s rounded once).
    """
    s = np.asarray(x, dtype=dtype)
    check_levels(s.shape[0], L)
    details = []
    for _j in range(1, L + 1):
        odd = s[0::2]            # 1-based positions 1, 3, ..., l-1
        even = s[1::2]           # 1-based positions 2, 4, ..., l
        d = odd - even           # predict with P_j = I
        s = even + d / 2         # update with U_j = I/2
        details.append(d)
    return np.concatenate([s] + details[::-1], axis=0)


def ilift(y, L):
    """Inverse transform W_[L]^{-1} (Algorithm 1 inverse loop, Eq. 3)."""
    y = np.asarray(y, dtype=np.float64)
    s, details = split_mallat(y, L)
    for d in details:            # j = L down to 1
        even = s - d / 2
        odd = d + even
        out = np.empty((2 * s.shape[0],) + s.shape[1:], dtype=np.float64)
        out[0::2] = odd
        out[1::2] = even
        s = out
    return s.copy()


def lift_adjoint(g, L):
    """Apply W_[L]^T: Mallat-ordered cotangent -> spatial cotangent.

    W = W_L ... W_1, so W^T = W_1^T ... W_L^T: the coarsest level's transpose
    acts first.
    """
    g = np.asarray(g, dtype=np.float64)
    gs, details = split_mallat(g, L)
    for gd in details:           # j = L down to 1
        ga = gs / 2 + gd
        gb = gs / 2 - gd
        out = np.empty((2 * gs.shape[0],) + gs.shape[1:], dtype=np.float64)
        out[0::2] = ga
        out[1::2] = gb
        gs = out
    return gs.copy()


def ilift_adjoint(h, L):
    """Apply W_[L]^{-T}: spatial cotangent -> Mallat-ordered cotangent.

    W^{-1} = W_1^{-1} ... W_L^{-1}, so W^{-T} = W_L^{-T} ... W_1^{-T}: the
    finest level's transpose acts first.
    """
    s = np.asarray(h, dtype=np.float64)
    check_levels(s.shape[0], L)
    details = []
    for _j in range(1, L + 1):
        ga = s[0::2]
        gb = s[1::2]
        details.append((ga - gb) / 2)
        s = ga + gb
    return np.concatenate([s] + details[::-1], axis=0)
