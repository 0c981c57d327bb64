"""Second-generation lifting with general per-level predict / update
operators (test oracle).  TEST INFRASTRUCTURE ONLY (see the package doc).

Sec. II-A, Eq. (2)-(3): every level j splits its input f_(j-1) into two
halves and applies
    W_j = [[I, U_j], [0, I]] [[I, 0], [-P_j, I]]   on (even; odd),
i.e.  d_j = odd - P_j(even),   s_j = even + U_j(d_j),
and the inverse  even = s_j - U_j(d_j),  odd = d_j + P_j(even).  Example 2.1
is the interpolating predict with U = 0; Remark 3.1 allows any operators per
level.  The lazy-Haar transform of the rest of the package is P_j = I,
U_j = I / 2.

Readings (the paper fixes neither):
  * even / odd follow Algorithm 1's 1-based positions, as in lifting.py:
    odd[k] = x[2k], even[k] = x[2k + 1] (0-based), so P = I, U = 1/2 gives
    d = x[2k] - x[2k+1], s = x[2k+1] + d / 2 exactly as the Haar oracle.
  * an operator is a stencil of taps c_0..c_{T-1} at offset o:
        (Op y)[k] = sum_t c_t y[k + o + t],
    with half-sample symmetric extension at both ends of the length-N
    sequence y: y[-1 - i] = y[i], y[N + i] = y[N - 1 - i].
  * coefficients are stored in the Mallat order (s_L, d_L, ..., d_1) of Eq. (1).
A level whose half-length is smaller than the stencil's reach is rejected.

The transforms are written two ways: level by level with explicit loops over
k (the steps in the paper's order), and as one dense p x p matrix built from
per-level block matrices (`dense`), which also gives the adjoints W^T and
W^{-T} by plain matrix transposition.
"""

import numpy as np

from .lifting import check_levels

# Example operator sets (each entry: (offset, taps)); see the module readings.
HAAR = ((0, (1.0,)), (0, (0.5,)))                         # P = I, U = I / 2
INTERP = ((-1, (0.5, 0.5)), (0, ()))                      # linear interpolating predict, U = 0 (Example 2.1)
CDF53 = ((-1, (0.5, 0.5)), (0, (0.25, 0.25)))            # interpolating predict + averaging update


def _reflect(i, n):
    """Half-sample symmetric extension index into [0, n)."""
    while i < 0 or i >= n:
        if i < 0:
            i = -1 - i
        if i >= n:
            i = 2 * n - 1 - i
    return i


def apply_op(op, y):
    """(Op y)[k] = sum_t c_t y[refl(k + o + t)] along axis 0 of y."""
    off, taps = op
    n = y.shape[0]
    out = np.zeros_like(y)
    for k in range(n):
        for t, c in enumerate(taps):
            out[k] = out[k] + c * y[_reflect(k + off + t, n)]
    return out


def op_matrix(op, n):
    """The n x n matrix of a stencil operator with the boundary rule."""
    M = np.zeros((n, n))
    off, taps = op
    for k in range(n):
        for t, c in enumerate(taps):
            M[k, _reflect(k + off + t, n)] += c
    return M


def _check_ops(levels, L, p):
    if len(levels) != L:
        raise ValueError(f"{len(levels)} level operators for L = {L}")
    for j, (P, U) in enumerate(levels, start=1):
        half = p >> j
        for op in (P, U):
            off, taps = op
            reach = max(abs(off), abs(off + len(taps) - 1)) if taps else 0
            if reach >= half:
                raise ValueError(f"level {j}: stencil reach {reach} >= half length {half}")


def glift(A, L, levels):
    """Forward transform of every mode-3 tube of A (p, n1, n2); Mallat order.
    levels[j-1] = (P_j, U_j), each (offset, taps)."""
    A = np.asarray(A, dtype=np.float64)
    p = A.shape[0]
    check_levels(p, L)
    _check_ops(levels, L, p)
    s = A.copy()
    details = []
    for j in range(1, L + 1):
        P, U = levels[j - 1]
        odd, even = s[0::2], s[1::2]
        d = odd - apply_op(P, even)
        s = even + apply_op(U, d)
        details.append(d)
    return np.concatenate([s] + details[::-1], axis=0)


def iglift(Y, L, levels):
    """Inverse transform (Eq. 3 with general operators): Mallat order in."""
    Y = np.asarray(Y, dtype=np.float64)
    p = Y.shape[0]
    check_levels(p, L)
    _check_ops(levels, L, p)
    s = Y[: p >> L]
    for j in range(L, 0, -1):
        P, U = levels[j - 1]
        half = p >> j
        d = Y[half: 2 * half]
        even = s - apply_op(U, d)
        odd = d + apply_op(P, even)
        x = np.empty((2 * half,) + Y.shape[1:])
        x[0::2], x[1::2] = odd, even
        s = x
    return s


def dense(p, L, levels):
    """W as an explicit p x p matrix: the product of per-level block matrices
    (split permutation, then [[I, 0], [-P, I]], then [[I, U], [0, I]]),
    embedded with the identity on the detail coefficients already produced."""
    check_levels(p, L)
    _check_ops(levels, L, p)
    W = np.eye(p)
    for j in range(1, L + 1):
        P, U = levels[j - 1]
        n = p >> (j - 1)
        h = n // 2
        S = np.zeros((n, n))                 # (x) -> (even; odd)
        for k in range(h):
            S[k, 2 * k + 1] = 1.0
            S[h + k, 2 * k] = 1.0
        Pm, Um = op_matrix(P, h), op_matrix(U, h)
        I = np.eye(h)
        Z = np.zeros((h, h))
        Wj = np.block([[I, Um], [Z, I]]) @ np.block([[I, Z], [-Pm, I]]) @ S
        # level j acts on the first n rows (the current smooth part)
        E = np.eye(p)
        E[:n, :n] = Wj
        W = E @ W
    # rows are now (s_L, d_L, ..., d_1) in Mallat order
    return W


def glift_adjoint(G, L, levels):
    """W^T applied along mode 3 (the backward of a product with W(.))."""
    G = np.asarray(G, dtype=np.float64)
    Wt = dense(G.shape[0], L, levels).T
    return np.einsum("ij,j...->i...", Wt, G)


def iglift_adjoint(G, L, levels):
    """W^{-T} applied along mode 3."""
    G = np.asarray(G, dtype=np.float64)
    Wit = np.linalg.inv(dense(G.shape[0], L, levels)).T
    return np.einsum("ij,j...->i...", Wit, G)


def gwprod(A, B, L, levels):
    """w-product with general operators: W^{-1}(W(A) Delta W(B)) (Def. 2.1)."""
    Ah, Bh = glift(A, L, levels), glift(B, L, levels)
    return iglift(np.einsum("kij,kjl->kil", Ah, Bh), L, levels)


def gwprod_grad(A, B, G, L, levels):
    """(dA, dB) of <G, A *w B> by the adjoint route:
    G_hat = W^{-T} G, dA = W^T(G_hat Delta B_hat^T), dB = W^T(A_hat^T Delta G_hat)."""
    Ah, Bh = glift(A, L, levels), glift(B, L, levels)
    Gh = iglift_adjoint(G, L, levels)
    dA = glift_adjoint(np.einsum("kil,kjl->kij", Gh, Bh), L, levels)
    dB = glift_adjoint(np.einsum("kij,kil->kjl", Ah, Gh), L, levels)
    return dA, dB
