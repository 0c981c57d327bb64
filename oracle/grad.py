"""Gradient of the w-product (test oracle).

The paper has no differentiation.  For the scalar f = <G, A *w B> (Frobenius
inner product), with C = W^{-1}(C_hat), C_hat_k = A_hat_k B_hat_k and
A_hat = W(A) (Def. 2.1), the chain rule gives the adjoint route

    G_hat   = W^{-T} G                  (cotangent of C_hat)
    dA_hat_k = G_hat_k B_hat_k^T,   dB_hat_k = A_hat_k^T G_hat_k
    dA      = W^T dA_hat,           dB = W^T dB_hat

W is not orthogonal (Remark 2.1), so W^T and W^{-T} are the adjoint
operators of `lifting.py`, not the inverse transform.
"""

import numpy as np

from .lifting import lift, lift_adjoint, ilift_adjoint


def wprod_grad(A, B, G, L):
    """Return (dA, dB) of f(A, B) = <G, A *w B> by the adjoint route."""
    Ah = lift(A, L)
    Bh = lift(B, L)
    Gh = ilift_adjoint(G, L)
    p = Ah.shape[0]
    dAh = np.empty_like(Ah)
    dBh = np.empty_like(Bh)
    for k in range(p):
        dAh[k] = Gh[k] @ Bh[k].T
        dBh[k] = Ah[k].T @ Gh[k]
    return lift_adjoint(dAh, L), lift_adjoint(dBh, L)
