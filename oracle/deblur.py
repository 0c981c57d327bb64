"""Deblurring under the w-product (test oracle): the two-sided pseudo-inverse
reconstruction of Sec. IV-C and a gradient-descent variant.

Two-sided model (Sec. IV-C): a cube X is blurred vertically and horizontally
by band-constant operators, B = A_V *w X *w A_H^T, and recovered as the
least-squares solution X = A_V^dagger *w B *w (A_H^T)^dagger
(`deblur_pinv`, written literally: the pseudo-inverse of the transposed
operator, Def. 2.2 and Def. 2.6).

Gradient-descent variant.

The paper's deblurring model (Sec. IV-C) observes a blurred cube through a
w-product with a band-constant blur tensor.  The one-sided form used here,
Y = K *w X + noise, is solved by gradient descent on

    f(X) = ||K *w X - Y||_F^2 + lam ||X||_F^2
    grad f(X) = 2 K^T *w (K *w X - Y) + 2 lam X

K^T *w is the exact adjoint of K *w: by the adjoint route of `grad.py`,
d<R, K *w X>/dX = W^T(K_hat^T Delta W^{-T} R), which equals K^T *w R because
W^T D W = I for the diagonal weight D of the lifting (see the tests).  The
gradient here is computed by the adjoint route itself.
"""

import numpy as np

from .wproduct import wprod, transpose
from .grad import wprod_grad
from .wpinv import wpinv


def deblur_loss(K, X, Y, L, lam):
    R = wprod(K, X, L) - Y
    return float(np.sum(R * R) + lam * np.sum(np.asarray(X) ** 2))


def deblur_grad(K, X, Y, L, lam):
    R = wprod(K, X, L) - Y
    _dK, dX = wprod_grad(K, X, R, L)
    return 2.0 * dX + 2.0 * lam * np.asarray(X, dtype=np.float64)


def deblur_steps(K, X0, Y, L, lam, eta, steps):
    """Run `steps` plain gradient steps X <- X - eta grad f(X); return X and
    the loss before every step and after the last."""
    X = np.array(X0, dtype=np.float64)
    losses = []
    for _ in range(steps):
        losses.append(deblur_loss(K, X, Y, L, lam))
        X = X - eta * deblur_grad(K, X, Y, L, lam)
    losses.append(deblur_loss(K, X, Y, L, lam))
    return X, losses


def deblur_pinv(AV, AH, B, L, rtol=None):
    """X = A_V^dagger *w B *w (A_H^T)^dagger for A_V (p, n1, n1), A_H (p, n2, n2)
    and B (p, n1, n2); `rtol` is the pseudo-inverse cut-off of `wpinv`."""
    PV = wpinv(AV, L, rtol)
    PHt = wpinv(transpose(AH), L, rtol)
    return wprod(wprod(PV, B, L), PHt, L)
