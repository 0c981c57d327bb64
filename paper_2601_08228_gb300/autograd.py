"""torch.autograd binding of the w-product with the hand-written backward.

WProd.forward calls wp_wprod; WProd.backward calls wp_wprod_backward, which
recomputes the wavelet-domain slices W(A), W(B) from the saved spatial
inputs (nothing wavelet-domain is kept between the passes) and applies the
adjoint lifting transforms W^T, W^{-T} -- not the inverse transform, since
the lifting is not orthogonal (Remark 2.1).
"""

import torch

from . import capi


class WProd(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, L, prec):
        ctx.L = int(L)
        ctx.prec = prec
        A = A.contiguous()
        B = B.contiguous()
        ctx.save_for_backward(A, B)
        return capi.wp_wprod(A, B, ctx.L, prec=prec)

    @staticmethod
    def backward(ctx, G):
        A, B = ctx.saved_tensors
        need_a, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_a or need_b):
            return None, None, None, None
        dA, dB = capi.wp_wprod_backward(A, B, G.contiguous(), ctx.L, need_dA=need_a, need_dB=need_b,
                                        prec=ctx.prec)
        return dA, dB, None, None


def wprod(A, B, L, prec="fp32"):
    """Differentiable C = A *w B (Def. 2.1) on the GPU."""
    return WProd.apply(A, B, L, prec)
