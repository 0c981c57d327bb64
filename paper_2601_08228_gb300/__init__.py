"""GB300-native (sm_103a) w-product library for arXiv 2601.08228.

The compute path is libwprod.so (hand-written CUDA behind the C ABI of
include/wprod.h); `capi` is its thin ctypes binding and `autograd` wraps the
w-product in a torch.autograd.Function with the hand-written adjoint
backward.  `synth` holds the seeded synthetic input generators.
"""

from .capi import (  # noqa: F401
    PREC, WPError, lib, wp_deblur_pinv, wp_deblur_step, wp_deblur_workspace, wp_facewise, wp_get_device_error,
    wp_lift_adjoint, wp_lift_forward, wp_lift_inverse, wp_wpinv, wp_wprod, wp_wprod_backward,
    wp_wprod_host, wp_wprod_host_workspace, wp_wprod_noalloc, wp_wprod_workspace, wp_wsvd,
)
from .autograd import WProd, wprod  # noqa: F401
