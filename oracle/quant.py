"""FP8 (E4M3) emulation of the face-product with one scale per slice (test oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper computes its face-products in floating point without fixing a
format; the FP8 variant is this project's reduced-precision mode, defined as:
every wavelet-domain slice X_k of each operand gets the scale
s_k = max|X_k| / 448 (448 = largest finite E4M3 value; s_k = 1 for an all-zero
slice), its entries become the E4M3 values q = rn(X_k / s_k), and
C_k = s_k^A s_k^B (q^A_k q^B_k).  The quantisation is a decision taken in the
kernel's precision, so this emulation takes it the same way: single-precision
coefficients (lift in float32), s_k and 1 / s_k rounded to float32, the
scaled value x * (1 / s_k) rounded to float32, then rounded to the nearest
E4M3 value (ties to an even mantissa), saturating at +-448.  The products of
E4M3 codes and everything after them are exact here (float64), so the
emulation differs from an FP32-accumulating GPU only by accumulation rounding.

E4M3 ("E4M3FN" of the OCP 8-bit floating-point specification): 1 sign bit, 4
exponent bits with bias 7, 3 mantissa bits; normal values 2^(e-7) (1 + f/8)
for e = 1..15 except the all-ones pattern (e = 15, f = 7), which is NaN;
subnormals 2^-6 (f/8); no infinities.  Largest finite value 448 = 2^8 * 1.75,
smallest subnormal 2^-9.
"""

import numpy as np

from .lifting import lift, ilift, check_levels

E4M3_MAX = 448.0


def e4m3_round(x):
    """Round float values to the nearest E4M3 value (ties to even), saturating
    finite overflow to +-448.  Returns float64."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    # quantum: 2^(E - 3) in the binade [2^E, 2^(E+1)), E >= -6; 2^-9 below
    _, e = np.frexp(np.where(a > 0, a, 1.0))          # a = f 2^e, f in [0.5, 1)
    E = np.maximum(e - 1, -6)
    quantum = np.ldexp(1.0, E - 3)
    q = np.round(a / quantum) * quantum                # np.round: ties to even
    q = np.minimum(q, E4M3_MAX)
    return np.copysign(q, x)


def slice_scales(Xh32):
    """Per-slice scale s_k = max|X_k| / 448 in float32 (1 for an all-zero slice)."""
    amax = np.abs(Xh32).reshape(Xh32.shape[0], -1).max(axis=1).astype(np.float32)
    s = amax / np.float32(E4M3_MAX)
    return np.where(amax > 0, s, np.float32(1.0)).astype(np.float32)


def quantize(Xh32):
    """(E4M3 values q as float64, float32 scales s) of a float32 slice stack."""
    Xh32 = np.asarray(Xh32, dtype=np.float32)
    s = slice_scales(Xh32)
    inv = (np.float32(1.0) / s).astype(np.float32)
    y = (Xh32 * inv[:, None, None]).astype(np.float32)
    return e4m3_round(y), s


def facewise_fp8(Ah32, Bh32):
    """FP8 face-product of float32 slice stacks Ah (p, n1, n2), Bh (p, n2, n4)."""
    qa, sa = quantize(Ah32)
    qb, sb = quantize(Bh32)
    scale = (sa * sb).astype(np.float32).astype(np.float64)
    C = np.empty((qa.shape[0], qa.shape[1], qb.shape[2]))
    for k in range(qa.shape[0]):
        C[k] = (qa[k] @ qb[k]) * scale[k]
    return C


def wprod_fp8(A, B, L):
    """FP8 w-product W^{-1}(FP8 face-product of W(A), W(B)) (Def. 2.1 with the
    face-product above); the forward transform in float32, the rest float64."""
    A = np.asarray(A, dtype=np.float32)
    B = np.asarray(B, dtype=np.float32)
    check_levels(A.shape[0], L)
    return ilift(facewise_fp8(lift(A, L, np.float32), lift(B, L, np.float32)), L)
