"""Seeded synthetic inputs for the w-product workloads.

This module only draws random numbers and builds closed-form arrays (Gaussian
spectral bumps, a Toeplitz blur matrix).  It contains none of the method's
arithmetic (no lifting, no face-products), so both the CUDA path and the FP64
oracle can take their inputs from it without sharing any of the computation.

Every tensor is returned slice-major, shape (p, rows, cols), C-contiguous:
element [k, i, j] is A[i+1, j+1, k+1] in the paper's notation (Sec. II).

Recipes (the paper's own data are hyperspectral images that are not available
here; these stand in for them with the same shapes and structure):

  plain_pair      A, B iid U[-1, 1] from one generator, A drawn before B, each
                  drawn in paper index order (n1, n2, p) and then made
                  slice-major.
  hsi_cube        rank-R sum of outer products u_r o v_r o t_r with
                  u_r, v_r ~ N(0, I) and smooth spectral tubes
                  t_r[k] = sum_{b=1..5} a_b exp(-(k - c_b)^2 / (2 w_b^2)),
                  a_b ~ U[0.5, 1], c_b ~ U[0, p), w_b ~ U[4, 24]; plus
                  noise * std(X) * N(0, 1); min-max normalised to [0, 1].
  scaled_pair     A, B iid N(0, 1), every spatial frontal slice of each
                  scaled by 10^U[-3, 3] (draw order: A, A scales, B, B scales).
  blur_operator   K[k] = T for all k, T the n x n banded Toeplitz matrix of the
                  normalised 9-tap Gaussian (sigma = 2): T_ij = g(|i - j|).
  batch_items     uneven items: n1, n2, n4 ~ U{16..64}, p ~ U{32, 64, 128},
                  L ~ U{1..log2(p) - 2}; A ~ U[-1, 1]^(p, n1, n2),
                  B ~ U[-1, 1]^(p, n2, n4).  All shapes are drawn first, then
                  A and B item by item.
"""

import math

import numpy as np


def _slice_major(x_paper):
    """(n1, n2, p) paper index order -> (p, n1, n2) contiguous."""
    return np.ascontiguousarray(np.moveaxis(x_paper, 2, 0))


def plain_pair(n1=32, n2=32, n4=32, p=16, seed=0, dtype=np.float64):
    """Two iid U[-1, 1] tensors A (p, n1, n2) and B (p, n2, n4)."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1.0, 1.0, size=(n1, n2, p))
    B = rng.uniform(-1.0, 1.0, size=(n2, n4, p))
    return _slice_major(A).astype(dtype), _slice_major(B).astype(dtype)


def spectral_tubes(rank, p, rng, bumps=5):
    """Smooth spectral tubes t_r[k], k = 0..p-1: sums of Gaussian bumps."""
    k = np.arange(p, dtype=np.float64)
    T = np.zeros((rank, p))
    for r in range(rank):
        a = rng.uniform(0.5, 1.0, size=bumps)
        c = rng.uniform(0.0, p, size=bumps)
        w = rng.uniform(4.0, 24.0, size=bumps)
        T[r] = np.sum(a[:, None] * np.exp(-((k[None, :] - c[:, None]) ** 2) / (2.0 * w[:, None] ** 2)), axis=0)
    return T


def hsi_cube(n1=256, n2=256, p=192, rank=20, noise=0.01, seed=0, dtype=np.float64,
             return_clean=False):
    """Synthetic hyperspectral cube (p, n1, n2) in [0, 1]; see module doc."""
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((rank, n1))
    V = rng.standard_normal((rank, n2))
    T = spectral_tubes(rank, p, rng)
    X = np.einsum("rk,ri,rj->kij", T, U, V, optimize=True)
    A = X + noise * X.std() * rng.standard_normal(X.shape) if noise > 0 else X.copy()
    lo, hi = A.min(), A.max()
    A = (A - lo) / (hi - lo)
    if return_clean:
        Xc = (X - lo) / (hi - lo)
        return A.astype(dtype), Xc.astype(dtype)
    return A.astype(dtype)


def scaled_pair(n1=1024, n2=1024, n4=512, p=256, seed=0, dtype=np.float32):
    """A (p, n1, n2), B (p, n2, n4): N(0, 1) with per-slice 10^U[-3, 3] scales."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((p, n1, n2), dtype=np.float32)
    sa = 10.0 ** rng.uniform(-3.0, 3.0, size=p)
    B = rng.standard_normal((p, n2, n4), dtype=np.float32)
    sb = 10.0 ** rng.uniform(-3.0, 3.0, size=p)
    A *= sa.astype(np.float32)[:, None, None]
    B *= sb.astype(np.float32)[:, None, None]
    return A.astype(dtype, copy=False), B.astype(dtype, copy=False)


def gaussian_taps(sigma=2.0, taps=9):
    half = taps // 2
    x = np.arange(-half, half + 1, dtype=np.float64)
    g = np.exp(-(x ** 2) / (2.0 * sigma ** 2))
    return g / g.sum()


def blur_operator(n, p, sigma=2.0, taps=9, dtype=np.float64):
    """Band-constant blur tensor K (p, n, n): the same Toeplitz T in every band."""
    g = gaussian_taps(sigma, taps)
    half = taps // 2
    T = np.zeros((n, n))
    for off in range(-half, half + 1):
        T += np.diag(np.full(n - abs(off), g[off + half]), k=off)
    return np.ascontiguousarray(np.broadcast_to(T, (p, n, n))).astype(dtype)


def linear_blur_operator(n, p, b=10, dtype=np.float64):
    """Band-constant linear blur tensor (p, n, n) of the two-sided deblurring
    experiment (Sec. IV-C): Toeplitz with entries c(|i - j|), c(k) = (b - k) / (3 b)
    for 0 <= k < b and 0 beyond, as printed (rows sum to about 10/3 at b = 10)."""
    c = np.array([(b - k) / (3.0 * b) if k < b else 0.0 for k in range(n)])
    i = np.arange(n)
    T = c[np.abs(i[:, None] - i[None, :])]
    return np.ascontiguousarray(np.broadcast_to(T, (p, n, n))).astype(dtype)


def unit_noise(shape, seed, dtype=np.float64):
    """iid N(0, 1) array of the given shape."""
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


def batch_shapes(count=4096, seed=1):
    """Draw the (n1, n2, n4, p, L) tuples of the uneven batch."""
    rng = np.random.default_rng(seed)
    shapes = []
    for _ in range(count):
        n1 = int(rng.integers(16, 65))
        n2 = int(rng.integers(16, 65))
        n4 = int(rng.integers(16, 65))
        p = int(rng.choice([32, 64, 128]))
        L = int(rng.integers(1, int(math.log2(p)) - 2 + 1))
        shapes.append((n1, n2, n4, p, L))
    return shapes, rng


def batch_items(count=4096, seed=1, dtype=np.float32):
    """Uneven batch: list of dicts with A, B, shapes; see module doc."""
    shapes, rng = batch_shapes(count, seed)
    items = []
    for (n1, n2, n4, p, L) in shapes:
        A = rng.uniform(-1.0, 1.0, size=(p, n1, n2)).astype(dtype)
        B = rng.uniform(-1.0, 1.0, size=(p, n2, n4)).astype(dtype)
        items.append(dict(n1=n1, n2=n2, n4=n4, p=p, L=L, A=A, B=B))
    return items
