"""Error metrics (test oracle).

rel_fro: relative Frobenius error ||X - Y||_F / ||Y||_F, the parity measure.
psnr: Sec. IV-A, 10 log10(N * MPP / ||X1 - X2||_F^2) with N the element count.
The paper writes MPP, not MPP^2; the data used here is min-max normalised to
[0, 1], so MPP = 1 and both forms agree.
"""

import numpy as np


def rel_fro(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref.ravel())
    num = np.linalg.norm((x - ref).ravel())
    return float(num / den) if den > 0 else float(num)


def psnr(x1, x2, mpp=1.0):
    x1 = np.asarray(x1, dtype=np.float64)
    x2 = np.asarray(x2, dtype=np.float64)
    err = float(np.sum((x1 - x2) ** 2))
    if err == 0.0:
        return float("inf")
    return float(10.0 * np.log10(x1.size * mpp / err))
