"""FP64 CPU oracle for the w-product hot path (arXiv 2601.08228).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's definitions in NumPy float64.  It exists so that the
CUDA path can be checked against something written independently of it.  Only
`tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / `--impl reference`
legs of `bench.py` may import it; the product path (`paper_2601_08228_gb300`)
never does, and shares no code with it.

Layout convention: a third-order tensor A in R^{n1 x n2 x p} is stored
slice-major, as an array of shape (p, n1, n2): A[k] is the k-th frontal slice
A(:, :, k+1) of the paper (Sec. II, first paragraph).  Wavelet-domain tensors
use the Mallat coefficient order (s_L, d_L, d_{L-1}, ..., d_1) of Eq. (1).

Modules:
  lifting    forward / inverse lazy-Haar lifting and their adjoints (Eq. 1-3,
             Algorithm 1 forward and inverse loops)
  dense      the lifting transform as an explicit p x p matrix built from the
             per-level block matrices W_j (Eq. 2); an independent formulation
  wproduct   face-product, w-product (Def. 2.1), transpose (Def. 2.2),
             identity (Def. 2.3), trace (Def. 2.7)
  wsvd       truncated w-svd (Algorithm 2, Thm 2.5) and sp-w-svd (Sec. IV-B)
  wpinv      Moore-Penrose inverse under the w-product (Def. 2.6, Thm 2.6)
  grad       gradient of <G, A *w B> with respect to A and B (adjoint route)
  deblur     two-sided pseudo-inverse deblurring A_V^+ *w B *w (A_H^T)^+ and the
             gradient-descent objective ||K *w X - Y||^2 + lam||X||^2
  metrics    relative Frobenius error, PSNR (Sec. IV-A)
  quant      emulation of the FP8 (E4M3, one scale per slice) face-product
  glifting   lifting with general per-level predict / update operators
             (Eq. 2-3 with arbitrary P_j, U_j; Example 2.1, Remark 3.1), its
             adjoints, the w-product and gradient built on it

Pinned by tests/test_oracle_*.py against the paper's worked examples
(Example 2.2, Remark 2.2), closed forms and invariants; the E4M3 rounding of
`quant` against the format's own value table and PyTorch's float8_e4m3fn;
`glifting` against the Haar oracle (its lazy-Haar case), perfect
reconstruction, its dense block-matrix form and brute-force probing.  Nothing here is
"parity unpinned".
"""

from .lifting import lift, ilift, lift_adjoint, ilift_adjoint, split_mallat, check_levels
from .dense import dense_lifting_matrix
from .wproduct import facewise, wprod, transpose, identity, trace
from .wsvd import wsvd, spwsvd
from .wpinv import wpinv
from .grad import wprod_grad
from .deblur import deblur_loss, deblur_grad, deblur_steps, deblur_pinv
from .metrics import rel_fro, psnr
from .quant import e4m3_round, facewise_fp8, wprod_fp8
from . import glifting

__all__ = [
    "lift", "ilift", "lift_adjoint", "ilift_adjoint", "split_mallat", "check_levels",
    "dense_lifting_matrix", "facewise", "wprod", "transpose", "identity", "trace",
    "wsvd", "spwsvd", "wpinv", "wprod_grad", "deblur_loss", "deblur_grad",
    "deblur_steps", "deblur_pinv", "rel_fro", "psnr", "e4m3_round", "facewise_fp8", "wprod_fp8", "glifting",
]
