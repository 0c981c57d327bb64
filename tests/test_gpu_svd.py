"""GPU parity of the batched Jacobi w-svd, sp-w-svd and wpinv against the FP64
oracle.  Tolerances (relative Frobenius): singular values 1e-4 (the stated
SVD bar); rank-r reconstructions and factor products U Sigma V^T per slice
1e-4, widened where the truncation itself is ill-conditioned: by the
Davis-Kahan bound an FP32 SVD with backward error ~sqrt(m) eps |A| moves the
rank-r subspace by ~sqrt(m) eps sigma_1 / (sigma_r - sigma_r+1), so the bar is
max(1e-4, 4 sqrt(m) eps max_k sigma_1 / gap_k); orthonormality 1e-5 sqrt(m).  Singular vectors are compared only through
sign-free quantities.  sp-w-svd's slice selection (which slices are kept,
which zeroed) is checked bit for bit on the wavelet-domain factors."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_08228_gb300 import capi, synth
from tests import _golden

pytestmark = pytest.mark.gpu

TOL_SIG = 1e-4
TOL_REC = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2601_08228_gb300 import build
    build.build()
    capi.lib()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(size=shape).astype(np.float32)


SVD_CASES = [
    # p, n1, n2, L, r
    (8, 16, 16, 3, 4),
    (24, 40, 24, 3, 5),      # tall slices: left vectors from Jacobi
    (24, 24, 40, 3, 5),      # wide slices: right vectors from Jacobi
    (12, 33, 17, 2, 17),     # full rank, odd column count (padded pair)
    (16, 64, 64, 4, 8),
    (6, 1, 5, 1, 1),         # single-row slices
    (4, 150, 130, 2, 10),    # cluster path
    (2, 256, 256, 1, 20),
    (2, 320, 300, 1, 10),    # more than 256 columns: 16-column blocks, 8-CTA cluster
]


def _rec_tol(A, L, r, nsl):
    """Gap-aware reconstruction bar (see the module docstring)."""
    s = np.linalg.svd(O.lift(A, L)[:nsl], compute_uv=False)
    m = max(A.shape[1], A.shape[2])
    if r >= s.shape[1]:
        return TOL_REC
    ratio = float(np.max(s[:, 0] / np.maximum(s[:, r - 1] - s[:, r], 1e-30)))
    return max(TOL_REC, 4 * np.sqrt(m) * 1.2e-7 * ratio)


@pytest.mark.parametrize("p,n1,n2,L,r", SVD_CASES)
@pytest.mark.parametrize("sparse", [False, True])
def test_wsvd_parity(p, n1, n2, L, r, sparse):
    A = rand((p, n1, n2), p + n1 + n2)
    C, U, S, V = capi.wp_wsvd(dev(A), L, r, sparse=sparse, factors=True)
    fn = O.spwsvd if sparse else O.wsvd
    Cr, Ur, Sr, Vr = fn(A, L, r, return_factors=True)
    nsl_ = min(2 * (p >> L), p) if sparse else p
    tol_rec = _rec_tol(A, L, r, nsl_)
    assert O.rel_fro(host(C), Cr) <= tol_rec
    assert O.rel_fro(host(S), Sr) <= TOL_SIG
    U, S, V = host(U), host(S), host(V)
    m = p >> L
    nsl = min(2 * m, p) if sparse else p
    # bit-exact selection: slices beyond the kept set are exactly zero
    assert np.all(U[nsl:] == 0) and np.all(S[nsl:] == 0) and np.all(V[nsl:] == 0)
    # every kept slice has r strictly positive, descending singular values
    assert np.all(S[:nsl] > 0) and np.all(np.diff(S[:nsl], axis=1) <= 0)
    # factor products reproduce the oracle's truncated slices; orthonormal columns
    Ch_gpu = np.einsum("kir,kr,kjr->kij", U, S, V)
    Ch_ref = np.einsum("kir,kr,kjr->kij", Ur, Sr, Vr)
    assert O.rel_fro(Ch_gpu, Ch_ref) <= tol_rec
    assert capi.wp_get_device_error() == 0
    eye = np.broadcast_to(np.eye(r), (nsl, r, r))
    assert np.max(np.abs(np.einsum("kir,kis->krs", U[:nsl], U[:nsl]) - eye)) <= 1e-5 * max(n1, n2)
    assert np.max(np.abs(np.einsum("kir,kis->krs", V[:nsl], V[:nsl]) - eye)) <= 1e-5 * max(n1, n2)


def test_wsvd_spatial_factors_thm_2_5():
    """Spatial-domain factors (Thm 2.5): U *w Sigma *w V^T equals C_r."""
    p, n1, n2, L, r = 16, 20, 12, 3, 4
    A = rand((p, n1, n2), 5)
    C, U, S, V = capi.wp_wsvd(dev(A), L, r, factors=True, factors_in_wavelet_domain=False)
    U, S, V = host(U), host(S), host(V)
    Sig = np.zeros((p, r, r))
    for k in range(p):
        Sig[k] = np.diag(S[k])
    rec = O.wprod(O.wprod(U, Sig, L), V, L, transB=True)
    assert O.rel_fro(rec, host(C)) <= TOL_REC
    assert O.rel_fro(host(C), O.wsvd(A, L, r)) <= TOL_REC


@pytest.mark.parametrize("r", [5, 10, 20])
def test_wsvd_hsi_256x256x192(r):
    """Synthetic HSI cube 256x256x192, L = 3, ranks 5/10/20; w-svd and
    sp-w-svd in the benchmark's launch configuration; PSNR equal to the
    oracle's to 1e-3 dB."""
    A = synth.hsi_cube(256, 256, 192, seed=0, dtype=np.float32)
    Ad = dev(A)
    for sparse, fn in ((False, O.wsvd), (True, O.spwsvd)):
        C = host(capi.wp_wsvd(Ad, 3, r, sparse=sparse))
        ref = fn(A, 3, r)
        assert O.rel_fro(C, ref) <= TOL_REC
        assert abs(O.psnr(C, A) - O.psnr(ref, A)) <= 1e-3
    assert capi.wp_get_device_error() == 0


def test_rank_deficient_slices_converge():
    """Collinear and zero columns (rank-deficient wavelet-domain slices) must
    not keep the Jacobi sweeps rotating rounding noise: no NOT_CONVERGED."""
    p, L, n = 8, 3, 24
    rng = np.random.default_rng(21)
    Ah = np.einsum("kir,krj->kij", rng.standard_normal((p, n, 3)), rng.standard_normal((p, 3, n)))
    Ah[:, :, 5] = Ah[:, :, 4]            # duplicated column
    Ah[:, :, 7] = 0.0                    # zero column
    A = O.ilift(Ah, L).astype(np.float32)
    capi.wp_get_device_error()
    C = host(capi.wp_wsvd(dev(A), L, 3))
    assert O.rel_fro(C, O.wsvd(A, L, 3)) <= 1e-4
    # FP32 rounding leaves noise singular values ~1e-7 sigma_1 in the rank-3
    # slices: compare at the GPU's cut-off max(m, n) eps_32, not the FP64 one
    X = host(capi.wp_wpinv(dev(A), L))
    assert O.rel_fro(X, O.wpinv(A, L, rtol=n * 1.1920929e-7)) <= 1e-3
    assert capi.wp_get_device_error() == 0


def test_wsvd_rank_errors():
    A = torch.zeros((8, 4, 6), device="cuda")
    for r in (0, 5):
        with pytest.raises(capi.WPError) as e:
            capi.wp_wsvd(A, 3, r)
        assert e.value.status == 4


# ---- Moore-Penrose inverse ------------------------------------------------------

def test_wpinv_remark_2_2():
    rem = _golden.load("remark_2_2.txt")
    AB = O.wprod(rem["A"], rem["B"], 1)
    C = host(capi.wp_wpinv(dev(AB), 1))
    np.testing.assert_allclose(C, rem["C"], atol=0.005)
    Ad = host(capi.wp_wpinv(dev(rem["A"]), 1))
    Bd = host(capi.wp_wpinv(dev(rem["B"]), 1))
    np.testing.assert_allclose(O.wprod(Bd, Ad, 1), rem["D"], atol=0.005)


PINV_CASES = [(8, 12, 7, 3), (8, 7, 12, 3), (24, 30, 22, 3), (24, 30, 30, 3), (16, 64, 40, 4), (4, 1, 6, 2),
              (8, 40, 72, 3), (8, 48, 48, 3)]   # the last two: wide and square slices of 32+ columns


def _kappa(A, L):
    """Largest condition number over the wavelet-domain slices."""
    s = np.linalg.svd(O.lift(A, L), compute_uv=False)
    return float(np.max(s[:, 0] / s[:, -1]))


@pytest.mark.parametrize("p,m,n,L", PINV_CASES)
@pytest.mark.parametrize("refine", [0, 2])
def test_wpinv_parity_and_penrose(p, m, n, L, refine):
    """Without refinement an FP32 pseudo-inverse is accurate to ~kappa eps
    (kappa: worst wavelet-slice condition number) and its Penrose residuals
    to ~kappa^2 eps; the refinement (compensated residuals) brings X to the 1e-4 bar and
    the residuals to ~kappa eps (the FP32 representation limit of X)."""
    A = rand((p, m, n), m * n + p)
    X = host(capi.wp_wpinv(dev(A), L, refine_iters=refine))
    ref = O.wpinv(A, L)
    kap, eps = _kappa(A, L), 1.2e-7
    tol = 1e-4 if refine else max(1e-4, 8 * kap * eps)
    tol_pen = max(1e-4, 8 * kap * eps) if refine else max(1e-4, 8 * kap * kap * eps)
    assert O.rel_fro(X, ref) <= tol
    AX, XA = O.wprod(A, X, L), O.wprod(X, A, L)
    assert O.rel_fro(O.wprod(AX, A, L), A) <= tol_pen
    assert O.rel_fro(O.wprod(XA, X, L), X) <= tol_pen
    assert O.rel_fro(O.transpose(AX), AX) <= tol_pen
    assert O.rel_fro(O.transpose(XA), XA) <= tol_pen
    assert capi.wp_get_device_error() == 0


def test_wpinv_refinement_reduces_error():
    p, m, n, L = 8, 48, 32, 3
    rng = np.random.default_rng(3)
    # moderately ill-conditioned slices in the wavelet domain
    Ah = np.einsum("kij,kj,klj->kil", rng.standard_normal((p, m, n)), np.logspace(0, -3, n)[None].repeat(p, 0),
                   np.linalg.qr(rng.standard_normal((p, n, n)))[0])
    A = O.ilift(Ah, L).astype(np.float32)
    ref = O.wpinv(A, L)
    e0 = O.rel_fro(host(capi.wp_wpinv(dev(A), L, refine_iters=0)), ref)
    e2 = O.rel_fro(host(capi.wp_wpinv(dev(A), L, refine_iters=2)), ref)
    assert e2 <= e0 and e2 <= 1e-3
    assert capi.wp_get_device_error() == 0


def test_wpinv_invertible_gives_identity():
    """Def. 2.4 via Thm 2.6.  A is made well conditioned in the wavelet
    domain (A_hat_k = R_k + 4 I); a spatial A + 4 I would not be, because the
    detail slices difference the 4 I away."""
    p, n, L = 8, 16, 3
    A = O.ilift(rand((p, n, n), 9) + 4 * np.eye(n), L).astype(np.float32)
    X = host(capi.wp_wpinv(dev(A), L, refine_iters=2))
    # even the FP32-rounded exact inverse leaves |A X - I| ~ kappa eps
    tol = max(1e-5, 8 * _kappa(A, L) * 1.2e-7)
    assert O.rel_fro(O.wprod(A, X, L), O.identity(n, p, L)) <= tol
    assert capi.wp_get_device_error() == 0


# ---- failure detection: sweep limit and bounded waits ---------------------------

@pytest.mark.parametrize("p,n1,n2,L,r", [(8, 40, 24, 3, 5), (4, 150, 130, 2, 10)])
def test_jacobi_sweep_limit_reports_not_converged(p, n1, n2, L, r):
    """With the sweep limit at 1 the Jacobi iteration on random slices cannot
    converge: the kernels must stop after one sweep and report
    WP_ERR_NOT_CONVERGED through the device status word (the narrow slices
    run the shared-memory kernel, the wide ones the block-cyclic kernel)."""
    A = dev(rand((p, n1, n2), 31))
    assert capi.wp_get_device_error() == capi.WP_OK
    capi.wp_set_jacobi_max_sweeps(1)
    try:
        capi.wp_wsvd(A, L, r)
        assert capi.wp_get_device_error() == capi.WP_ERR_NOT_CONVERGED
    finally:
        capi.wp_set_jacobi_max_sweeps(40)
    # back at the default limit the same call converges and matches the oracle
    Cr = host(capi.wp_wsvd(A, L, r))
    assert capi.wp_get_device_error() == capi.WP_OK
    ref = O.wsvd(host(A), L, r)
    assert O.rel_fro(Cr, ref) <= _rec_tol(host(A), L, r, p)


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_expiry_reports_timeout(which):
    """A bounded wait on a barrier that nothing completes expires after 1 ms,
    records WP_ERR_TIMEOUT and returns: the context stays usable and the
    status word is cleared by the read."""
    assert capi.wp_get_device_error() == capi.WP_OK
    capi.wp_selftest_bounded_wait(which, 1_000_000)
    assert capi.wp_get_device_error() == capi.WP_ERR_TIMEOUT
    assert capi.wp_get_device_error() == capi.WP_OK
    A, B = rand((8, 16, 12), 1), rand((8, 12, 10), 2)
    C = host(capi.wp_wprod(dev(A), dev(B), 3))
    assert O.rel_fro(C, O.wprod(A, B, 3)) <= 1e-5


# ---- slices larger than a cluster's shared memory (global-memory Jacobi) ---------

BIG_CASES = [
    # p, n1, n2, L, r   (n1 * n2 > ~400k: beyond the 8-CTA cluster kernels)
    (2, 640, 640, 1, 12),     # square, 16-column blocks
    (4, 700, 600, 2, 30),     # tall: left vectors from Jacobi
    (2, 600, 700, 1, 8),      # wide: the working columns are the slice's rows
    (2, 1700, 260, 1, 5),     # 1700 rows: 8-column blocks
]


@pytest.mark.parametrize("p,n1,n2,L,r", BIG_CASES)
def test_wsvd_large_slices(p, n1, n2, L, r):
    A = rand((p, n1, n2), n1 + n2)
    C, U, S, V = capi.wp_wsvd(dev(A), L, r, factors=True)
    Cr, Ur, Sr, Vr = O.wsvd(A, L, r, return_factors=True)
    assert O.rel_fro(host(S), Sr) <= TOL_SIG
    assert O.rel_fro(host(C), Cr) <= _rec_tol(A, L, r, p)
    assert capi.wp_get_device_error() == 0


def test_wpinv_large_square_slice():
    """A 640 x 640 slice pair, inverted through the global-memory Jacobi, then
    refined: the Penrose equations at the kappa-aware bars."""
    p, n, L = 2, 640, 1
    A = rand((p, n, n), 77)
    X = host(capi.wp_wpinv(dev(A), L, refine_iters=2))
    kap, eps = _kappa(A, L), 1.2e-7
    assert O.rel_fro(X, O.wpinv(A, L)) <= max(1e-4, 8 * kap * eps)
    AX = O.wprod(A, X, L)
    assert O.rel_fro(O.wprod(AX, A, L), A) <= max(1e-4, 8 * kap * eps)
    assert capi.wp_get_device_error() == 0


def test_wpinv_zero_detail_slices_large():
    """A band-constant operator (zero detail slices, as the blur operators of
    Sec. IV-C) with 610 x 610 slices: the zero slices converge at once and
    their pseudo-inverse is zero; the result matches the oracle."""
    p, n, L = 4, 610, 1
    T = np.random.default_rng(5).standard_normal((n, n)).astype(np.float32) + 30 * np.eye(n, dtype=np.float32)
    A = np.broadcast_to(T, (p, n, n)).copy()
    X = host(capi.wp_wpinv(dev(A), L, refine_iters=1))
    assert O.rel_fro(X, O.wpinv(A, L)) <= 1e-4
    assert capi.wp_get_device_error() == 0


@pytest.mark.parametrize("n1,n2", [(96, 96), (120, 64), (64, 120)])
def test_qr_preconditioning_fewer_sweeps_same_result(n1, n2):
    """The QR-preconditioned Jacobi (on the columns of R^T) needs fewer
    sweeps than the Jacobi on the slices themselves and gives the same
    singular values and rank-r reconstruction, within the SVD bars, against
    the oracle."""
    p, L, r = 48, 3, 10
    A = synth.hsi_cube(n1, n2, p, seed=3, dtype=np.float32)
    Ad = dev(A)
    res = {}
    try:
        for pre in (False, True):
            capi.wp_set_jacobi_precondition(pre)
            capi.wp_jacobi_stats()
            C, _, S, _ = capi.wp_wsvd(Ad, L, r, factors=True)
            torch.cuda.synchronize()
            res[pre] = (host(C), host(S), capi.wp_jacobi_stats()[0])
    finally:
        capi.wp_set_jacobi_precondition(True)
    Cr, _, Sr, _ = O.wsvd(A, L, r, return_factors=True)
    tol = _rec_tol(A.astype(np.float64), L, r, p)
    for pre in (False, True):
        assert O.rel_fro(res[pre][1], Sr) <= TOL_SIG
        assert O.rel_fro(res[pre][0], Cr) <= tol
    assert res[True][2] < res[False][2]
    assert capi.wp_get_device_error() == 0


@pytest.mark.parametrize("n1,n2,pre,p", [(256, 256, True, 48), (256, 250, True, 48), (256, 200, False, 48),
                                         (200, 256, False, 48), (256, 256, True, 16), (256, 256, True, 96),
                                         (256, 256, True, 192)])
def test_jacobi_column_split_matches_row_split(n1, n2, pre, p):
    """The column-split kernel (whole columns per CTA, 8 rows per lane) and
    the row-split block kernel compute the same one-sided Jacobi SVD in a
    different pair order: both meet the SVD bars against the oracle, on the
    QR path (R^T of 256 and of 250 columns, the latter padded to 256) and on
    tall and wide slices without it (200 columns padded to 208; the wide one
    works on the transpose).  The slice counts take the automatic cluster
    sizes' cases on a 152-SM GPU: 16 slices in one wave of 4-CTA clusters,
    48 as a wave of 3-CTA clusters plus two 2-CTA clusters beside it, 96 and
    192 as full waves of 2-CTA clusters plus the rest on 3-CTA clusters."""
    L, r = 3, 20
    A = synth.hsi_cube(n1, n2, p, seed=4, dtype=np.float32)
    Ad = dev(A)
    res = {}
    try:
        capi.wp_set_jacobi_precondition(pre)
        for split in (False, True):
            capi.wp_set_jacobi_column_split(split)
            capi.wp_jacobi_stats()
            C, _, S, _ = capi.wp_wsvd(Ad, L, r, factors=True)
            torch.cuda.synchronize()
            res[split] = (host(C), host(S), capi.wp_jacobi_stats())
            assert capi.wp_get_device_error() == 0
    finally:
        capi.wp_set_jacobi_precondition(True)
        capi.wp_set_jacobi_column_split(True)
    Cr, _, Sr, _ = O.wsvd(A, L, r, return_factors=True)
    tol = _rec_tol(A.astype(np.float64), L, r, p)
    for split in (False, True):
        print(f"{n1}x{n2} pre={pre} split={split}: sig {O.rel_fro(res[split][1], Sr):.2e} "
              f"C_r {O.rel_fro(res[split][0], Cr):.2e} sweeps {res[split][2]}")
        assert O.rel_fro(res[split][1], Sr) <= TOL_SIG
        assert O.rel_fro(res[split][0], Cr) <= tol
    # same method: sweep counts within one per slice of each other
    assert abs(res[True][2][0] - res[False][2][0]) <= p


@pytest.mark.parametrize("cl", [2, 3, 4])
def test_jacobi_column_split_each_cluster_size(cl):
    """Every launch of the column-split kernel forced onto clusters of 2, 3
    or 4 CTAs (CTA boundaries at different warps, 1..3 boundaries): the same
    SVD, within the bars, against the oracle; 24 slices of 256 x 256, R^T
    path, ranks 20."""
    p, L, r = 24, 3, 20
    A = synth.hsi_cube(256, 256, p, seed=6, dtype=np.float32)
    try:
        capi.wp_set_jacobi_cluster_size(cl)
        assert capi.wp_jacobi_cluster_capacity(cl) > 0
        C, _, S, _ = capi.wp_wsvd(dev(A), L, r, factors=True)
        torch.cuda.synchronize()
        assert capi.wp_get_device_error() == 0
    finally:
        capi.wp_set_jacobi_cluster_size(0)
    Cr, _, Sr, _ = O.wsvd(A, L, r, return_factors=True)
    assert O.rel_fro(host(S), Sr) <= TOL_SIG
    assert O.rel_fro(host(C), Cr) <= _rec_tol(A.astype(np.float64), L, r, p)


def test_wsvd_cuda_graph_with_paired_jacobi():
    """192 slices of 256 x 256: the QR on 2-CTA clusters and the Jacobi as
    two launches side by side, the second on the library's own stream,
    forked from and joined back to the call's stream with events.  The call
    captured in a CUDA graph (after one eager call, which sets up the side
    stream and the kernels' attributes) and replayed twice gives the eager
    result bit for bit."""
    import ctypes
    p, L, r = 192, 3, 20
    A = dev(synth.hsi_cube(256, 256, p, seed=2, dtype=np.float32))
    nb = ctypes.c_size_t(0)
    assert capi.lib().wp_wsvd_workspace(256, 256, p, L, r, ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        eager = capi.wp_wsvd(A, L, r, ws=ws)
    s.synchronize()
    eager = host(eager)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        Cg = capi.wp_wsvd(A, L, r, ws=ws)
    for _ in range(2):
        Cg.zero_()
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host(Cg), eager)
    assert capi.wp_get_device_error() == 0


@pytest.mark.parametrize("n1,n2", [(200, 193), (193, 200), (130, 77), (256, 33), (250, 250)])
def test_qr_preconditioned_ragged_shapes(n1, n2):
    """The register-resident cluster QR on working matrices whose column
    count is not a multiple of its 4-column panels (193, 77, 33, 250: zero
    padding columns), with fewer than 256 rows, and wide slices (the QR of
    the transpose); the Jacobi then takes R^T on the column-split kernel
    (193, 250 columns) or the row-split one (77, 33).  Singular values and
    the rank-r reconstruction against the oracle."""
    p, L, r = 16, 2, 10
    A = synth.hsi_cube(n1, n2, p, seed=12, dtype=np.float32)
    C, _, S, _ = capi.wp_wsvd(dev(A), L, r, factors=True)
    torch.cuda.synchronize()
    Cr, _, Sr, _ = O.wsvd(A, L, r, return_factors=True)
    assert O.rel_fro(host(S), Sr) <= TOL_SIG
    assert O.rel_fro(host(C), Cr) <= _rec_tol(A.astype(np.float64), L, r, p)
    assert capi.wp_get_device_error() == 0


@pytest.mark.parametrize("r", [3, 6])
@pytest.mark.parametrize("sparse", [False, True])
def test_qr_preconditioned_rank_deficient(r, sparse):
    """Exactly low-rank slices on the QR path: a noise-free rank-3 cube
    (rank 4 in the approximation slices with the normalisation's constant),
    so R has only a few rows above rounding level and R^T as many
    numerically-zero columns, which the Jacobi must leave alone (numerically
    zero rule) and still converge.  Ranks inside and beyond the numerical
    rank; w-svd and sp-w-svd; 48 slices of 256 x 256 (the column-split
    kernel's cluster policy)."""
    p, L = 48, 3
    A = synth.hsi_cube(256, 256, p, rank=3, noise=0.0, seed=13, dtype=np.float32)
    capi.wp_jacobi_stats()
    C, _, S, _ = capi.wp_wsvd(dev(A), L, r, sparse=sparse, factors=True)
    torch.cuda.synchronize()
    total, mx = capi.wp_jacobi_stats()
    fn = O.spwsvd if sparse else O.wsvd
    Cr, _, Sr, _ = fn(A, L, r, return_factors=True)
    assert 0 < mx < 40                    # converged well inside the default sweep limit
    nsl = min(2 * (p >> L), p) if sparse else p
    assert O.rel_fro(host(S), Sr) <= TOL_SIG
    assert O.rel_fro(host(C), Cr) <= max(1e-5, _rec_tol(A.astype(np.float64), L, r, nsl))
    assert capi.wp_get_device_error() == 0
