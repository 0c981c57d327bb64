"""CPU simulations of the index arithmetic of the streaming kernels (the
mappings from grid / block / thread indices to tensor elements, restated
from the kernels' formulas), checked for exact coverage and in-bounds
accesses over ragged shapes.  Compute-sanitizer is not available to these
builds; these checks stand in for its bounds checking."""

import itertools

import numpy as np
import pytest


def cdiv(a, b):
    return (a + b - 1) // b


# ---- lift_reg_kernel: grid-stride and group-fastest chunk orders -------------------

def lift_items(p, L, plane, vec, grid, gf, threads=256):
    """(g, e) visited by every (CTA, thread) of lift_reg_kernel."""
    G = 1 << L
    m = p >> L
    nvec = plane // vec
    total = m * nvec
    nchunk = cdiv(nvec, threads)
    seen = []
    for bx in range(grid):
        for t in range(threads):
            if gf:
                w, stride, nwork = bx, grid, m * nchunk
            else:
                w, stride, nwork = bx * threads + t, grid * threads, total
            while w < nwork:
                if gf:
                    g, iv = w % m, (w // m) * threads + t
                    if iv < nvec:
                        seen.append((g, iv * vec))
                else:
                    g, iv = w // nvec, w % nvec
                    seen.append((g, iv * vec))
                w += stride
    return seen


@pytest.mark.parametrize("p,L,plane,vec,grid", [(16, 4, 4096, 4, 7), (32, 5, 2 * 257, 2, 5), (24, 3, 85, 1, 3),
                                                (64, 4, 1000, 4, 9)])
@pytest.mark.parametrize("gf", [False, True])
def test_lift_chunk_orders_cover_every_item_once(p, L, plane, vec, grid, gf):
    seen = lift_items(p, L, plane, vec, grid, gf)
    want = {(g, e) for g in range(p >> L) for e in range(0, plane - vec + 1, vec)}
    assert len(seen) == len(set(seen)) == len(want) and set(seen) == want
    G = 1 << L
    assert all((g * G + G - 1) * plane + e + vec - 1 < p * plane for g, e in seen)


# ---- transpose_bytes_kernel: (batch, R, C) -> (batch, C, Rp) in 64 x 64 tiles -------

def transpose_bytes_accesses(R, C, Rp, batch, vec16):
    T = 64
    reads, writes = [], []
    for bz, by, bx in itertools.product(range(batch), range(cdiv(Rp, T)), range(cdiv(C, T))):
        c0, r0 = bx * T, by * T
        for tid in range(256):
            i, j = tid >> 2, (tid & 3) * 16
            r, c = r0 + i, c0 + j
            if r < R:
                if vec16 and c + 15 < C:
                    reads += [(bz, r, c + k) for k in range(16)]
                else:
                    reads += [(bz, r, c + k) for k in range(16) if c + k < C]
            cc, k = tid & 63, tid >> 6
            c, rs = c0 + cc, r0 + k * 16
            if c < C and rs < Rp:
                writes += [(bz, c, rs + q) for q in range(16)]
    return reads, writes


@pytest.mark.parametrize("R,C,batch", [(17, 40, 2), (64, 64, 1), (100, 33, 2), (16, 128, 1)])
def test_transpose_bytes_covers_the_output_once(R, C, batch):
    Rp = cdiv(R, 16) * 16
    for vec16 in ([False, True] if C % 16 == 0 else [False]):
        reads, writes = transpose_bytes_accesses(R, C, Rp, batch, vec16)
        assert all(r < R and c < C for _, r, c in reads)
        want = {(b, c, r) for b in range(batch) for c in range(C) for r in range(Rp)}
        assert len(writes) == len(set(writes)) and set(writes) == want


# ---- split_transpose4_kernel: (p, R, C) fp32 -> (p, C, Rp) bf16, 64 x 64 tiles -------

@pytest.mark.parametrize("R,C,Rp,batch", [(17, 40, 24, 2), (64, 64, 64, 1), (100, 36, 104, 1), (8, 132, 8, 1)])
def test_split_transpose4_covers_the_output_once(R, C, Rp, batch):
    assert C % 4 == 0 and Rp % 8 == 0 and Rp >= R
    T = 64
    writes, reads = [], []
    for b, by, bx in itertools.product(range(batch), range(cdiv(Rp, T)), range(cdiv(C, T))):
        c0, r0 = bx * T, by * T
        for tid in range(256):
            for k in range(4):
                i, j = (tid >> 4) + 16 * k, (tid & 15) * 4
                r, c = r0 + i, c0 + j
                if r < R and c < C:
                    assert c + 3 < C          # whole 16-byte vector inside the row
                    reads += [(b, r, c + q) for q in range(4)]
            for k in range(2):
                w = tid + 256 * k
                cc, chunk = w & 63, w >> 6
                c, rs = c0 + cc, r0 + chunk * 8
                if c < C and rs < Rp:
                    writes += [(b, c, rs + q) for q in range(8)]
    want = {(b, c, r) for b in range(batch) for c in range(C) for r in range(Rp)}
    assert len(writes) == len(set(writes)) and set(writes) == want
    assert {(b, r, c) for b, r, c in reads} == {(b, r, c) for b in range(batch) for r in range(R) for c in range(C)}


# ---- batched lift: descriptor chunks -----------------------------------------------

def batched_vec(L, plane, a16):
    vm = 4 if L <= 2 else (2 if L == 3 else 1)
    if vm >= 4 and plane % 4 == 0 and a16:
        return 4
    if vm >= 2 and plane % 2 == 0 and a16:
        return 2
    return 1


@pytest.mark.parametrize("plane,p,L", [(16 * 17, 32, 2), (40 * 41, 64, 3), (63 * 17, 128, 5), (1, 4, 1),
                                       (64 * 64, 32, 1)])
def test_batched_lift_chunks_cover_each_tensor_once(plane, p, L):
    vec = batched_vec(L, plane, True)
    cpg = cdiv(plane, 256 * vec)
    seen = []
    for local in range((p >> L) * cpg):
        g = local // cpg
        for t in range(256):
            e = ((local % cpg) * 256 + t) * vec
            if e < plane:
                assert e + vec <= plane
                seen += [(g, e + q) for q in range(vec)]
    want = {(g, e) for g in range(p >> L) for e in range(plane)}
    assert len(seen) == len(set(seen)) and set(seen) == want


# ---- FP8 passes: lift_amax_kernel (2-D grid) and lift_quant_rows_kernel (two operands) --

@pytest.mark.parametrize("p,L,plane_a,plane_b,vec,bx", [(16, 4, 64 * 80, 80 * 48, 2, 3), (8, 2, 33 * 17, 17 * 40, 1, 5),
                                                       (24, 3, 96 * 64, 64 * 72, 4, 2)])
def test_fp8_amax_grid_covers_both_operands_once(p, L, plane_a, plane_b, vec, bx):
    m = p >> L
    seen = []
    for by in range(2 * m):
        op, g = (0, by) if by < m else (1, by - m)
        nvec = (plane_a if op == 0 else plane_b) // vec
        for x in range(bx):
            for t in range(256):
                i = x * 256 + t
                while i < nvec:
                    seen.append((op, g, i))
                    i += bx * 256
    want = {(0, g, i) for g in range(m) for i in range(plane_a // vec)} | \
           {(1, g, i) for g in range(m) for i in range(plane_b // vec)}
    assert len(seen) == len(set(seen)) and set(seen) == want


@pytest.mark.parametrize("p,L,plane_a,plane_b,vec,blocks", [(16, 4, 64 * 80, 80 * 48, 2, 7), (8, 2, 33 * 17, 17 * 40, 1, 3)])
def test_fp8_quant_rows_two_operands_once(p, L, plane_a, plane_b, vec, blocks):
    m = p >> L
    items0 = m * (plane_a // vec)
    total = items0 + m * (plane_b // vec)
    seen = []
    for it in range(total):       # the grid-stride loop visits 0 .. total - 1 once
        first = it < items0
        item = it if first else it - items0
        nvec = (plane_a if first else plane_b) // vec
        seen.append((0 if first else 1, item // nvec, (item % nvec) * vec))
    want = {(0, g, e) for g in range(m) for e in range(0, plane_a, vec)} | \
           {(1, g, e) for g in range(m) for e in range(0, plane_b, vec)}
    assert len(seen) == len(set(seen)) and set(seen) == want
    # the grid-stride loop itself: every item index exactly once
    visits = [it for b in range(blocks) for t in range(256) for it in range(b * 256 + t, total, blocks * 256)]
    assert sorted(visits) == list(range(total))


@pytest.mark.parametrize("L", [4, 5])
@pytest.mark.parametrize("op", ["inverse", "adjoint"])
def test_split_mallat_inverse_maps(L, op):
    """The two-pass Mallat-input inverse / adjoint at L = 4, 5 (lift.cu,
    launch_split), restated on the CPU: the coarse pass applies the
    (L-2)-level transform to the first p/4 coefficient slices and writes
    s_2[k] to output slice 4k + 3; the fine pass reads s_2[k] there and d_2,
    d_1 from their Mallat positions and writes slices 4k .. 4k + 3.  Every
    slice index stays in bounds, every output slice is written once by the
    fine pass, and the result equals the one-pass transform."""
    import oracle as O
    p = 3 << L                                    # three tube groups
    y = np.random.default_rng(L).uniform(-1, 1, size=(p, 2, 3))
    one = O.ilift if op == "inverse" else O.lift_adjoint
    x = np.full_like(y, np.nan)
    # coarse pass
    s2 = one(y[: p // 4], L - 2)                  # natural order, p/4 slices
    for k in range(p // 4):
        assert 0 <= 4 * k + 3 < p
        x[4 * k + 3] = s2[k]
    # fine pass
    written = np.zeros(p, dtype=int)
    for k in range(p // 4):
        src = [4 * k + 3, p // 4 + k, p // 2 + 2 * k, p // 2 + 2 * k + 1]
        assert all(0 <= i < p for i in src)
        grp = np.stack([x[src[0]], y[src[1]], y[src[2]], y[src[3]]])
        out = one(grp, 2)
        for t in range(4):
            x[4 * k + t] = out[t]
            written[4 * k + t] += 1
    assert np.all(written == 1)
    np.testing.assert_allclose(x, one(y, L), rtol=0, atol=1e-14)



def _blocked_qr_r(X, B=16):
    """The steps of qr_r_kernel (qr.cu) in NumPy: panels of B columns,
    Householder reflections H = I - tau v v^T with v[c] = 1 and
    beta = -sign(alpha)|x|, the compact-WY T (T[c][c] = tau_c,
    T[0:c, c] = -tau_c T[0:c, 0:c] V^T v_c), the trailing update
    C -= V T^T V^T C; returns R^T as the kernel stores it."""
    m, n = X.shape
    W = X.astype(np.float64).copy()
    Rt = np.zeros((n, n))
    for k0 in range(0, n, B):
        kb = min(B, n - k0)
        V = W[k0:, k0:k0 + kb].copy()            # panel, rows relative to k0
        tau = np.zeros(kb)
        beta = np.zeros(kb)
        for c in range(kb):
            x = V[:, c]
            alpha, s2 = x[c], float(np.sum(x[c + 1:] ** 2))
            t, b = 0.0, alpha
            if s2 > 0:
                nrm = np.sqrt(alpha * alpha + s2)
                b = -nrm if alpha >= 0 else nrm
                t = (b - alpha) / b
                x[c + 1:] /= (alpha - b)
            tau[c], beta[c] = t, b
            x[c] = 1.0
            for j in range(c + 1, kb):
                w = float(x[c:] @ V[c:, j]) * t
                V[c:, j] -= w * x[c:]
        for c in range(kb):
            for j in range(c, kb):
                Rt[k0 + j, k0 + c] = beta[c] if c == j else V[c, j]
        for j in range(kb):
            V[:j, j] = 0.0
        T = np.zeros((kb, kb))
        T[0, 0] = tau[0]
        for c in range(1, kb):
            z = V[:, :c].T @ V[:, c]
            T[:c, c] = -tau[c] * (T[:c, :c] @ z)
            T[c, c] = tau[c]
        C = W[k0:, k0 + kb:]
        C -= V @ (T.T @ (V.T @ C))
        Rt[k0 + kb:, k0:k0 + kb] = C[:kb].T      # rows k0..k0+kb of R, trailing columns
    return Rt


@pytest.mark.parametrize("m,n", [(40, 33), (64, 64), (256, 48), (100, 17), (35, 35)])
def test_blocked_qr_restatement(m, n):
    X = np.random.default_rng(m + n).standard_normal((m, n))
    X[:, 5] = 0.0                                  # a zero column: no reflection (tau = 0)
    Rt = _blocked_qr_r(X)
    R = Rt.T
    assert np.allclose(np.tril(R, -1), 0.0)
    Rref = np.linalg.qr(X, mode="r")
    # R is unique up to the signs of its rows
    sgn = np.sign(np.diag(R)) * np.sign(np.diag(Rref))
    sgn[sgn == 0] = 1.0
    np.testing.assert_allclose(R * sgn[:, None], Rref, atol=1e-10 * np.abs(Rref).max())
    np.testing.assert_allclose(np.linalg.svd(R, compute_uv=False), np.linalg.svd(X, compute_uv=False), rtol=1e-10,
                               atol=1e-12)


def _panel4_qr_rt(X):
    """Restatement of qr_cols_kernel's arithmetic (fp64): 4-column panels,
    each factored column by column (H_c = I - tau v v^T, v[k] = 1, beta =
    -sign(alpha)|x|), T from the panel's Gram entries, the trailing columns
    updated with Y = V^T C, Y' = T^T Y, C -= V Y'; returns R^T as written."""
    PB, ROWS = 4, 256
    m, n = X.shape
    nbk = (n + PB - 1) // PB
    Xp = np.zeros((ROWS, nbk * PB))
    Xp[:m, :n] = X
    rows = np.arange(ROWS)
    for b in range(nbk):
        k0 = b * PB
        P = Xp[:, k0:k0 + PB]
        tau = np.zeros(PB)
        for c in range(PB):
            k = k0 + c
            alpha, s2 = P[k, c], np.sum(P[rows > k, c] ** 2)
            t, beta, scl = 0.0, alpha, 0.0
            if s2 > 0:
                nrm = np.sqrt(alpha * alpha + s2)
                beta = -nrm if alpha >= 0 else nrm
                t, scl = (beta - alpha) / beta, 1 / (alpha - beta)
            tau[c] = t
            P[rows > k, c] *= scl
            v = np.where(rows > k, P[:, c], np.where(rows == k, 1.0, 0.0))
            for c2 in range(c + 1, PB):
                P[:, c2] -= (v @ P[:, c2]) * t * v
            P[k, c] = beta
        V = np.stack([np.where(rows > k0 + c, P[:, c], np.where(rows == k0 + c, 1.0, 0.0)) for c in range(PB)], 1)
        G = V.T @ V
        T = np.zeros((PB, PB))
        for c in range(PB):
            T[c, c] = tau[c]
            for l in range(c):
                T[l, c] = -tau[c] * sum(T[l, q] * G[q, c] for q in range(l, c))
        for c in range(PB):
            P[rows > k0 + c, c] = 0.0
        C = Xp[:, k0 + PB:]
        Xp[:, k0 + PB:] = C - V @ (T.T @ (V.T @ C))
    return Xp[:n, :n].T.copy()


@pytest.mark.parametrize("m,n", [(256, 256), (256, 250), (200, 193), (256, 64), (37, 5)])
def test_panel4_qr_restatement(m, n):
    """The register-resident cluster QR's steps reproduce R of X = QR: upper
    triangular, |R| equal to LAPACK's, R^T R = X^T X."""
    X = np.random.default_rng(m + n).standard_normal((m, n))
    R = _panel4_qr_rt(X).T
    assert np.allclose(np.tril(R, -1), 0)
    np.testing.assert_allclose(np.abs(R), np.abs(np.linalg.qr(X, mode="r")), atol=1e-9)
    np.testing.assert_allclose(R.T @ R, X.T @ X, atol=1e-8)


# ---- tc_wprod_lift_kernel: converter-warp maps onto the MMA operand layouts ----------

def _lift_layout(L, nprod):
    G = 1 << L
    BN = 512 // G
    ncopy = 1 if nprod == 1 else 2
    a_tile, b_tile = 128 * 16 * 2, BN * 16 * 2
    stage = ncopy * G * (a_tile + b_tile)
    conv = 12 if L == 3 else 16
    a_units, b_units = 128 // 8, 8 * (BN // 64)
    return dict(G=G, BN=BN, a_tile=a_tile, b_tile=b_tile, b_off=ncopy * G * a_tile, stage=stage,
                stages=min(8, 196608 // stage), conv=conv, a_units=a_units, units=a_units + b_units,
                upw=cdiv(a_units + b_units, conv))


def _lift_stage_writes(L, M, N, K, m0, n0, k0, nprod=3):
    """Every 8-byte shared-memory store of one K step of one CTA, restated from
    the kernel: (warp, lane, slice t, copy, byte offset in the stage,
    global element coordinates of the 4 values or None for zero fill)."""
    lay = _lift_layout(L, nprod)
    G, BN = lay["G"], lay["BN"]
    out = []
    for cw in range(lay["conv"]):
        for i in range(lay["upw"]):
            u = cw + i * lay["conv"]
            if u >= lay["units"]:
                break
            for lane in range(32):
                if u < lay["a_units"]:
                    ar, aq = (lane & 15) >> 1, ((lane >> 4) << 1) | (lane & 1)
                    row, kc = m0 + 8 * u + ar, k0 + 4 * aq
                    src = ("A", row, kc) if (row < M and kc < K) else None
                    off = u * 256 + (lane >> 4) * 128 + ar * 16 + (lane & 1) * 8
                    base, tile = 0, lay["a_tile"]
                    elem = ("A", 8 * u + ar, 4 * aq)          # (row, k) within the tile
                else:
                    ub = u - lay["a_units"]
                    j, cb = ub % 8, ub // 8
                    bh, bc = lane >> 4, lane & 15
                    krow, col = k0 + 2 * j + bh, n0 + 64 * cb + 4 * bc
                    src = ("B", krow, col) if (krow < K and col < N) else None
                    kr = 2 * j + bh
                    off = cb * 2048 + kr * 128 + (((bc >> 1) ^ (kr & 7)) << 4) + (bc & 1) * 8
                    base, tile = lay["b_off"], lay["b_tile"]
                    elem = ("B", kr, 64 * cb + 4 * bc)        # (k, column) within the tile
                for t in range(G):
                    for copy in range(1 if nprod == 1 else 2):
                        out.append((cw, lane, t, copy, base + (copy * G + t) * tile + off, src, elem))
    return lay, out


def _a_canonical(r, k):
    """K-major, no swizzle: 8-row x 16-byte core matrices, K neighbours 128 B
    apart (leading byte offset), 8-row groups 256 B apart (stride byte offset)."""
    return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2


def _b_canonical(k, n):
    """MN-major, 128-byte swizzle, 16 K rows per 64-column block (blocks 2 KB
    apart): row k of block n // 64 at 128 k, 16-byte chunk (n % 64) / 8 XOR k % 8."""
    return (n // 64) * 2048 + k * 128 + ((((n % 64) >> 3) ^ (k & 7)) << 4) + (n & 7) * 2


@pytest.mark.parametrize("L", [1, 2, 3])
def test_lift_kernel_stage_layout(L):
    """One K step: every (row, k) of the 2G A tiles and every (k, column) of the
    2G B tiles is written exactly once, at the address the MMA descriptors read
    (the canonical layouts above), inside the stage; the stage ring, the
    epilogue staging and the barriers fit the shared memory."""
    lay, writes = _lift_stage_writes(L, 4096, 4096, 4096, 0, 0, 0)
    G, BN = lay["G"], lay["BN"]
    seen = {}
    for cw, lane, t, copy, addr, src, elem in writes:
        assert 0 <= addr and addr + 8 <= lay["stage"]
        kind, a, b = elem
        for v in range(4):
            if kind == "A":
                exp = (copy * G + t) * lay["a_tile"] + _a_canonical(a, b + v)
            else:
                exp = lay["b_off"] + (copy * G + t) * lay["b_tile"] + _b_canonical(a, b + v)
            assert addr + 2 * v == exp
            assert exp not in seen
            seen[exp] = (kind, t, copy, a, b + v)
    # all bytes of the stage written once (2 bytes per value)
    assert len(seen) * 2 == lay["stage"]
    # tile bases: 1024-byte aligned for the swizzled B tiles
    assert lay["b_off"] % 1024 == 0 and lay["b_tile"] % 1024 == 0 and lay["stage"] % 1024 == 0
    spp = G
    while spp > 0 and spp * 128 * BN * 4 > lay["stages"] * lay["stage"]:
        spp >>= 1
    assert spp >= 1
    smem = lay["stages"] * lay["stage"] + (2 * lay["stages"] + 1) * 8 + 16 + 1024
    assert smem <= 232448


@pytest.mark.parametrize("L", [1, 2, 3])
def test_lift_kernel_stage_stores_conflict_free(L):
    """The 8-byte stores of each half-warp fill 128 distinct bytes of one
    128-byte line set (no bank conflicts)."""
    lay, writes = _lift_stage_writes(L, 4096, 4096, 4096, 0, 0, 0)
    # one store instruction per (warp, unit, slice, copy); a half-warp's 16
    # lanes are served together and their 8-byte stores must touch 32
    # distinct banks
    per = {}
    for cw, lane, t, copy, addr, src, elem in writes:
        unit = (elem[0], elem[1] // 8) if elem[0] == "A" else (elem[0], elem[1] // 2, elem[2] // 64)
        key = (cw, unit, t, copy, lane >> 4)
        per.setdefault(key, []).extend([(addr // 4) % 32, (addr // 4 + 1) % 32])
    for key, banks in per.items():
        assert len(banks) == 32 and len(set(banks)) == 32, key


@pytest.mark.parametrize("M,N,K", [(200, 260, 100), (1, 4, 4), (130, 516, 36), (256, 256, 256)])
@pytest.mark.parametrize("L", [1, 3])
def test_lift_kernel_loads_in_bounds(L, M, N, K):
    """Every load of every K step of every tile stays inside the operand
    (K % 4 == 0, N % 4 == 0; rows, columns and K beyond the edges read as
    zero), and together the loads cover each element of A and B."""
    lay = _lift_layout(L, 3)
    BN = lay["BN"]
    seen_a, seen_b = set(), set()
    for n0 in range(0, N, BN):
        for m0 in range(0, M, 128):
            for k0 in range(0, K, 16):
                _, writes = _lift_stage_writes(L, M, N, K, m0, n0, k0)
                for cw, lane, t, copy, addr, src, elem in writes:
                    if src is None or t or copy:
                        continue
                    kind, a, b = src
                    if kind == "A":
                        assert 0 <= a < M and 0 <= b and b + 4 <= K
                        seen_a.update((a, b + v) for v in range(4))
                    else:
                        assert 0 <= a < K and 0 <= b and b + 4 <= N
                        seen_b.update((a, b + v) for v in range(4))
    assert len(seen_a) == M * K and len(seen_b) == K * N


@pytest.mark.parametrize("L", [1, 2, 3])
def test_lift_kernel_epilogue_covers_tile_once(L):
    """Epilogue of tc_wprod_lift_kernel: the converter warps (TMEM lane
    quarter = warp & 3, column group = converter index // 4) cover every
    (row, column) of the 128 x BN tile exactly once per store pass, and the
    staged float4s of a pass (SPP slices, 32-column blocks of 128-byte rows,
    128-byte swizzle) land at distinct addresses inside the pipeline buffers."""
    lay = _lift_layout(L, 3)
    G, BN = lay["G"], lay["BN"]
    CH = min(64 // G, 16)
    conv, first = lay["conv"], 1
    ngrp = conv // 4
    spp = G
    while spp > 0 and spp * 128 * BN * 4 > lay["stages"] * lay["stage"]:
        spp >>= 1
    seen, addrs = set(), set()
    for cw in range(conv):
        warp = cw + first
        quad, grp = warp & 3, cw // 4
        for lane in range(32):
            r = quad * 32 + lane
            for c0 in range(grp * CH, BN, ngrp * CH):
                h, q0 = c0 // 32, (c0 % 32) // 4
                for j in range(0, CH, 4):
                    for tt in range(spp):
                        a = (h * spp + tt) * 16384 + r * 128 + (((q0 + j // 4) ^ (r & 7)) << 4)
                        assert 0 <= a and a + 16 <= lay["stages"] * lay["stage"]
                        assert a not in addrs
                        addrs.add(a)
                    for jj in range(4):
                        key = (r, c0 + j + jj)
                        assert key not in seen
                        seen.add(key)
    assert len(seen) == 128 * BN
