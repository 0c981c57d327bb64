"""GPU parity of the batched launch (w-product + rank-r w-svd over many
uneven items) against the FP64 oracle, item by item; the run captured in a
CUDA graph; the autotuned plan; and the 4096-item batch (sampled items)."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_08228_gb300 import capi, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2601_08228_gb300 import build
    build.build()
    capi.lib()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def _device_items(items, r):
    out = []
    for it in items:
        A = torch.from_numpy(it["A"]).cuda()
        B = torch.from_numpy(it["B"]).cuda()
        out.append(dict(A=A, B=B, C=torch.empty((it["p"], it["n1"], it["n4"]), device="cuda"),
                        C_r=torch.empty_like(A), L=it["L"], r=r))
    return out


def _rec_tol(A, L, r):
    s = np.linalg.svd(O.lift(A, L), compute_uv=False)
    if r >= s.shape[1]:
        return 1e-4
    ratio = float(np.max(s[:, 0] / np.maximum(s[:, r - 1] - s[:, r], 1e-30)))
    return max(1e-4, 4 * np.sqrt(max(A.shape[1:])) * 1.2e-7 * ratio)


def _check_items(host_items, dev_items, idx, r):
    for i in idx:
        h, d = host_items[i], dev_items[i]
        assert O.rel_fro(host(d["C"]), O.wprod(h["A"], h["B"], h["L"])) <= 1e-5
        assert O.rel_fro(host(d["C_r"]), O.wsvd(h["A"], h["L"], r)) <= _rec_tol(h["A"], h["L"], r)


def test_batched_small_every_item():
    items = synth.batch_items(count=48, seed=1)
    dev = _device_items(items, 8)
    bl = capi.BatchedLaunch(dev)
    bl.run()
    _check_items(items, dev, range(len(items)), 8)
    assert capi.wp_get_device_error() == 0


@pytest.mark.parametrize("group,threads", [(1, 128), (0, 128), (0, 256)])
def test_batched_both_jacobi_kernels(group, threads):
    """The Jacobi phase on the lane-group kernel (the default plan) and on
    the block-cyclic kernel with either CTA size for the widest class:
    every item of a mixed batch against the oracle."""
    items = synth.batch_items(count=40, seed=9)
    dev = _device_items(items, 6)
    bl = capi.BatchedLaunch(dev)
    assert bl.plan.svd_group == 1
    bl.plan.svd_group = group
    bl.plan.svd_threads = threads
    bl.run()
    _check_items(items, dev, range(len(items)), 6)
    assert capi.wp_get_device_error() == 0


def test_batched_rank_above_min_dims_rejected():
    items = synth.batch_items(count=4, seed=5)
    dev = _device_items(items, 8)
    dev[2]["r"] = min(items[2]["n1"], items[2]["n2"]) + 1
    with pytest.raises(capi.WPError) as e:
        capi.BatchedLaunch(dev)
    assert e.value.status == 4


def test_batched_cuda_graph_and_autotune():
    items = synth.batch_items(count=64, seed=2)
    dev = _device_items(items, 8)
    bl = capi.BatchedLaunch(dev, tune=True)
    assert bl.plan.gemm_threads in (64, 128, 256, 512) and bl.plan.svd_threads in (64, 128, 256)
    bl.run()
    torch.cuda.synchronize()
    ref = [(host(d["C"]), host(d["C_r"])) for d in dev]
    for d in dev:
        d["C"].zero_()
        d["C_r"].zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            bl.run()
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for (c, cr), d in zip(ref, dev):
        np.testing.assert_array_equal(host(d["C"]), c)
        np.testing.assert_array_equal(host(d["C_r"]), cr)
    _check_items(items, dev, range(0, 64, 7), 8)


def test_batched_4096_items_sampled():
    """The 4096-item batch (n1, n2, n4 ~ U{16..64}, p ~ U{32,64,128},
    L ~ U{1..log2 p - 2}, seed 1), rank 8; 24 sampled items against the oracle."""
    items = synth.batch_items(count=4096, seed=1)
    dev = _device_items(items, 8)
    bl = capi.BatchedLaunch(dev)
    bl.run()
    torch.cuda.synchronize()
    idx = np.random.default_rng(0).choice(4096, 24, replace=False)
    _check_items(items, dev, idx, 8)
    assert capi.wp_get_device_error() == 0


def test_batched_small_and_degenerate_items():
    """Items narrower than one 8-column block pair (n1, n2 in 1..20, padded
    with zero columns in the Jacobi phase), L = 0..2, ranks up to min(n1, n2),
    every item against the oracle."""
    rng = np.random.default_rng(7)
    items = []
    for _ in range(40):
        n1, n2, n4 = (int(x) for x in rng.integers(1, 21, size=3))
        L = int(rng.integers(0, 3))
        p = (1 << L) * int(rng.integers(1, 4))
        items.append(dict(n1=n1, n2=n2, n4=n4, p=p, L=L,
                          A=rng.uniform(-1, 1, (p, n1, n2)).astype(np.float32),
                          B=rng.uniform(-1, 1, (p, n2, n4)).astype(np.float32)))
    dev = _device_items(items, 1)
    for d, it in zip(dev, items):
        d["r"] = int(rng.integers(1, min(it["n1"], it["n2"]) + 1))
    bl = capi.BatchedLaunch(dev)
    bl.run()
    for h, d in zip(items, dev):
        assert O.rel_fro(host(d["C"]), O.wprod(h["A"], h["B"], h["L"])) <= 1e-5
        assert O.rel_fro(host(d["C_r"]), O.wsvd(h["A"], h["L"], d["r"])) <= _rec_tol(h["A"], h["L"], d["r"])
    assert capi.wp_get_device_error() == 0
