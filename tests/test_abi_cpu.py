"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/wprod.h declares, and rejects bad arguments on the
host before touching the device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libwprod():
    from paper_2601_08228_gb300 import build
    build.build()
    from paper_2601_08228_gb300 import capi
    return capi.lib()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "wprod.h")).read()
    return sorted(set(re.findall(r"WP_API\s+(?:const\s+char\s*\*|int|uint64_t)\s+(wp_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(libwprod):
    names = _declared_symbols()
    assert len(names) >= 28
    for n in names:
        assert hasattr(libwprod, n), n


def test_status_strings_and_version(libwprod):
    assert libwprod.wp_status_string(0) == b"WP_OK"
    for code in range(1, 13):
        assert libwprod.wp_status_string(code).startswith(b"WP_ERR_")
    assert libwprod.wp_version() >= 100


def test_host_validation_needs_no_gpu(libwprod):
    L = libwprod
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: validation fails first
    assert L.wp_lift_forward(None, fake, 4, 4, 8, 3, None) == 1          # NULL
    assert L.wp_lift_forward(fake, ctypes.c_void_p(2 << 20), 4, 4, 12, 3, None) == 3  # p % 2^L
    assert L.wp_lift_forward(fake, ctypes.c_void_p(2 << 20), 4, 4, 8, -1, None) == 3
    assert L.wp_lift_forward(fake, ctypes.c_void_p(2 << 20), 0, 4, 8, 3, None) == 2   # shape
    assert L.wp_lift_forward(fake, ctypes.c_void_p((2 << 20) + 4), 4, 4, 8, 3, None) == 6  # align
    assert L.wp_lift_forward(fake, fake, 4, 4, 8, 3, None) == 11         # alias
    n = ctypes.c_size_t(0)
    assert L.wp_wprod_workspace(4, 4, 4, 8, 3, 9, ctypes.byref(n)) == 5  # prec
    assert L.wp_wprod_workspace(4, 4, 4, 8, 3, 0, ctypes.byref(n)) == 0 and n.value > 0
    assert L.wp_wprod(fake, ctypes.c_void_p(2 << 20), ctypes.c_void_p(3 << 20), 4, 4, 4, 8, 3, 0, 0, 0,
                      ctypes.c_void_p(4 << 20), 16, None) == 7           # workspace too small
    # two-sided pseudo-inverse deblurring
    assert L.wp_deblur_pinv_workspace(4, 4, 12, 3, 0, ctypes.byref(n)) == 3      # p % 2^L
    assert L.wp_deblur_pinv_workspace(4, 4, 8, 3, 0, ctypes.byref(n)) == 0 and n.value > 0
    f2, f3, f4 = ctypes.c_void_p(2 << 20), ctypes.c_void_p(3 << 20), ctypes.c_void_p(4 << 20)
    assert L.wp_deblur_pinv(None, f2, f3, f4, 4, 4, 8, 3, -1.0, 2, 0, fake, 1 << 30, None) == 1   # NULL
    assert L.wp_deblur_pinv(fake, f2, f3, f3, 4, 4, 8, 3, -1.0, 2, 0, fake, 1 << 30, None) == 11  # X aliases B
    assert L.wp_deblur_pinv(fake, f2, f3, f4, 4, 4, 8, 3, -1.0, 2, 0, fake, 16, None) == 7        # workspace
    # host-buffer w-product: chunks of whole tube groups, validated before any copy
    assert L.wp_wprod_host_workspace(4, 4, 4, 16, 3, 0, 12, ctypes.byref(n)) == 2   # 12 % 2^3 != 0
    assert L.wp_wprod_host_workspace(4, 4, 4, 12, 3, 0, 0, ctypes.byref(n)) == 3    # p % 2^L
    assert L.wp_wprod_host_workspace(4, 4, 4, 16, 3, 0, 8, ctypes.byref(n)) == 0
    two_chunks = n.value
    assert L.wp_wprod_host_workspace(4, 4, 4, 16, 3, 0, 16, ctypes.byref(n)) == 0 and n.value > two_chunks
    assert L.wp_wprod_host(None, fake, fake, 4, 4, 4, 16, 3, 0, 8, fake, 1 << 20, None) == 1
    assert L.wp_wprod_host(fake, ctypes.c_void_p(2 << 20), ctypes.c_void_p(3 << 20), 4, 4, 4, 16, 3, 0, 8,
                           ctypes.c_void_p(4 << 20), 16, None) == 7           # workspace too small


def test_limits_validated_on_the_host(libwprod):
    L = libwprod
    assert L.wp_set_jacobi_max_sweeps(0) == 2              # WP_ERR_SHAPE, limit unchanged
    assert L.wp_set_jacobi_max_sweeps(1001) == 2
    assert L.wp_set_jacobi_max_sweeps(40) == 0             # the default
    assert L.wp_set_jacobi_precondition(2) == 2            # on / off only
    assert L.wp_set_jacobi_precondition(1) == 0            # the default
    assert L.wp_set_jacobi_column_split(-1) == 2           # on / off only
    assert L.wp_set_jacobi_column_split(1) == 0            # the default
    assert L.wp_set_jacobi_cluster_size(1) == 2            # 0, 2, 3 or 4
    assert L.wp_set_jacobi_cluster_size(5) == 2
    assert L.wp_set_jacobi_cluster_size(0) == 0            # the default
    assert L.wp_jacobi_cluster_capacity(2, None) == 1      # WP_ERR_NULL
    assert L.wp_selftest_bounded_wait(2, 1000000, None) == 2      # unknown wait kind
    assert L.wp_selftest_bounded_wait(0, 999, None) == 2          # limit below 1 us
    assert L.wp_selftest_bounded_wait(1, 100000001, None) == 2    # limit above 0.1 s


def test_plan_cache_round_trip(libwprod, tmp_path):
    """The w-product plan cache (host only): set / get / remove, validation,
    and the JSON-lines file written by wp_plan_save read back by wp_plan_load."""
    from paper_2601_08228_gb300 import capi
    capi.wp_plan_clear()
    capi.wp_plan_set(256, 256, 256, 192, 3, "bf16x3", "persistent")
    capi.wp_plan_set(64, 32, 48, 16, 2, "bf16", "fused")
    assert capi.wp_plan_get(256, 256, 256, 192, 3, "bf16x3") == 2
    assert capi.wp_plan_get(256, 256, 256, 192, 3, "bf16") == 0          # another key
    with pytest.raises(capi.WPError) as e:
        capi.wp_plan_set(256, 256, 256, 192, 3, "bf16x3", 4)               # no such variant
    assert e.value.status == capi.WP_ERR_SHAPE
    with pytest.raises(capi.WPError) as e:
        capi.wp_plan_set(256, 256, 256, 12, 3, "bf16x3", 1)               # p % 2^L
    assert e.value.status == capi.WP_ERR_LEVELS
    path = tmp_path / "plans.jsonl"
    capi.wp_plan_save(str(path))
    lines = path.read_text().splitlines()
    assert len(lines) == 2 and all('"op": "wprod"' in x and '"variant"' in x for x in lines)
    capi.wp_plan_clear()
    assert capi.wp_plan_get(64, 32, 48, 16, 2, "bf16") == 0
    assert capi.wp_plan_load(str(path)) == 2
    assert capi.wp_plan_get(64, 32, 48, 16, 2, "bf16") == 1
    assert capi.wp_plan_get(256, 256, 256, 192, 3, "bf16x3") == 2
    capi.wp_plan_set(64, 32, 48, 16, 2, "bf16", 0)                        # removes the entry
    assert capi.wp_plan_get(64, 32, 48, 16, 2, "bf16") == 0
    bad = tmp_path / "bad.jsonl"
    bad.write_text('{"op": "wprod", "n1": 4, "n2": 4, "n4": 4, "p": 8, "L": 3, "prec": 2, "variant": 7, "ms": 1}\n')
    with pytest.raises(capi.WPError):
        capi.wp_plan_load(str(bad))
    with pytest.raises(capi.WPError):
        capi.wp_plan_load(str(tmp_path / "missing.jsonl"))
    capi.wp_plan_clear()
