"""The C ABI library loads and exports every function include/pk.h declares (no GPU needed)."""

import ctypes
import os

import pytest

from paper_1512_07295_gb300 import build, ffi


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(build.lib_path()):
        build.build()
    return ffi.lib()


def test_header_declares_the_boundary():
    names = ffi.header_functions()
    for required in ("pk_assign", "pk_fft_estimate", "pk_power", "pk_bispectrum", "pk_power_backward"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in ffi.header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    assert set(ffi.header_functions()) == set(ffi.SIGNATURES)


def test_config_struct_layout():
    assert ctypes.sizeof(ffi.PkConfig) == 48
    assert ffi.PkConfig.box.offset == 16


def test_host_only_calls(lib):
    cfg = ffi.PkConfig()
    lib.pk_default_config(ctypes.byref(cfg), 64, 1000.0)
    assert (cfg.ng, cfg.order, cfg.interlace, cfg.prec, cfg.nbins, cfg.bin_lo2, cfg.bin_w2) == (64, 4, 1, ffi.PK_FP32, 32, 1, 2)
    tc = ctypes.c_int32(0)
    assert lib.pk_tiles_per_axis(ctypes.byref(cfg), ctypes.byref(tc)) == 8 and tc.value == 8
    assert lib.pk_bispectrum_ntri(16) == 508
    assert lib.pk_bispectrum_ntri(0) == 0


def test_bispectrum_triangle_list(lib):
    # Shells of width w hold w s <= |k| < w (s + 1) (shell_lo = 0). Three wave vectors with those
    # lengths can close (k1 + k2 + k3 = 0) iff the longest can be at most the sum of the other two: the
    # smallest k1 (w s1) below the largest k2 + k3 (w (s2 + s3 + 2), an open bound). The list must be
    # every such ordered triple s1 >= s2 >= s3 once, s1 slowest, with 508 triangles for the 16 shells
    # of the bispectrum configuration.
    for nshells in (1, 2, 5, 16):
        n = lib.pk_bispectrum_ntri(nshells)
        tri = (ctypes.c_int32 * (3 * n))()
        assert lib.pk_bispectrum_triangles(nshells, tri) == n
        got = [tuple(tri[3 * i:3 * i + 3]) for i in range(n)]
        closable = []
        for s1 in range(nshells):
            for s2 in range(s1 + 1):
                for s3 in range(s2 + 1):
                    if s1 < s2 + s3 + 2:  # min |k1| < max(|k2| + |k3|), in units of w
                        closable.append((s1, s2, s3))
        assert got == closable
    assert lib.pk_bispectrum_ntri(16) == 508
    assert lib.pk_bispectrum_triangles(0, (ctypes.c_int32 * 3)()) == 0
    assert lib.pk_bispectrum_triangles(16, None) == 0


def test_invalid_config_is_rejected_before_any_launch(lib):
    cfg = ffi.PkConfig()
    lib.pk_default_config(ctypes.byref(cfg), 63, 1000.0)  # odd grid
    st = lib.pk_prepare(ctypes.byref(cfg), None, 0, None, None)
    assert st == ffi.PK_EINVAL
    assert "ng" in ffi.last_error()
    lib.pk_default_config(ctypes.byref(cfg), 64, -1.0)
    assert lib.pk_prepare(ctypes.byref(cfg), None, 0, None, None) == ffi.PK_EINVAL
    lib.pk_default_config(ctypes.byref(cfg), 64, 1000.0)
    cfg.order = 5
    assert lib.pk_power(ctypes.byref(cfg), None, 0, None, 10, None, None, None, None, None, 0, None) == ffi.PK_EINVAL
