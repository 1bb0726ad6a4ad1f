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
