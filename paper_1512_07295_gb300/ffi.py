"""ctypes binding of libpk.so (include/pk.h): loads the in-tree library and declares every entry
point with the same names. Argument marshalling only; all computation happens in the CUDA library.
Loading fails loudly when the library has not been built (there is no fallback path)."""

import ctypes
import os
import re

from . import build as _build

c_int32, c_int64, c_double, c_size_t, c_void_p, c_char_p = (ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                                             ctypes.c_size_t, ctypes.c_void_p, ctypes.c_char_p)

PK_OK, PK_EINVAL, PK_ESIZE, PK_ECUDA, PK_ECUFFT, PK_ETIMEOUT, PK_EDEVICE = range(7)
PK_FP64, PK_FP32, PK_FIXED64 = 0, 1, 2
PK_POS_F64_XYZ, PK_POS_CELL_F32OFF = 0, 1
(PK_WS_ASSIGN, PK_WS_FFT_ESTIMATE, PK_WS_POWER, PK_WS_POWER_BINNED, PK_WS_BIN, PK_WS_BACKWARD, PK_WS_BISPECTRUM,
 PK_WS_BISPECTRUM_COUNTS, PK_WS_POWER_HOST, PK_WS_DIRECT, PK_WS_CROSS, PK_WS_ALIASING) = range(12)
PK_DERR_NONFINITE, PK_DERR_CELLRANGE, PK_DERR_TIMEOUT = 1, 2, 4


class PkConfig(ctypes.Structure):
    _fields_ = [
        ("ng", c_int32),
        ("order", c_int32),
        ("interlace", c_int32),
        ("prec", c_int32),
        ("box", c_double),
        ("bin_lo2", c_int32),
        ("bin_w2", c_int32),
        ("nbins", c_int32),
        ("subtract_shot", c_int32),
        ("tile_run", c_int32),
    ]


_CFG = ctypes.POINTER(PkConfig)

# name -> (restype, argtypes)
SIGNATURES = {
    "pk_default_config": (None, [_CFG, c_int32, c_double]),
    "pk_workspace_size": (c_size_t, [_CFG, c_int64, c_int32]),
    "pk_batch_workspace_size": (c_size_t, [_CFG, c_int32, c_int64]),
    "pk_tiles_per_axis": (c_int32, [_CFG, ctypes.POINTER(c_int32)]),
    "pk_prepare": (c_int32, [_CFG, c_void_p, c_int64, c_void_p, c_void_p]),
    "pk_bin": (c_int32, [_CFG, c_void_p, c_int32, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                         c_void_p]),
    "pk_assign": (c_int32, [_CFG, c_void_p, c_int32, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "pk_fft_estimate": (c_int32, [_CFG, c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_size_t, c_void_p]),
    "pk_power": (c_int32, [_CFG, c_void_p, c_int32, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                           c_size_t, c_void_p]),
    "pk_power_host": (c_int32, [_CFG, c_void_p, c_int32, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                c_void_p]),
    "pk_power_binned": (c_int32, [_CFG, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_size_t, c_void_p]),
    "pk_bispectrum_ntri": (c_int32, [c_int32]),
    "pk_bispectrum_triangles": (c_int32, [c_int32, c_void_p]),
    "pk_bispectrum_counts": (c_int32, [_CFG, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
    "pk_bispectrum": (c_int32, [_CFG, c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "pk_power_backward": (c_int32, [_CFG, c_void_p, c_int32, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_size_t,
                                    c_void_p]),
    "pk_batch_power": (c_int32, [_CFG, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_size_t,
                                 c_void_p]),
    "pk_direct_modes": (c_int32, [_CFG, c_void_p, c_int32, c_void_p, c_int64, c_void_p, c_void_p, c_size_t, c_void_p]),
    "pk_cross_power": (c_int32, [_CFG, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "pk_multigrid_workspace_size": (c_size_t, [_CFG, c_int32, c_int64]),
    "pk_power_multigrid": (c_int32, [_CFG, c_int32, c_void_p, c_int32, c_void_p, c_int64, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_size_t, c_void_p]),
    "pk_aliasing_residual": (c_int32, [_CFG, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "pk_estimate_noalloc": (c_int32, [_CFG, c_void_p, c_void_p, c_double, c_double, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pk_profile_enable": (c_int32, [c_int32]),
    "pk_profile_read": (c_int32, [c_void_p, c_int32]),
    "pk_profile_launches": (c_int64, []),
    "pk_last_error": (c_char_p, []),
    "pk_device_error": (c_int32, [c_void_p]),
}

_LIB = None


def header_functions(path=None):
    """Names of the functions declared in include/pk.h."""
    path = path or os.path.join(_build.ROOT, "include", "pk.h")
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pk_[a-z_0-9]+)\s*\(", text)))


def lib():
    """The loaded libpk.so with every signature declared. Raises if the library is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libpk.so is not built ({path}); run `python -c 'import __graft_entry__ as g; g.build()'`")
    handle = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(handle, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = handle
    return _LIB


def last_error():
    msg = lib().pk_last_error()
    return msg.decode() if msg else ""


class PkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"pk status {status}: {msg}")
        self.status = status


def check(status):
    if status != PK_OK:
        raise PkError(status, last_error())
