"""pk_estimate_noalloc: the estimate stage for callers that cannot allocate device memory (a
framework that owns all device memory, a fixed memory budget, a host callback that must not enter
the allocator). Its scratch is a fixed device array inside the library. Through the C ABI, two calls
in a row (the second starting from the first one's scratch contents) must give the FP64 oracle's
P(k), k_eff and exact mode counts, for FP32, FP64 and the deterministic FIXED64 mode, with and
without interlacing, and with weights and shot-noise subtraction; sizes beyond the array are refused.
The file is named to be collected last."""

import ctypes

import numpy as np
import pytest
import torch

import _ref
from paper_1512_07295_gb300 import api, catalogs, ffi

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _noalloc(cfg, g1h, g2h, wsum, w2sum):
    lib = ffi.lib()
    pk = torch.empty(cfg.nb, dtype=torch.float64, device=DEV)
    km = torch.empty(cfg.nb, dtype=torch.float64, device=DEV)
    nm = torch.empty(cfg.nb, dtype=torch.int64, device=DEV)
    st = lib.pk_estimate_noalloc(ctypes.byref(cfg.c()), ctypes.c_void_p(g1h.data_ptr()),
                                 ctypes.c_void_p(g2h.data_ptr() if g2h is not None else 0), float(wsum), float(w2sum),
                                 ctypes.c_void_p(pk.data_ptr()), ctypes.c_void_p(km.data_ptr()),
                                 ctypes.c_void_p(nm.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, pk, km, nm


def _rfft(g, prec):
    """The forward DFT of a mass grid on the half-complex layout, computed on the host (test side)."""
    ctype = np.complex64 if prec == "fp32" else np.complex128
    return torch.from_numpy(np.ascontiguousarray(np.fft.rfftn(g.cpu().numpy()).astype(ctype))).to(DEV)


@pytest.mark.parametrize("prec", ["fp32", "fp64", "fixed64"])
@pytest.mark.parametrize("interlace", [True, False])
@pytest.mark.parametrize("weighted", [False, True])
def test_noalloc_estimate_matches_the_oracle_twice(prec, interlace, weighted):
    box, ng = 300.0, 32
    pos_np = catalogs.zeldovich(32, box, rms=6.0, seed=91)
    w_np = catalogs.random_weights(len(pos_np), seed=92).astype(np.float32) if weighted else None
    pos = torch.from_numpy(pos_np).to(DEV)
    w = torch.from_numpy(w_np).to(DEV) if weighted else None
    cfg = api.Config(ng=ng, box=box, prec=prec, interlace=interlace, subtract_shot=weighted)
    g1, g2 = api.assign(pos, cfg, weights=w)
    g1h = _rfft(g1, prec)
    g2h = _rfft(g2, prec) if interlace else None
    wd = None if w_np is None else w_np.astype(np.float64)
    wsum = float(len(pos_np)) if wd is None else float(wd.sum())
    w2sum = float(len(pos_np)) if wd is None else float((wd * wd).sum())
    ref_pk, ref_km, ref_cnt, _ = _ref.power(pos_np, box, ng, 4, interlace, weights=wd, subtract=weighted)
    # FP64: the oracle-parity bar; FP32, and FIXED64 (deterministic, its contributions computed in FP32
    # before the exact 64-bit sums): the FP32 bar
    tol = 1e-10 if prec == "fp64" else 1e-5
    for _ in range(2):  # the second call starts from the first call's scratch contents
        st, pk, km, nm = _noalloc(cfg, g1h, g2h, wsum, w2sum)
        assert st == ffi.PK_OK, ffi.last_error()
        torch.cuda.synchronize()
        assert np.array_equal(nm.cpu().numpy(), ref_cnt)
        # shot noise subtracted: compare against the level of the unsubtracted power
        scale = np.abs(ref_pk) + (_ref.oracle.power.shot_noise(box, wd, len(pos_np)) if weighted else 0.0)
        assert np.max(np.abs(pk.cpu().numpy() - ref_pk) / scale) <= tol
        assert np.max(np.abs(km.cpu().numpy() / ref_km - 1.0)) <= (1e-12 if prec == "fp64" else 1e-6)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    cfg = api.Config(ng=32, box=100.0, nbins=1500, bin_w2=1)
    g = torch.zeros((32, 32, 17), dtype=torch.complex64, device=DEV)
    st, _, _, _ = _noalloc(cfg, g, g, 1.0, 1.0)
    assert st == ffi.PK_ESIZE
    assert "1024" in ffi.last_error()
    big = api.Config(ng=2048, box=100.0)  # beyond any grid the library takes: rejected before the scratch
    st, _, _, _ = _noalloc(big, g, g, 1.0, 1.0)
    assert st == ffi.PK_EINVAL
