"""pk_estimate_noalloc: the estimate stage for callers that cannot allocate device memory (a
framework that owns all device memory, a fixed memory budget, a host callback that must not enter
the allocator). Its scratch is a fixed device array inside the library; this checks, through the C
ABI, that two calls in a row reproduce the workspace-based pk_power on the same catalogue, and that
sizes beyond the array's limit are refused. The file is named to be collected last."""

import ctypes

import numpy as np
import pytest
import torch

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


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_estimate_matches_power_twice(prec):
    box, ng = 300.0, 32
    pos = torch.from_numpy(catalogs.zeldovich(32, box, rms=6.0, seed=91)).to(DEV)
    n = pos.shape[0]
    cfg = api.Config(ng=ng, box=box, prec=prec)
    ref_pk, ref_km, ref_nm = api.power(pos, cfg)
    g1, g2 = api.assign(pos, cfg)
    # the forward DFT of each mass grid on the half-complex layout (computed on the host)
    ctype = np.complex64 if prec == "fp32" else np.complex128
    g1h = torch.from_numpy(np.ascontiguousarray(np.fft.rfftn(g1.cpu().numpy()).astype(ctype))).to(DEV)
    g2h = torch.from_numpy(np.ascontiguousarray(np.fft.rfftn(g2.cpu().numpy()).astype(ctype))).to(DEV)
    tol = 1e-5 if prec == "fp32" else 1e-10
    for _ in range(2):  # the second call starts from the first call's scratch contents
        st, pk, km, nm = _noalloc(cfg, g1h, g2h, float(n), float(n))
        assert st == ffi.PK_OK, ffi.last_error()
        torch.cuda.synchronize()
        assert torch.equal(nm, ref_nm)
        r = ref_pk.cpu().numpy()
        assert np.max(np.abs(pk.cpu().numpy() / r - 1.0)) <= tol
        assert np.max(np.abs(km.cpu().numpy() / ref_km.cpu().numpy() - 1.0)) <= tol


def test_noalloc_rejects_sizes_beyond_its_scratch():
    cfg = api.Config(ng=32, box=100.0, nbins=1500, bin_w2=1)
    g = torch.zeros((32, 32, 17), dtype=torch.complex64, device=DEV)
    st, _, _, _ = _noalloc(cfg, g, g, 1.0, 1.0)
    assert st == ffi.PK_ESIZE
    assert "1024" in ffi.last_error()
