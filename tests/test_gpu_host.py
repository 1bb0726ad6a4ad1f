"""pk_power_host: P(k) end to end from host memory. Pinned positions are read by the GPU over the
CPU-GPU link, pageable ones are staged through the workspace; both must give the device path's
result (FP32 atomics make the summation order differ between any two runs: 1e-6 relative per bin on
the sparse catalogues, 1e-5 on the dense one) and the FP64 oracle's (1e-5 in FP32 mode, 1e-10 in FP64
mode), with mode counts bit-exact."""

import ctypes

import numpy as np
import pytest
import torch

import _ref
from paper_1512_07295_gb300 import api, catalogs, ffi

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ffi.lib()


def _host(a, pinned):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-10), ("fixed64", 1e-5)])
def test_host_positions_match_device_path_and_oracle(pinned, prec, tol):
    box, ng = 300.0, 32
    pos = catalogs.zeldovich(32, box, rms=6.0, seed=71)
    cfg = api.Config(ng=ng, box=box, prec=prec)
    pk_h, km_h, cnt_h = api.power_host(_host(pos, pinned), cfg)
    torch.cuda.synchronize()
    pk_d, km_d, cnt_d = api.power(torch.from_numpy(pos).to(DEV), cfg)
    assert torch.equal(cnt_h, cnt_d.cpu())
    assert _ref.rel(pk_h.numpy(), pk_d.cpu().numpy()) <= (1e-12 if prec == "fp64" else 1e-6)
    ref_pk, ref_k, ref_cnt, _ = _ref.power(pos, box, ng, 4)
    assert np.array_equal(cnt_h.numpy(), ref_cnt)
    assert _ref.rel(pk_h.numpy(), ref_pk) <= tol
    assert _ref.rel(km_h.numpy(), ref_k) <= 1e-6


@pytest.mark.parametrize("pinned", [True, False])
def test_host_weights_and_packed_records(pinned):
    box, ng = 200.0, 24
    pos = catalogs.poisson(30000, box, seed=72)
    w = catalogs.random_weights(len(pos), seed=73).astype(np.float32)
    cfg = api.Config(ng=ng, box=box, order=3, prec="fp32")
    pk_h, _, cnt_h = api.power_host(_host(pos, pinned), cfg, weights=_host(w, pinned))
    torch.cuda.synchronize()
    ref_pk, _, ref_cnt, _ = _ref.power(pos, box, ng, 3, weights=w.astype(np.float64))
    assert np.array_equal(cnt_h.numpy(), ref_cnt)
    assert _ref.rel(pk_h.numpy(), ref_pk) <= 1e-5
    # the packed cell + offset format from host memory
    cells = api.prepare(torch.from_numpy(pos).to(DEV), cfg).cpu()
    pk_c, _, _ = api.power_host(_host(cells.numpy(), pinned), cfg, weights=_host(w, pinned))
    torch.cuda.synchronize()
    assert _ref.rel(pk_c.numpy(), pk_h.numpy()) <= 1e-6


def test_pageable_positions_in_several_pieces():
    # FP32 from FP64 positions crosses the link in pieces of at least 2^20 particles: five pieces here,
    # each binned and added to the grids while the next one is copied
    box, ng, n = 1000.0, 64, 5_000_000
    pos = catalogs.poisson(n, box, seed=74)
    cfg = api.Config(ng=ng, box=box, prec="fp32")
    pk_h, _, cnt_h = api.power_host(torch.from_numpy(pos), cfg)
    torch.cuda.synchronize()
    pk_d, _, cnt_d = api.power(torch.from_numpy(pos).to(DEV), cfg)
    assert torch.equal(cnt_h, cnt_d.cpu())
    # 19 particles per cell: the lowest bins' power is a small difference of large FP32 grid sums, so
    # two FP32 runs differ there by more than in the sparser cases above (summation order only)
    assert _ref.rel(pk_h.numpy(), pk_d.cpu().numpy()) <= 1e-5


def test_pinned_weighted_positions_in_several_pieces():
    # pinned positions and weights in four pieces (the last one short): the weights of each piece
    # follow its positions
    box, ng, n = 800.0, 48, 3_500_000
    pos = catalogs.poisson(n, box, seed=76)
    w = catalogs.random_weights(n, seed=77).astype(np.float32)
    cfg = api.Config(ng=ng, box=box, prec="fp32")  # a Poisson catalogue: P is the shot noise, kept in
    pk_h, km_h, cnt_h = api.power_host(_host(pos, True), cfg, weights=_host(w, True))
    torch.cuda.synchronize()
    pk_d, km_d, cnt_d = api.power(torch.from_numpy(pos).to(DEV), cfg, weights=torch.from_numpy(w).to(DEV))
    assert torch.equal(cnt_h, cnt_d.cpu())
    assert _ref.rel(pk_h.numpy(), pk_d.cpu().numpy()) <= 1e-5
    assert _ref.rel(km_h.numpy(), km_d.cpu().numpy()) <= 1e-6


def test_device_pointer_is_rejected():
    box, ng = 100.0, 16
    cfg = api.Config(ng=ng, box=box)
    pos = torch.from_numpy(catalogs.poisson(100, box, seed=75)).to(DEV)
    ws = api.workspace(cfg, 100, ffi.PK_WS_POWER_HOST, pos.device)
    out = np.zeros(cfg.nb)
    cnt = np.zeros(cfg.nb, dtype=np.int64)
    st = ffi.lib().pk_power_host(ctypes.byref(cfg.c()), api._p(pos), ffi.PK_POS_F64_XYZ, None, 100,
                                 out.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                                 cnt.ctypes.data_as(ctypes.c_void_p), api._p(ws), ws.numel(), api._stream(pos.device))
    assert st == ffi.PK_EINVAL
