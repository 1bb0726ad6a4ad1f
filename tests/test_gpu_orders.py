"""GPU parity of the B-spline orders beyond PCS (p = 5, 6; the top hat convolved with itself p - 1
times, Sec. 2.3) against the FP64 oracle: power spectra (FP64 1e-10, FP32 1e-5 per bin, exact
counts), the adjoint (1e-9 of the largest component), multi-grid interlacing and the residual
aliasing factor; and the calls that do not take these orders refuse them."""

import numpy as np
import pytest
import torch

import _ref
import oracle
from paper_1512_07295_gb300 import api, catalogs, ffi

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ffi.lib()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("order", [5, 6])
@pytest.mark.parametrize("interlace", [False, True])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_power_orders_5_6_match_oracle(order, interlace, prec, tol):
    box, ng = 300.0, 24
    pos = catalogs.zeldovich(24, box, rms=7.0, seed=81)
    ref_pk, ref_k, ref_cnt, _ = _ref.power(pos, box, ng, order, interlace)
    cfg = api.Config(ng=ng, box=box, order=order, interlace=interlace, prec=prec)
    pk, km, cnt = api.power(_t(pos), cfg)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert _ref.rel(pk.cpu().numpy(), ref_pk) <= tol
    assert _ref.rel(km.cpu().numpy(), ref_k) <= (1e-12 if prec == "fp64" else 1e-6)  # FP32 sums |k| in FP32 pairs


@pytest.mark.parametrize("order", [5, 6])
def test_grids_orders_5_6_packed_records_and_weights(order):
    box, ng = 100.0, 16
    u = np.random.default_rng(82).uniform(0, ng, (4000, 3))
    cells = _ref.pack_cellpos(u, ng)
    uu = _ref.cellpos_to_units(cells, ng)
    w = catalogs.random_weights(len(u), seed=83).astype(np.float32)
    r1 = oracle.assign.assign_units(uu, ng, order, w.astype(np.float64))
    r2 = oracle.assign.assign_units(uu, ng, order, w.astype(np.float64), shift=True)
    g1, g2 = api.assign(_t(cells), api.Config(ng=ng, box=box, order=order, prec="fp32"), weights=_t(w))
    scale = float(r1.max())
    assert np.max(np.abs(g1.cpu().numpy() - r1)) <= 2e-6 * scale
    assert np.max(np.abs(g2.cpu().numpy() - r2)) <= 2e-6 * scale


@pytest.mark.parametrize("order", [5, 6])
@pytest.mark.parametrize("weighted", [False, True])
def test_tiles_orders_5_6_sparse_dense_and_heavy(order, weighted):
    # the tiled scatter takes every tile for p = 5, 6: sparse tiles, a dense one (~2000 particles) and
    # a heavy one (>= 16384 particles: 64-bit region); grids node by node against the oracle
    box, ng = 64.0, 32
    rng = np.random.default_rng(88 + order)
    base = rng.uniform(0.0, box, (6000, 3))
    dense = rng.uniform(0.0, 16.0, (2000, 3)) + np.array([0.0, 16.0, 32.0])
    heavy = rng.uniform(0.0, 16.0, (20000, 3)) + np.array([48.0, 48.0, 0.0])
    pos = np.concatenate([base, dense, heavy]) % box
    cfg = api.Config(ng=ng, box=box, order=order, prec="fp32")
    cells = api.prepare(_t(pos), cfg)
    uu = _ref.cellpos_to_units(cells.cpu().numpy(), ng)
    w = catalogs.random_weights(len(pos), seed=89).astype(np.float32) if weighted else None
    w64 = None if w is None else w.astype(np.float64)
    r1 = oracle.assign.assign_units(uu, ng, order, w64)
    r2 = oracle.assign.assign_units(uu, ng, order, w64, shift=True)
    api.device_error()
    g1, g2 = api.assign(cells, cfg, weights=None if w is None else _t(w))
    assert api.device_error() == 0
    scale = float(np.max(np.abs(r1)))
    assert np.max(np.abs(g1.cpu().numpy() - r1)) <= 2e-6 * scale
    assert np.max(np.abs(g2.cpu().numpy() - r2)) <= 2e-6 * scale


@pytest.mark.parametrize("order", [5, 6])
def test_batch_orders_5_6_match_oracle(order):
    box, ng = 200.0, 24
    cats = [catalogs.poisson(n, box, seed=90 + i) for i, n in enumerate([700, 3000, 1500])]
    cfg = api.Config(ng=ng, box=box, order=order, prec="fp32")
    cells = torch.cat([api.prepare(_t(c), cfg) for c in cats])
    offs = np.concatenate([[0], np.cumsum([len(c) for c in cats])])
    pk, nm = api.batch_power(cells, offs, cfg, batch=2)
    for i in range(len(cats)):
        u = _ref.cellpos_to_units(cells[offs[i]:offs[i + 1]].cpu().numpy(), ng)
        ref_pk, _, ref_cnt = _ref.power_units(u, box, ng, order)
        assert np.array_equal(nm[i].cpu().numpy(), ref_cnt)
        assert _ref.rel(pk[i].cpu().numpy(), ref_pk) <= 1e-5, i


@pytest.mark.parametrize("order", [5, 6])
def test_backward_orders_5_6_match_oracle(order):
    box, ng = 100.0, 16
    pos = catalogs.zeldovich(12, box, rms=4.0, seed=84)
    dl = np.random.default_rng(85).standard_normal(ng // 2)
    ref = oracle.adjoint.position_gradient(pos, box, ng, order, dl, interlace=True)
    cfg = api.Config(ng=ng, box=box, order=order, interlace=True, prec="fp64")
    g = api.power_backward(_t(pos), cfg, _t(dl)).cpu().numpy()
    assert np.max(np.abs(g - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_multigrid_and_aliasing_order_5():
    box, ng = 200.0, 16
    pos = catalogs.zeldovich(16, box, rms=5.0, seed=86)
    shifts = oracle.fourier.multigrid_shifts(4)
    uu = oracle.assign.grid_units(pos, box, ng)
    rhos = [oracle.assign.assign_units(uu, ng, 5, shift=d) for d in shifts]
    ref_pk, _, ref_cnt = oracle.power.power_spectrum(oracle.fourier.density_modes_multi(rhos, shifts, 5), box)
    cfg = api.Config(ng=ng, box=box, order=5, prec="fp64")
    pk, _, cnt = api.power_multigrid(_t(pos), cfg, 4)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert _ref.rel(pk.cpu().numpy(), ref_pk) <= 1e-10
    for order in (5, 6):
        for inter in (False, True):
            c = api.Config(ng=ng, box=box, order=order, interlace=inter, prec="fp64")
            mean, mx, _, n = (t.cpu().numpy() for t in api.aliasing_residual(c, DEV))
            ref_mean, ref_max, ref_n = oracle.aliasing.fres_binned(ng, order, inter)
            assert np.array_equal(n, ref_n)
            assert _ref.rel(mean, ref_mean) <= 1e-10
            assert _ref.rel(mx, ref_max) <= 1e-10


def test_orders_5_6_are_refused_where_unsupported():
    pos = _t(catalogs.poisson(1000, 100.0, seed=87))
    with pytest.raises(ffi.PkError):
        api.power(pos, api.Config(ng=16, box=100.0, order=5, prec="fixed64"))
    with pytest.raises(ffi.PkError):
        api.power(pos, api.Config(ng=16, box=100.0, order=7, prec="fp64"))

