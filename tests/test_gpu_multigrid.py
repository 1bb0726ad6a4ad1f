"""GPU parity of multi-grid interlacing (pk_power_multigrid, J = 1, 2, 4, 8 half-cell-shifted grids)
against the FP64 oracle: FP64 mode 1e-10 relative per bin, FP32 1e-5 (the tolerances of pk_power);
mode counts bit-exact; the combined delta(n) on every stored mode, compared as W(n) |delta - delta_ref|
(1e-12 in FP64, 20 FP32 ulps in FP32)."""

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


def _oracle(u, ng, p, box, ngrids, weights=None):
    shifts = oracle.fourier.multigrid_shifts(ngrids)
    rhos = [oracle.assign.assign_units(u, ng, p, weights, shift=d) for d in shifts]
    delta = oracle.fourier.density_modes_multi(rhos, shifts, p)
    return oracle.power.power_spectrum(delta, box) + (delta,)


@pytest.mark.parametrize("ngrids", [1, 2, 4, 8])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_multigrid_power_matches_oracle(ngrids, prec, tol):
    # N = 24: three 8-cell tiles per axis; a clustered catalogue
    box, ng, p = 300.0, 24, 3
    pos = catalogs.zeldovich(24, box, rms=7.0, seed=71)
    ref_pk, ref_k, ref_cnt, ref_delta = _oracle(oracle.assign.grid_units(pos, box, ng), ng, p, box, ngrids)
    cfg = api.Config(ng=ng, box=box, order=p, prec=prec)
    pk, km, cnt, delta = api.power_multigrid(_t(pos), cfg, ngrids, return_delta=True)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert _ref.rel(pk.cpu().numpy(), ref_pk) <= tol
    assert _ref.rel(km.cpu().numpy(), ref_k) <= 1e-12
    # delta before the window division: an FP32 transform errs by a few ulps of the mean density on
    # every mode, which 1/W(n) enlarges near the Nyquist corner (as in the full-size test)
    err = np.abs(delta.cpu().numpy() - _ref.half_complex(ref_delta)) * _ref.half_complex(oracle.fourier.window_3d(p, ng))
    assert err.max() <= (20 * np.finfo(np.float32).eps if prec == "fp32" else 1e-12)


@pytest.mark.parametrize("ngrids", [4, 8])
def test_multigrid_weights_packed_records_and_shot_noise(ngrids):
    box, ng, p = 200.0, 16, 4
    u = np.random.default_rng(72).uniform(0, ng, (5000, 3))
    cells = _ref.pack_cellpos(u, ng)
    uu = _ref.cellpos_to_units(cells, ng)
    w = catalogs.random_weights(len(u), seed=73).astype(np.float32)
    ref_pk, _, ref_cnt, _ = _oracle(uu, ng, p, box, ngrids, w.astype(np.float64))
    shot = oracle.power.shot_noise(box, w.astype(np.float64))
    cfg = api.Config(ng=ng, box=box, order=p, prec="fp32", subtract_shot=True)
    pk, _, cnt = api.power_multigrid(_t(cells), cfg, ngrids, weights=_t(w))
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    # compare before the subtraction: the shot noise is several times the residual power here
    assert _ref.rel(pk.cpu().numpy() + shot, ref_pk) <= 1e-5


def test_two_grids_agree_with_the_interlaced_power():
    box, ng = 400.0, 32
    pos = _t(catalogs.zeldovich(32, box, rms=6.0, seed=74))
    cfg = api.Config(ng=ng, box=box, order=4, interlace=True, prec="fp64")
    a, _, ca = api.power(pos, cfg)
    b, _, cb = api.power_multigrid(pos, cfg, 2)
    assert torch.equal(ca, cb)
    assert _ref.rel(b.cpu().numpy(), a.cpu().numpy()) <= 1e-12


def test_multigrid_rejects_other_grid_counts():
    cfg = api.Config(ng=16, box=100.0)
    pos = _t(catalogs.poisson(100, 100.0, seed=75))
    for bad in (0, 3, 16):
        with pytest.raises(ffi.PkError):
            api.power_multigrid(pos, cfg, bad)


@pytest.mark.parametrize("fmt", ["records", "f64"])
def test_offsets_whose_half_shift_rounds_to_one(fmt):
    # f = 1/2 - 2^-25 is the one FP32 offset below 1/2 whose f + 1/2 rounds to 1: the shifted record
    # must move to the next cell (offset 0) rather than be reported invalid and dropped. Packed records
    # carry it directly; from FP64 positions, x = (c + f) H prepares to the same offset.
    box, ng, p = 64.0, 16, 4
    rng = np.random.default_rng(76)
    u = rng.uniform(0, ng, (3000, 3))
    f = np.float64(np.float32(0.5) - np.float32(2.0 ** -25))
    edge = np.floor(rng.uniform(0, ng, (60, 3))) + f  # every axis at the edge offset
    uu = np.concatenate([u, edge])
    cells = _ref.pack_cellpos(uu, ng)
    exact = _ref.cellpos_to_units(cells, ng)
    assert np.array_equal(exact[-60:], edge)  # the edge offsets survive packing
    ref_pk, _, ref_cnt, _ = _oracle(exact, ng, p, box, 8)
    cfg = api.Config(ng=ng, box=box, order=p, prec="fp32")
    pos = _t(cells) if fmt == "records" else _t(exact * (box / ng))
    api.device_error()
    pk, _, cnt = api.power_multigrid(pos, cfg, 8)
    assert api.device_error() == 0
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert _ref.rel(pk.cpu().numpy(), ref_pk) <= 1e-5
