"""GPU parity of the direct summation of eq:deltaDS (pk_direct_modes) and of the half-complex cross
power (pk_cross_power) against the FP64 oracle, through the C ABI.

Tolerances. FP64 mode: 1e-12 absolute on delta (|delta| <= sum|w|/sum w = 1 for positive weights).
FP32 mode (tensor cores, three TF32 products per term): each product w e^{-i k.x} = a b carries the
hardware sine/cosine of its two factors (absolute error 2^-21.4 each), about 3 x 2^-21 from the TF32
split and a few FP32 roundings, and each run of 64 products is summed in FP32 before the compensated
total (at most 63 eps_32 of the sum of the magnitudes), so the error is bounded by about
(2 x 2^-21.4 + 3 x 2^-21 + 4 eps_32 + 63 eps_32) sum|w| / sum w = 6.2e-6; the tests use 7e-6.
Binned cross powers of given fields: 1e-12 relative per bin (FP64 sums), counts bit-exact."""

import numpy as np
import pytest
import torch

import _ref
import oracle
from paper_1512_07295_gb300 import api, catalogs, ffi

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL32 = 7e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ffi.lib()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _oracle_half(pos, box, ng, weights=None):
    return _ref.half_complex(oracle.direct.direct_modes(pos, box, ng, weights))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", TOL32)])
@pytest.mark.parametrize("weighted", [False, True])
def test_direct_modes_match_oracle(prec, tol, weighted):
    # N = 24: 24 columns of a 32-wide tile and 312 rows (i_x, i_z) of two 256-row tiles, both ragged;
    # 6859 particles: a ragged last chunk and several particle slices
    box, ng = 300.0, 24
    pos = catalogs.zeldovich(19, box, rms=8.0, seed=51)
    w = catalogs.random_weights(len(pos), seed=52) if weighted else None
    ref = _oracle_half(pos, box, ng, w)
    cfg = api.Config(ng=ng, box=box, prec=prec)
    d = api.direct_modes(_t(pos), cfg, weights=_t(w.astype(np.float32)) if weighted else None).cpu().numpy()
    if weighted:  # the library takes FP32 weights: compare with the oracle on the same values
        ref = _oracle_half(pos, box, ng, w.astype(np.float32).astype(np.float64))
    assert d.shape == ref.shape
    assert np.max(np.abs(d - ref)) <= tol
    assert d[0, 0, 0] == 0


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", TOL32)])
def test_direct_modes_from_packed_records(prec, tol):
    box, ng = 200.0, 16
    u = np.random.default_rng(53).uniform(0, ng, (3000, 3))
    cells = _ref.pack_cellpos(u, ng)
    pos = _ref.cellpos_to_units(cells, ng) * (box / ng)
    ref = _oracle_half(pos, box, ng)
    d = api.direct_modes(_t(cells), api.Config(ng=ng, box=box, prec=prec)).cpu().numpy()
    assert np.max(np.abs(d - ref)) <= tol


def test_direct_modes_single_particle_and_positions_outside_the_box():
    # one particle: |delta(n)| = 1 on every mode but n = 0; positions in any periodic image agree
    box, ng = 64.0, 8
    x = np.array([[12.3, 45.6, 7.8]])
    ref = _oracle_half(x, box, ng)
    cfg = api.Config(ng=ng, box=box, prec="fp64")
    d1 = api.direct_modes(_t(x), cfg).cpu().numpy()
    d2 = api.direct_modes(_t(x + np.array([[box, -3 * box, 7 * box]])), cfg).cpu().numpy()
    assert np.max(np.abs(d1 - ref)) <= 1e-12
    assert np.max(np.abs(d2 - ref)) <= 1e-12
    mag = np.abs(d1).ravel()[1:]
    assert np.max(np.abs(mag - 1.0)) <= 1e-12


def test_direct_modes_at_the_largest_grid_size_sampled():
    # N = 1024 (the library's maximum) with 2048 particles: 537 M stored modes, compared at sampled
    # modes (Nyquist components included) with the oracle's sum at those vectors
    box, ng = 1000.0, 1024
    pos = catalogs.poisson(2048, box, seed=54)
    cfg = api.Config(ng=ng, box=box, prec="fp32")
    d = api.direct_modes(_t(pos), cfg)
    rng = np.random.default_rng(55)
    idx = np.concatenate([rng.integers(0, [ng, ng, ng // 2 + 1], (40, 3)),
                          [[ng // 2, ng // 2, ng // 2], [ng // 2, 0, 1], [0, ng - 1, ng // 2], [1, 2, 3]]])
    sn = lambda i: np.where(i < ng // 2, i, i - ng)
    nvec = np.stack([sn(idx[:, 0]), sn(idx[:, 1]), np.where(idx[:, 2] == ng // 2, -(ng // 2), idx[:, 2])], 1)
    ref = oracle.direct.direct_modes_at(pos, box, nvec)
    got = d[idx[:, 0], idx[:, 1], idx[:, 2]].cpu().numpy()
    assert np.max(np.abs(got - ref)) <= TOL32
    del d
    torch.cuda.empty_cache()


def test_cross_power_bins_given_fields():
    # the binning alone, on fields made on the host: FP64 sums, exact counts
    box, ng = 150.0, 20
    rng = np.random.default_rng(56)
    shape = (ng, ng, ng // 2 + 1)
    a = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    b = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    ref_pk, ref_k, ref_cnt = oracle.power.cross_power_half(a, b, box)
    cfg = api.Config(ng=ng, box=box, prec="fp64")
    pk, km, cnt = api.cross_power(_t(a), _t(b), cfg)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert _ref.rel(pk.cpu().numpy(), ref_pk) <= 1e-12
    assert _ref.rel(km.cpu().numpy(), ref_k) <= 1e-12


def test_grid_estimate_against_direct_summation():
    # Sec. 3.2 comparison on the GPU: P_DS, P_G and the cross power P_{G-DS} of a clustered catalogue,
    # each against the oracle; PCS + interlacing agrees with the direct sum far better than CIC.
    box, ng = 400.0, 32
    pos = catalogs.zeldovich(32, box, rms=6.0, seed=57)
    ds_ref = _oracle_half(pos, box, ng)
    p_ds_ref, _, cnt_ref = oracle.power.cross_power_half(ds_ref, ds_ref, box)
    cfg = api.Config(ng=ng, box=box, order=4, interlace=True, prec="fp32")
    ds = api.direct_modes(_t(pos), cfg)
    p_ds, _, cnt = api.cross_power(ds, ds, cfg)
    assert np.array_equal(cnt.cpu().numpy(), cnt_ref)
    assert _ref.rel(p_ds.cpu().numpy(), p_ds_ref) <= 1e-5
    errs = {}
    for order, inter in ((2, False), (4, True)):
        c = api.Config(ng=ng, box=box, order=order, interlace=inter, prec="fp32")
        _, _, _, dg = api.power(_t(pos), c, return_delta=True)
        p_x, _, _ = api.cross_power(dg, ds, c)
        _, _, _, dg_ref = _ref.power(pos, box, ng, order, inter)
        p_x_ref, _, _ = oracle.power.cross_power_half(_ref.half_complex(dg_ref), ds_ref, box)
        assert _ref.rel(p_x.cpu().numpy(), p_x_ref) <= 1e-5
        errs[(order, inter)] = np.max(np.abs(p_x.cpu().numpy() / p_ds.cpu().numpy() - 1.0))
    assert errs[(4, True)] < errs[(2, False)]


def test_direct_modes_rejects_bad_arguments():
    cfg = api.Config(ng=16, box=100.0, prec="fp32")
    with pytest.raises(ffi.PkError):
        api.direct_modes(torch.empty((0, 3), dtype=torch.float64, device=DEV), cfg)
    api.device_error()
    pos = np.array([[1.0, np.nan, 3.0], [4.0, 5.0, 6.0]])
    api.direct_modes(_t(pos), cfg)
    assert api.device_error() & ffi.PK_DERR_NONFINITE
