"""GPU parity of the power-spectrum path (a1..a6) against the FP64 oracle, through the C ABI.

Tolerances: FP64 mode 1e-10 relative per bin (the oracle-parity mode); FP32 and FIXED64 modes 1e-5
relative per bin; integer mode counts bit-exact."""

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


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("interlace", [False, True])
def test_fp64_power_matches_oracle(order, interlace):
    box, ng = 500.0, 32
    pos = catalogs.poisson(20000, box, seed=31)
    ref_pk, ref_k, ref_cnt, _ = _ref.power(pos, box, ng, order, interlace)
    cfg = api.Config(ng=ng, box=box, order=order, interlace=interlace, prec="fp64")
    pk, km, cnt = api.power(_t(pos), cfg)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert _ref.rel(pk.cpu().numpy(), ref_pk) <= 1e-10
    assert _ref.rel(km.cpu().numpy(), ref_k) <= 1e-12


@pytest.mark.parametrize("ng", [32, 36])
@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("interlace", [False, True])
def test_fp32_power_matches_oracle(ng, order, interlace):
    # clustered (Zel'dovich) catalogue; ng = 36 leaves a ragged last tile (36 = 4 * 8 + 4)
    box = 300.0
    pos = catalogs.zeldovich(32, box, rms=6.0, seed=32)
    ref_pk, _, ref_cnt, _ = _ref.power(pos, box, ng, order, interlace)
    cfg = api.Config(ng=ng, box=box, order=order, interlace=interlace, prec="fp32")
    pk, _, cnt = api.power(_t(pos), cfg)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert _ref.rel(pk.cpu().numpy(), ref_pk) <= 1e-5


def test_fixed64_is_order_independent_and_matches_oracle():
    box, ng = 400.0, 32
    pos = catalogs.zeldovich(32, box, rms=5.0, seed=33)
    ref_pk, _, _, _ = _ref.power(pos, box, ng, 4)
    cfg = api.Config(ng=ng, box=box, prec="fixed64")
    a, _, _ = api.power(_t(pos), cfg)
    b, _, _ = api.power(_t(pos), cfg)
    perm = np.random.default_rng(1).permutation(len(pos))
    c, _, _ = api.power(_t(pos[perm]), cfg)
    a, b, c = a.cpu().numpy(), b.cpu().numpy(), c.cpu().numpy()
    assert np.array_equal(a.view(np.int64), b.view(np.int64))
    assert np.array_equal(a.view(np.int64), c.view(np.int64))
    assert _ref.rel(a, ref_pk) <= 1e-5


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6), ("fixed64", 2e-6)])
@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_assign_grids_match_oracle(prec, tol, order):
    box, ng = 100.0, 20
    pos = catalogs.poisson(3000, box, seed=34)
    w = catalogs.random_weights(3000, seed=35)
    r1, r2 = _ref.grids(pos, box, ng, order, w)
    cfg = api.Config(ng=ng, box=box, order=order, prec=prec)
    g1, g2 = api.assign(_t(pos), cfg, weights=_t(w.astype(np.float32)))
    # the GPU takes FP32 weights: compare with the oracle on the same (rounded) weights
    r1, r2 = _ref.grids(pos, box, ng, order, w.astype(np.float32).astype(np.float64))
    scale = np.max(r1)
    assert np.max(np.abs(g1.cpu().numpy() - r1)) <= tol * scale
    assert np.max(np.abs(g2.cpu().numpy() - r2)) <= tol * scale


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_fft_estimate_from_oracle_grids(prec, tol):
    box, ng, p = 200.0, 24, 3
    pos = catalogs.zeldovich(16, box, rms=4.0, seed=36)
    r1, r2 = _ref.grids(pos, box, ng, p)
    _, _, _, delta = _ref.power(pos, box, ng, p)
    cfg = api.Config(ng=ng, box=box, order=p, prec=prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    d = api.fft_estimate(_t(r1).to(dt), _t(r2).to(dt), cfg, float(r1.sum())).cpu().numpy()
    ref = _ref.half_complex(delta)
    assert np.max(np.abs(d - ref)) <= tol * np.max(np.abs(ref))


def test_binned_path_equals_unbinned():
    box, ng = 300.0, 32
    pos = catalogs.zeldovich(32, box, rms=6.0, seed=37)
    cfg = api.Config(ng=ng, box=box, prec="fp32")
    tpos = _t(pos)
    a, _, ca = api.power(tpos, cfg)
    b, _, cb = api.power_binned(api.bin_particles(tpos, cfg), cfg)
    assert torch.equal(ca, cb)
    assert _ref.rel(b.cpu().numpy(), a.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_weighted_catalogue_and_shot_noise(prec, tol):
    box, ng = 250.0, 32
    pos = catalogs.poisson(15000, box, seed=38)
    w = catalogs.random_weights(15000, seed=39).astype(np.float32).astype(np.float64)
    ref_pk, _, _, _ = _ref.power(pos, box, ng, 4, weights=w, subtract=True)
    cfg = api.Config(ng=ng, box=box, prec=prec, subtract_shot=True)
    pk, _, _ = api.power(_t(pos), cfg, weights=_t(w.astype(np.float32)))
    # shot-noise subtracted bins of a Poisson catalogue are near zero: compare on the scale of 1/nbar
    shot = box ** 3 * np.sum(w * w) / np.sum(w) ** 2
    assert np.max(np.abs(pk.cpu().numpy() - ref_pk)) <= tol * shot


def test_cellpos_input_fp64_mode():
    box, ng = 150.0, 32
    pos = catalogs.zeldovich(24, box, rms=3.0, seed=40)
    cfg = api.Config(ng=ng, box=box, prec="fp64")
    cells = api.prepare(_t(pos), cfg)
    u = _ref.cellpos_to_units(cells.cpu().numpy(), ng)
    ref_pk, _, ref_cnt = _ref.power_units(u, box, ng, 4)
    pk, _, cnt = api.power(cells, cfg)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert _ref.rel(pk.cpu().numpy(), ref_pk) <= 1e-10


def test_prepare_offsets_and_cells():
    box, ng = 100.0, 16
    pos = np.array([[0.0, 50.0, 99.999999], [100.0, -1.0, 250.0], [12.5, 6.25, 93.75]])
    cells = api.prepare(_t(pos), api.Config(ng=ng, box=box)).cpu().numpy()
    u = _ref.cellpos_to_units(cells, ng)
    expect = np.mod(pos, box) * ng / box
    expect[expect >= ng] -= ng
    d = np.abs(u - expect)
    d = np.minimum(d, ng - d)  # periodic
    assert np.max(d) < 1e-6
    f = cells[:, 1:].copy().view(np.float32)
    assert np.all((f >= 0) & (f < 1))


def test_prepare_is_the_fp64_definition_bit_for_bit():
    # N = L, so u = x exactly: the record must hold c = floor(u) and f = float32(u - c) (round to
    # nearest, ties to even; an f that rounds to 1 moves to the next cell, periodically). Random
    # positions, exact FP32 ties of the fraction, fractions that round up to 1 and the last cell.
    ng = 64
    box = float(ng)
    rng = np.random.default_rng(43)
    x = [rng.uniform(0.0, box, 200000)]
    k = rng.integers(0, ng, 4000).astype(np.float64)
    j = rng.integers(0, 2 ** 20, 4000).astype(np.float64)
    x.append(k + 0.25 + (2 * j + 1) * 2.0 ** -26)  # halfway between FP32 neighbours in [1/4, 1/2)
    x.append(k + 0.5 + (2 * j + 1) * 2.0 ** -25)  # halfway in [1/2, 1)
    x.append(k + 1.0 - 2.0 ** -26)  # rounds up to 1: next cell
    x.append(k + 1.0 - 3 * 2.0 ** -26)
    x.append(np.array([box - 2.0 ** -40, box - 2.0 ** -26, 0.0, 2.0 ** -60, 0.5 - 2.0 ** -25]))
    x = np.concatenate(x)
    x = x[(x >= 0.0) & (x < box)]
    pos = np.stack([x, np.roll(x, 1), np.roll(x, 2)], axis=1)
    cells = api.prepare(_t(pos), api.Config(ng=ng, box=box)).cpu().numpy()
    c = np.floor(pos).astype(np.int64)
    f = (pos - c).astype(np.float32)
    up = f >= np.float32(1.0)
    c = np.where(up, c + 1, c) % ng
    f = np.where(up, np.float32(0.0), f).astype(np.float32)
    got_c = cells[:, 0].view(np.uint32).astype(np.int64)
    assert np.array_equal((got_c >> 20) & 1023, c[:, 0])
    assert np.array_equal((got_c >> 10) & 1023, c[:, 1])
    assert np.array_equal(got_c & 1023, c[:, 2])
    assert np.array_equal(cells[:, 1:], f.view(np.int32))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fixed64"])
def test_edge_positions_and_tiny_grid(prec):
    # positions on the box faces, outside the box and on nodes; ng = 8 makes the shared-memory
    # region (8 + 4 nodes per axis) wrap onto itself
    box, ng = 80.0, 8
    rng = np.random.default_rng(41)
    pos = np.concatenate([rng.uniform(-80.0, 160.0, size=(500, 3)), np.array([[0.0, 0.0, 0.0], [80.0, 80.0, 80.0],
                                                                                 [40.0, 10.0, 70.0], [79.9999, 0.0, 80.0]])])
    ref_pk, _, ref_cnt, _ = _ref.power(pos, box, ng, 4)
    pk, _, cnt = api.power(_t(pos), api.Config(ng=ng, box=box, prec=prec))
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert _ref.rel(pk.cpu().numpy(), ref_pk) <= (1e-10 if prec == "fp64" else 1e-5)


def test_single_particle_and_full_lattice():
    box, ng = 64.0, 16
    one = np.array([[10.3, 20.7, 33.3]])
    ref_pk, _, _, _ = _ref.power(one, box, ng, 4)
    pk, _, _ = api.power(_t(one), api.Config(ng=ng, box=box, prec="fp64"))
    assert _ref.rel(pk.cpu().numpy(), ref_pk) <= 1e-10
    lat = catalogs.lattice(ng, box, offset=0.0)
    pk, _, _ = api.power(_t(lat), api.Config(ng=ng, box=box, prec="fp64"))
    assert np.max(np.abs(pk.cpu().numpy())) < 1e-20 * box ** 3 / ng ** 3


def test_custom_bins_and_empty_bins():
    box, ng = 100.0, 16
    pos = catalogs.poisson(5000, box, seed=42)
    # edges 0, 1, 2, ... in units of k_f/2: the first bin starts at 0 (k = 0 must stay out) and the
    # first two bins (|n| < 1/2 and 1/2 <= |n| < 1) hold no mode at all
    lo2, w2, nb = 0, 1, 24
    edges = lo2 + w2 * np.arange(nb + 1)
    ref_pk, _, ref_cnt, _ = _ref.power(pos, box, ng, 4, edges=edges)
    pk, _, cnt = api.power(_t(pos), api.Config(ng=ng, box=box, prec="fp64", bin_lo2=lo2, bin_w2=w2, nbins=nb))
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    pk = pk.cpu().numpy()
    empty = ref_cnt == 0
    assert np.all(np.isnan(pk[empty]))
    assert _ref.rel(pk[~empty], ref_pk[~empty]) <= 1e-10


def test_nonfinite_position_sets_device_error():
    box, ng = 100.0, 16
    pos = catalogs.poisson(1000, box, seed=43)
    api.device_error()  # clear
    bad = pos.copy()
    bad[5, 1] = np.nan
    pk, _, _ = api.power(_t(bad), api.Config(ng=ng, box=box, prec="fp64"))
    err = api.device_error()
    assert err & ffi.PK_DERR_NONFINITE
    assert np.all(np.isfinite(pk.cpu().numpy()))
    assert api.device_error() == 0


def test_small_workspace_is_rejected():
    import ctypes

    box, ng = 100.0, 16
    cfg = api.Config(ng=ng, box=box)
    pos = _t(catalogs.poisson(100, box, seed=44))
    ws = torch.empty(64, dtype=torch.uint8, device=DEV)
    out = torch.empty(ng // 2, dtype=torch.float64, device=DEV)
    cnt = torch.empty(ng // 2, dtype=torch.int64, device=DEV)
    st = ffi.lib().pk_power(ctypes.byref(cfg.c()), api._p(pos), ffi.PK_POS_F64_XYZ, None, 100, api._p(out), api._p(out),
                            api._p(cnt), None, api._p(ws), 64, None)
    assert st == ffi.PK_ESIZE


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("lo2, w2, nb", [(0, 1, 200), (0, 1, 400), (0, 1, 700), (2, 300, 200)])
def test_estimate_paths_by_bin_count(prec, lo2, w2, nb):
    # N = 64 puts four rows in each warp of the row estimate. 200 and 400 bins need its blocks of
    # four and two warps (private copies within 96 KB); 700 bins go to the item kernel with shared
    # atomics; edges up to 2 + 200 x 300 squared exceed 32 bits, so the last case takes the 64-bit bin
    # test. Bins past the grid's largest |n| stay empty.
    box, ng = 200.0, 64
    pos = catalogs.zeldovich(32, box, rms=3.0, seed=71)
    edges = lo2 + w2 * np.arange(nb + 1)
    ref_pk, _, ref_cnt, _ = _ref.power(pos, box, ng, 4, edges=edges)
    pk, _, cnt = api.power(_t(pos), api.Config(ng=ng, box=box, prec=prec, bin_lo2=lo2, bin_w2=w2, nbins=nb))
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    pk = pk.cpu().numpy()
    full = ref_cnt > 0
    assert np.all(np.isnan(pk[~full]))
    assert _ref.rel(pk[full], ref_pk[full]) <= (1e-10 if prec == "fp64" else 1e-5)
