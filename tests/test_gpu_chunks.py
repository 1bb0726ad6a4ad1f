"""GPU parity of the FP32 assignment on tiles too dense to stage at once: a tile's key cells are
summed piece by piece, a half-cell slab can straddle two pieces, and the order of the particles inside
a tile is free. Grids are compared with the FP64 oracle node by node (2e-6 of the
largest node, as the other FP32 grid tests), P(k) per bin at 1e-5, counts bit-exact."""

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
@pytest.mark.parametrize("weighted", [False, True])
def test_dense_tiles_grids_match_oracle(order, weighted):
    # 48^3 clustered particles on N = 16 (8 tiles of 8^3 cells): ~14k particles per tile, staged in
    # 3 (unit weights) or 4 (weighted) pieces of the 32-bit-region kernel
    box, ng = 100.0, 16
    pos = catalogs.zeldovich(48, box, rms=3.0, seed=61)
    w = catalogs.random_weights(len(pos), seed=62).astype(np.float32) if weighted else None
    cfg = api.Config(ng=ng, box=box, order=order, prec="fp32")
    api.device_error()
    g1, g2 = api.assign(_t(pos), cfg, weights=_t(w) if weighted else None)
    assert api.device_error() == 0
    r1, r2 = _ref.grids(pos, box, ng, order, None if w is None else w.astype(np.float64))
    scale = np.max(np.abs(r1))
    assert np.max(np.abs(g1.cpu().numpy() - r1)) <= 2e-6 * scale
    assert np.max(np.abs(g2.cpu().numpy() - r2)) <= 2e-6 * scale


@pytest.mark.parametrize("order", [2, 3, 4])
def test_dense_tiles_power_matches_oracle(order):
    box, ng = 100.0, 16
    pos = catalogs.zeldovich(48, box, rms=3.0, seed=63)
    ref_pk, _, ref_cnt, _ = _ref.power(pos, box, ng, order, True)
    pk, _, cnt = api.power(_t(pos), api.Config(ng=ng, box=box, order=order, prec="fp32"))
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert _ref.rel(pk.cpu().numpy(), ref_pk) <= 1e-5


@pytest.mark.parametrize("order", [2, 3, 4])
def test_one_slab_spans_several_pieces(order):
    # every particle in the first half-cell slab along x of a one-tile grid: 6000 particles in one
    # slab, more than one staged piece holds
    box, ng, n = 8.0, 8, 6000
    rng = np.random.default_rng(64)
    pos = np.stack([rng.uniform(0.0, 0.5, n), rng.uniform(0.0, box, n), rng.uniform(0.0, box, n)], axis=1)
    cfg = api.Config(ng=ng, box=box, order=order, prec="fp32")
    api.device_error()
    g1, g2 = api.assign(_t(pos), cfg)
    assert api.device_error() == 0
    r1, r2 = _ref.grids(pos, box, ng, order)
    scale = np.max(np.abs(r1))
    assert np.max(np.abs(g1.cpu().numpy() - r1)) <= 2e-6 * scale
    assert np.max(np.abs(g2.cpu().numpy() - r2)) <= 2e-6 * scale


def test_binned_layout_in_any_order_inside_a_tile():
    # one tile of 20000 particles (a heavy tile: 3 staged pieces); the binned order reversed puts every half-cell
    # slab in descending order: key cells are sorted per piece, so the order inside a tile is free
    box, ng = 8.0, 8
    pos = catalogs.poisson(20000, box, seed=65)
    cfg = api.Config(ng=ng, box=box, prec="fp32")
    sorted_, wsorted, offsets = api.bin_particles(_t(pos), cfg)
    ref_pk, _, ref_cnt, _ = _ref.power(pos, box, ng, 4, True)
    api.device_error()
    for layout in (sorted_, torch.flip(sorted_, dims=[0]).contiguous()):
        pk, _, cnt = api.power_binned((layout, wsorted, offsets), cfg)
        assert api.device_error() == 0
        assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
        assert _ref.rel(pk.cpu().numpy(), ref_pk) <= 1e-5


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("weighted", [False, True])
def test_fixed64_dense_tiles_are_order_independent_and_match_oracle(order, weighted):
    # PK_FIXED64 on tiles of ~14k particles (the key cells, every product rounded at the tile's scale
    # and the integers summed exactly): the same grids bit for bit from a permuted catalogue, and within
    # 1e-5 of the largest node of the FP64 oracle. The 32-bit region bounds the scale by the tile's
    # population (14k x node share x 2^e < 2^30: e = 16 for CIC), so each rounding is up to 2^-17 of a
    # unit weight and a node of ~10^3 contributions carries ~2e-6 of the largest node.
    box, ng = 100.0, 16
    pos = catalogs.zeldovich(48, box, rms=3.0, seed=66)
    w = catalogs.random_weights(len(pos), seed=67).astype(np.float32) if weighted else None
    cfg = api.Config(ng=ng, box=box, order=order, prec="fixed64")
    perm = np.random.default_rng(68).permutation(len(pos))
    api.device_error()
    g1, g2 = api.assign(_t(pos), cfg, weights=_t(w) if weighted else None)
    h1, h2 = api.assign(_t(pos[perm]), cfg, weights=_t(w[perm]) if weighted else None)
    assert api.device_error() == 0
    assert torch.equal(g1, h1) and torch.equal(g2, h2)
    r1, r2 = _ref.grids(pos, box, ng, order, None if w is None else w.astype(np.float64))
    scale = np.max(np.abs(r1))
    assert np.max(np.abs(g1.cpu().numpy() - r1)) <= 1e-5 * scale
    assert np.max(np.abs(g2.cpu().numpy() - r2)) <= 1e-5 * scale


def test_fixed64_clump_tile_is_order_independent():
    # a clump of 30000 particles inside two cells (one heavy tile on the deterministic key cells, its
    # scale set by the population) among 5000 uniform ones: bit-identical grids from a permuted
    # catalogue, within 1e-5 of the largest node of the FP64 oracle
    box, ng = 100.0, 16
    rng = np.random.default_rng(69)
    clump = 40.0 + rng.uniform(0.0, 2.0 * box / ng, size=(30000, 3))
    pos = np.concatenate([clump, rng.uniform(0.0, box, size=(5000, 3))])
    cfg = api.Config(ng=ng, box=box, order=4, prec="fixed64")
    perm = rng.permutation(len(pos))
    api.device_error()
    g1, g2 = api.assign(_t(pos), cfg)
    h1, h2 = api.assign(_t(pos[perm]), cfg)
    assert api.device_error() == 0
    assert torch.equal(g1, h1) and torch.equal(g2, h2)
    r1, r2 = _ref.grids(pos, box, ng, 4)
    scale = np.max(np.abs(r1))
    assert np.max(np.abs(g1.cpu().numpy() - r1)) <= 1e-5 * scale
    assert np.max(np.abs(g2.cpu().numpy() - r2)) <= 1e-5 * scale
