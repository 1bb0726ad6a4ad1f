"""GPU parity of the FP32 tile assignment on both sides of the scatter / key-cell switch (a3).

Each tile (8^3 cells) goes to the direct scatter when it holds fewer particles than a per-order
threshold (PCS 768, TSC 1024, CIC 512; NGP always) and to the key-cell kernel otherwise. The
catalogues below sit just under and just over each threshold, and add the layouts that exercise the
split and the scatter's piece pipeline: dense tiles among sparse ones, and runs of empty tiles
between occupied ones (a finished tile's region is flushed while the next tile's first piece is
scattered). Grids are compared with the FP64 oracle node by node at 2e-6 of the largest node, as
the other FP32 grid tests."""

import numpy as np
import pytest
import torch

import _ref
from paper_1512_07295_gb300 import api, catalogs, ffi

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
THRESHOLD = {1: None, 2: 512, 3: 1024, 4: 768}


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _check(pos, box, ng, order, w=None):
    cfg = api.Config(ng=ng, box=box, order=order, prec="fp32")
    api.device_error()
    g1, g2 = api.assign(_t(pos), cfg, weights=None if w is None else _t(w))
    assert api.device_error() == 0
    r1, r2 = _ref.grids(pos, box, ng, order, None if w is None else w.astype(np.float64))
    scale = np.max(np.abs(r1))
    assert np.max(np.abs(g1.cpu().numpy() - r1)) <= 2e-6 * scale
    assert np.max(np.abs(g2.cpu().numpy() - r2)) <= 2e-6 * scale


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("side", ["under", "over"])
def test_both_sides_of_the_switch(order, side):
    # N = 16: 8 tiles; mean tile population 0.9x or 1.1x the order's threshold
    box, ng = 100.0, 16
    n = int(THRESHOLD[order] * 8 * (0.9 if side == "under" else 1.1))
    pos = catalogs.poisson(n, box, seed=70 + order)
    _check(pos, box, ng, order)


def test_ngp_dense_tiles_take_the_scatter():
    box, ng = 100.0, 16
    pos = catalogs.poisson(8 * 9000, box, seed=75)
    _check(pos, box, ng, 1)


@pytest.mark.parametrize("weighted", [False, True])
def test_dense_tiles_among_sparse_ones(weighted):
    # N = 32 (64 tiles), ~250 particles per tile (scatter), but one tile holds ~3250 particles and
    # another ~1350 (key cells), and a third ~700 (two 512-record pieces on the scatter)
    box, ng = 64.0, 32
    rng = np.random.default_rng(76)
    base = catalogs.poisson(16000, box, seed=77)
    clump1 = rng.uniform(0.0, 16.0, (3000, 3)) + np.array([16.0, 32.0, 48.0])
    clump2 = rng.uniform(0.0, 16.0, (1100, 3)) + np.array([48.0, 0.0, 16.0])
    clump3 = rng.uniform(0.0, 16.0, (450, 3)) + np.array([0.0, 48.0, 32.0])
    pos = np.concatenate([base, clump1, clump2, clump3])
    w = catalogs.random_weights(len(pos), seed=78).astype(np.float32) if weighted else None
    _check(pos, box, ng, 4, w)


@pytest.mark.parametrize("run", [1, 2, 4])
@pytest.mark.parametrize("order", [2, 3, 4])
def test_scatter_runs_of_tiles_along_z(run, order):
    # runs of 1, 2, 4 tiles along z share one scatter region: ~200 particles per tile, one dense tile
    # (key cells) inside a run, so the run's records form two segments, and weights
    box, ng = 64.0, 32
    rng = np.random.default_rng(93 + run + order)
    base = catalogs.poisson(12000, box, seed=94 + order)
    dense = rng.uniform(0.0, 16.0, (2500, 3)) + np.array([16.0, 32.0, 16.0])
    pos = np.concatenate([base, dense])
    w = catalogs.random_weights(len(pos), seed=95).astype(np.float32)
    cfg = api.Config(ng=ng, box=box, order=order, prec="fp32", tile_run=run)
    api.device_error()
    for weights in (None, w):
        g1, g2 = api.assign(_t(pos), cfg, weights=None if weights is None else _t(weights))
        assert api.device_error() == 0
        r1, r2 = _ref.grids(pos, box, ng, order, None if weights is None else weights.astype(np.float64))
        scale = np.max(np.abs(r1))
        assert np.max(np.abs(g1.cpu().numpy() - r1)) <= 2e-6 * scale
        assert np.max(np.abs(g2.cpu().numpy() - r2)) <= 2e-6 * scale


def test_tile_run_is_validated():
    with pytest.raises(ffi.PkError):
        api.power(_t(catalogs.poisson(100, 10.0, seed=96)), api.Config(ng=16, box=10.0, tile_run=3))


@pytest.mark.parametrize("order", [2, 4])
def test_scatter_across_runs_of_empty_tiles(order):
    # N = 64 (512 tiles): 900 particles in three small clumps, so most of a block's tiles are empty
    # and the region of one occupied tile is flushed while the next occupied tile is scattered
    box, ng = 128.0, 64
    rng = np.random.default_rng(79)
    centres = np.array([[10.0, 20.0, 30.0], [70.0, 90.0, 110.0], [120.0, 5.0, 60.0]])
    pos = np.concatenate([c + rng.normal(0.0, 3.0, (300, 3)) for c in centres]) % box
    _check(pos, box, ng, order)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_dense_clump_keeps_sparse_nodes_accurate(order):
    # 10^5 particles in a 2^3-cell cube inside one 8^3-cell tile, next to a background of one particle
    # per cell: the clump's tile also holds background nodes ~10^4 times smaller than its peak. Every
    # node of value >= 0.25 (background nodes are ~1) must match the FP64 oracle relative to its OWN
    # value at 1e-5 (FP32 sums of the window products reach a few 1e-7). Tiles of at least 16384
    # particles are accumulated in 64-bit fixed point: at 32 bits the clump tile's rounding step
    # (2^-15 of a particle's weight) would leave ~1e-4 relative error on its quarter-unit nodes. Lighter
    # nodes of ordinary tiles carry the 32-bit step of their own tile (absolute, ~1e-6 for CIC at one
    # particle per cell), which the other grid tests bound against the largest node.
    box, ng = 64.0, 32
    rng = np.random.default_rng(91)
    base = catalogs.poisson(ng ** 3, box, seed=92)
    clump = rng.uniform(0.0, 4.0, (100000, 3)) + np.array([20.0, 36.0, 52.0])  # cells 10-11, 18-19, 26-27
    pos = np.concatenate([base, clump])
    cfg = api.Config(ng=ng, box=box, order=order, prec="fp32")
    api.device_error()
    g1, g2 = api.assign(_t(pos), cfg)
    assert api.device_error() == 0
    r1, r2 = _ref.grids(pos, box, ng, order)
    for g, r in ((g1.cpu().numpy(), r1), (g2.cpu().numpy(), r2)):
        sel = np.abs(r) >= 0.25
        rel = np.abs(g[sel] - r[sel]) / np.abs(r[sel])
        assert rel.max() <= 1e-5, (rel.max(), np.argmax(rel))
