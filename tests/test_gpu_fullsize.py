"""Parity at the benchmark's full size: 1024^3 Zel'dovich particles, L = 2000 Mpc/h, N_G = 512, PCS +
interlacing, FP32 cell + offset positions. This is the catalogue and the pk_power_binned call that
bench.py times.

The FP64 oracle cannot assign 10^9 particles, so the checks are of two kinds:
- sampled outputs it computes one by one: mass-grid nodes, each from the particles near it;
- properties that hold at any size: mass conservation. The transforms, the window-corrected modes
  and P(k) are recomputed by the oracle from the GPU's own mass grids.

Tolerances are those of the small FP32 tests: grids within 2e-6 of the largest node, modes within
1e-5 of the largest, P(k) within 1e-5 per bin, mode counts exact."""

import numpy as np
import pytest
import torch

import _ref
import oracle
from paper_1512_07295_gb300 import api, catalogs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
NSIDE, NG, BOX = 1024, 512, 2000.0


@pytest.fixture(scope="module")
def big():
    cfg = api.Config(ng=NG, box=BOX, order=4, interlace=True, prec="fp32")
    pos = catalogs.zeldovich_torch(NSIDE, BOX, 4.0, seed=3, device=DEV)
    cells = api.prepare(pos, cfg)
    del pos
    torch.cuda.empty_cache()
    g1, g2 = api.assign(cells, cfg)
    yield cfg, cells, g1, g2
    del cells, g1, g2
    torch.cuda.empty_cache()


def _near(cells, node, ng):
    """Records of the particles whose cell lies within 2 cells below / 3 above a node on every axis
    (a superset of those inside the PCS support on either grid)."""
    c = cells[:, 0]
    keep = None
    for axis, shift in ((0, 20), (1, 10), (2, 0)):
        d = torch.remainder(node[axis] - ((c >> shift) & 1023), ng)
        m = (d <= 3) | (d >= ng - 2)
        keep = m if keep is None else keep & m
    return cells[keep].cpu().numpy()


def test_fullsize_mass_and_sampled_nodes(big):
    cfg, cells, g1, g2 = big
    n = cells.shape[0]
    for g in (g1, g2):  # partition of unity: every unit weight lands on the grid
        assert abs(float(g.sum(dtype=torch.float64)) - n) <= 1e-6 * n
    rng = np.random.default_rng(81)
    nodes = [tuple(int(v) for v in rng.integers(0, NG, 3)) for _ in range(12)] + [(0, 0, 0), (NG - 1, 0, NG - 1)]
    scale = float(torch.max(g1))
    for node in nodes:
        u = _ref.cellpos_to_units(_near(cells, node, NG), NG)
        for g, shift in ((g1, False), (g2, True)):
            ref = oracle.assign.node_value(u, NG, 4, node, shift=shift)
            assert abs(float(g[node]) - ref) <= 2e-6 * scale, (node, shift)


def test_fullsize_modes_and_power_from_the_gpu_grids(big):
    cfg, cells, g1, g2 = big
    n = cells.shape[0]
    r1 = g1.double().cpu().numpy()
    r2 = g2.double().cpu().numpy()
    delta = oracle.fourier.density_modes(r1, 4, r2)
    # FFT, window division and interlacing on the GPU from the same grids
    d = api.fft_estimate(g1, g2, cfg, float(n)).cpu().numpy()
    ref = _ref.half_complex(delta)
    # FP32 transforms of the mass grid carry an absolute error of a few FP32 ulps of its mean (the
    # n = 0 term, 1 in these units) on every mode, which the window division then enlarges: compare
    # before that division, W(n) |delta_GPU - delta|, with 20 ulps (measured: 2.1e-8, 0.2 ulp)
    w = _ref.half_complex(oracle.fourier.window_3d(4, NG))
    err = np.abs(d - ref) * w
    assert err.max() <= 20 * np.finfo(np.float32).eps
    # the benchmark's call: P(k) of the binned catalogue (its own assignment, summed in another order)
    ref_pk, ref_k, ref_cnt = oracle.power.power_spectrum(delta, BOX)
    pk, km, cnt = api.power_binned(api.bin_particles(cells, cfg), cfg)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert _ref.rel(pk.cpu().numpy(), ref_pk) <= 1e-5  # measured: 3.1e-7 at most, 2.8e-7 typical
    assert _ref.rel(km.cpu().numpy(), ref_k) <= 1e-6


def test_fullsize_fp32_error_per_bin_against_fp64_positions(big):
    # The benchmark's FP32 P(k) (cell + FP32 offset records, FP32 grids and transforms) against FP64
    # from the FP64 positions (FP64 grids and transforms, the mode that matches the oracle at 1e-10):
    # the whole FP32 path's error, positions and assignment included, bin by bin, within the FP32 bar.
    cfg, cells, g1, g2 = big
    pk32, _, n32 = api.power_binned(api.bin_particles(cells, cfg), cfg)
    pos = catalogs.zeldovich_torch(NSIDE, BOX, 4.0, seed=3, device=DEV)
    pk64, _, n64 = api.power(pos, api.Config(ng=NG, box=BOX, order=4, interlace=True, prec="fp64"))
    del pos
    torch.cuda.empty_cache()
    assert torch.equal(n32, n64)
    rel = np.abs(pk32.cpu().numpy() / pk64.cpu().numpy() - 1.0)
    assert rel.max() <= 1e-5, rel.max()
