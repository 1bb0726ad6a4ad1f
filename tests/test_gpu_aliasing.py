"""GPU parity of the residual aliasing factor F_res (eq:res, pk_aliasing_residual) against the FP64
oracle: per-bin mean and maximum over the modes of the full grid, 1e-10 relative (both evaluate the
one-dimensional Hurwitz-zeta forms in FP64); mode counts bit-exact and equal to those of P(k)."""

import numpy as np
import pytest

import _ref
from oracle import aliasing, power
from paper_1512_07295_gb300 import api, ffi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ffi.lib()


@pytest.mark.parametrize("ng", [16, 36])
@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("interlace", [False, True])
def test_fres_bins_match_oracle(ng, order, interlace):
    cfg = api.Config(ng=ng, box=100.0, order=order, interlace=interlace, prec="fp64")
    mean, mx, km, cnt = (t.cpu().numpy() for t in api.aliasing_residual(cfg, "cuda:0"))
    ref_mean, ref_max, ref_cnt = aliasing.fres_binned(ng, order, interlace)
    assert np.array_equal(cnt, ref_cnt)
    assert _ref.rel(mean, ref_mean) <= 1e-10
    assert _ref.rel(mx, ref_max) <= 1e-10
    _, ref_k, pcnt = power.power_spectrum(np.ones((ng, ng, ng)), 100.0)
    assert np.array_equal(cnt, pcnt)
    assert _ref.rel(km, ref_k) <= 1e-12


def test_fres_custom_bins_and_interlacing_gain():
    # wide bins from 0 (the k = 0 mode excluded); interlacing lowers the residual in every bin
    cfg = api.Config(ng=64, box=100.0, order=4, interlace=False, prec="fp32", bin_lo2=0, bin_w2=8, nbins=8)
    edges = 8 * np.arange(9)
    m0, _, _, c0 = (t.cpu().numpy() for t in api.aliasing_residual(cfg, "cuda:0"))
    ref, _, rc = aliasing.fres_binned(64, 4, False, edges)
    assert np.array_equal(c0, rc)
    assert _ref.rel(m0, ref) <= 1e-10
    cfg.interlace = True
    m1, _, _, _ = (t.cpu().numpy() for t in api.aliasing_residual(cfg, "cuda:0"))
    assert np.all(m1 < m0)
