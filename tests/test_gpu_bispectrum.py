"""GPU parity of the FFT bispectrum (a7) and of its exact triangle counts against the oracle."""

import numpy as np
import pytest
import torch

import _ref
import oracle
from paper_1512_07295_gb300 import api, catalogs, ffi

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("ng,lo,w,ns", [(16, 1, 1, 4), (32, 0, 2, 5), (36, 1, 3, 3)])
def test_triangle_counts_exact(ng, lo, w, ns):
    cfg = api.Config(ng=ng, box=1.0)
    counts = api.bispectrum_counts(cfg, lo, w, ns, DEV).cpu().numpy()
    ref = oracle.bispectrum.triangle_counts(ng, lo, w, ns)
    assert np.array_equal(counts, ref)
    assert len(api.triangles(ns)) == len(ref) == api.bispectrum_ntri(ns)


def test_triangle_counts_brute_force_tiny():
    ng, lo, w, ns = 12, 1, 1, 3
    cfg = api.Config(ng=ng, box=1.0)
    counts = api.bispectrum_counts(cfg, lo, w, ns, DEV).cpu().numpy()
    _, brute = oracle.bispectrum.bispectrum_brute(np.ones((ng, ng, ng), dtype=complex), 1.0, lo, w, ns)
    assert np.array_equal(counts, brute)


# Up to 16 shells the FP32 triple product keeps the triangles in registers (16 shells: all 508 of them;
# 11 shells on N = 36: a prefix of the list, tiles of 128 points that cross rows, a ragged last tile)
# and the FP64 one takes warps over triangles; 23 shells (276 shell pairs) run the per-triangle kernel.
@pytest.mark.parametrize("ng,lo,w,ns", [(32, 1, 2, 5), (36, 0, 1, 11), (64, 1, 1, 16), (72, 1, 1, 23)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_bispectrum_matches_oracle(prec, tol, ng, lo, w, ns):
    box = 200.0
    pos = catalogs.zeldovich(32, box, rms=8.0, seed=51)
    _, _, _, delta = _ref.power(pos, box, ng, 4)
    ref_b, ref_c = oracle.bispectrum.bispectrum_fft(delta, box, lo, w, ns)
    cfg = api.Config(ng=ng, box=box, prec=prec)
    _, _, _, d = api.power(_t(pos), cfg, return_delta=True)
    b, c = api.bispectrum(d, cfg, lo, w, ns)
    b, c = b.cpu().numpy(), c.cpu().numpy()
    assert np.array_equal(c, ref_c)
    ok = ref_c > 0
    assert np.all(np.isnan(b[~ok]))
    # relative to the bin's own magnitude scale (B can cross zero): |dB| <= tol * max|B|
    assert np.max(np.abs(b[ok] - ref_b[ok])) <= tol * np.max(np.abs(ref_b[ok]))


def test_shell_limit_rejected():
    cfg = api.Config(ng=16, box=1.0)
    with pytest.raises(ffi.PkError):
        api.bispectrum_counts(cfg, 0, 2, 4, DEV)  # |n| up to 7: 3 * 7 >= 16
