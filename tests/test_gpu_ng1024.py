"""The N_G = 1024 transform path: two 1024^3 grids hold more than 2^31 padded reals, so their R2C runs
as one call per grid. delta(n) from pk_fft_estimate is compared on sampled modes with an FP64
transform of the same grids (torch.fft.rfftn) combined by eq:intdelta and eq:windowcorrection."""

import numpy as np
import pytest
import torch

from paper_1512_07295_gb300 import api

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _signed(i, n):
    return i if i < n // 2 else i - n


@pytest.mark.parametrize("order", [4])
def test_fft_estimate_at_ng1024_matches_fp64_transform(order):
    ng, box = 1024, 1000.0
    cfg = api.Config(ng=ng, box=box, order=order, interlace=True, prec="fp32")
    gen = torch.Generator(device=DEV)
    gen.manual_seed(97)
    g1 = torch.rand((ng, ng, ng), generator=gen, device=DEV, dtype=torch.float32)
    g2 = torch.rand((ng, ng, ng), generator=gen, device=DEV, dtype=torch.float32)
    wsum = float(ng) ** 3 * 0.5
    delta = api.fft_estimate(g1, g2, cfg, wsum)
    rng = np.random.default_rng(98)
    idx = [tuple(int(v) for v in rng.integers(0, [ng, ng, ng // 2], 3)) for _ in range(400)]
    idx = [t for t in idx if ng // 2 not in (t[0], t[1]) and t != (0, 0, 0)]
    ii = [torch.tensor([t[a] for t in idx], device=DEV) for a in range(3)]
    got = delta[ii[0], ii[1], ii[2]].cpu().numpy()
    del delta
    f = []
    for g in (g1, g2):
        F = torch.fft.rfftn(g.double())
        f.append(F[ii[0], ii[1], ii[2]].cpu().numpy())
        del F
        torch.cuda.empty_cache()
    for k, t in enumerate(idx):
        n = np.array([_signed(t[0], ng), _signed(t[1], ng), t[2]], dtype=np.float64)
        w = np.prod(np.sinc(n / ng) ** order)
        phase = np.exp(1j * np.pi * n.sum() / ng)
        ref = (f[0][k] + phase * f[1][k]) / (2.0 * wsum * w)
        assert abs(got[k] - ref) <= 1e-5 * max(abs(ref), 1e-3), (t, got[k], ref)
