"""GPU parity of the hand-written adjoint dP/dx (a8): against the FP64 oracle gradient, and the
oracle gradient against central finite differences (pinned in test_oracle_pins)."""

import numpy as np
import pytest
import torch

import oracle
from paper_1512_07295_gb300 import api, catalogs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("interlace", [False, True])
def test_backward_fp64_matches_oracle(order, interlace):
    box, ng = 100.0, 16
    pos = catalogs.zeldovich(12, box, rms=4.0, seed=61)
    dl = np.random.default_rng(62).standard_normal(ng // 2)
    ref = oracle.adjoint.position_gradient(pos, box, ng, order, dl, interlace=interlace)
    cfg = api.Config(ng=ng, box=box, order=order, interlace=interlace, prec="fp64")
    g = api.power_backward(_t(pos), cfg, _t(dl)).cpu().numpy()
    assert np.max(np.abs(g - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_backward_fp32_and_weights():
    box, ng = 120.0, 16
    pos = catalogs.poisson(3000, box, seed=63)
    w = catalogs.random_weights(3000, seed=64).astype(np.float32)
    dl = np.random.default_rng(65).standard_normal(ng // 2)
    ref = oracle.adjoint.position_gradient(pos, box, ng, 4, dl, weights=w.astype(np.float64))
    g = api.power_backward(_t(pos), api.Config(ng=ng, box=box, prec="fp32"), _t(dl), weights=_t(w)).cpu().numpy()
    assert np.max(np.abs(g - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_autograd_function_and_finite_differences():
    # loss = sum_b (P_b - T_b)^2 / sigma_b^2 with sigma_b^2 = 2 T_b^2 / M_b (Gaussian mode variance)
    box, ng = 100.0, 16
    pos = catalogs.zeldovich(12, box, rms=3.0, seed=66)
    cfg = api.Config(ng=ng, box=box, prec="fp64")
    x = _t(pos).requires_grad_(True)
    target, _, m = api.power(_t(catalogs.zeldovich(12, box, rms=3.0, seed=67)), cfg)
    sig2 = 2.0 * target ** 2 / m.to(torch.float64)

    def loss_of(xx):
        pk = api.power_spectrum(xx, cfg)
        return torch.sum((pk - target) ** 2 / sig2)

    loss = loss_of(x)
    loss.backward()
    g = x.grad.cpu().numpy()
    h = 1e-4
    for i in (0, 100, 1000):
        for a in range(3):
            xp = pos.copy(); xp[i, a] += h
            xm = pos.copy(); xm[i, a] -= h
            with torch.no_grad():
                fd = (loss_of(_t(xp)) - loss_of(_t(xm))).item() / (2 * h)
            assert abs(fd - g[i, a]) <= 1e-5 * max(1.0, np.max(np.abs(g)))
