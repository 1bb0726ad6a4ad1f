"""GPU parity of the batched path (a9): each catalogue's P(k) equals the single-catalogue path and
the oracle."""

import numpy as np
import pytest
import torch

import _ref
from paper_1512_07295_gb300 import api, catalogs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_batch_matches_single_and_oracle():
    box, ng = 300.0, 32
    sizes = catalogs.batch_sizes(11, 200, 20000, seed=71)
    cats = [catalogs.poisson(s, box, seed=100 + i) if i % 2 == 0 else
            catalogs.zeldovich(int(np.ceil(s ** (1 / 3))), box, rms=5.0, seed=200 + i)[:s] for i, s in enumerate(sizes)]
    cfg = api.Config(ng=ng, box=box, prec="fp32")
    cells = torch.cat([api.prepare(_t(c), cfg) for c in cats])
    offs = np.concatenate([[0], np.cumsum([len(c) for c in cats])])
    pk, nm = api.batch_power(cells, offs, cfg, batch=4)  # 3 groups, the last one partial
    pk, nm = pk.cpu().numpy(), nm.cpu().numpy()
    for i, c in enumerate(cats):
        single, _, cnt = api.power(cells[offs[i]:offs[i + 1]].contiguous(), cfg)
        assert np.array_equal(nm[i], cnt.cpu().numpy())
        assert _ref.rel(pk[i], single.cpu().numpy()) <= 1e-6
    u = _ref.cellpos_to_units(cells[offs[3]:offs[4]].cpu().numpy(), ng)
    ref_pk, _, _ = _ref.power_units(u, box, ng, 4)
    assert _ref.rel(pk[3], ref_pk) <= 1e-5


def test_batch_with_empty_catalogue():
    box, ng = 100.0, 16
    cfg = api.Config(ng=ng, box=box, prec="fp32")
    a = api.prepare(_t(catalogs.poisson(500, box, seed=72)), cfg)
    offs = np.array([0, 500, 500, 500])
    pk, nm = api.batch_power(a, offs, cfg, batch=3)
    single, _, _ = api.power(a, cfg)
    assert _ref.rel(pk[0].cpu().numpy(), single.cpu().numpy()) <= 1e-6
    assert torch.all(nm[1] == nm[0])
