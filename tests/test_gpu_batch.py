"""GPU parity of the batched path (a9): every catalogue's P(k) equals the single-catalogue path and
the FP64 oracle."""

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
        # every catalogue against the FP64 oracle on the exact positions of its records
        u = _ref.cellpos_to_units(cells[offs[i]:offs[i + 1]].cpu().numpy(), ng)
        ref_pk, _, ref_cnt = _ref.power_units(u, box, ng, 4)
        assert np.array_equal(nm[i], ref_cnt)
        assert _ref.rel(pk[i], ref_pk) <= 1e-5, i


@pytest.mark.parametrize("run", [2, 4])
def test_batch_runs_of_tiles_match_oracle(run):
    box, ng = 300.0, 32
    sizes = [3000, 700, 12000, 5]
    cats = [catalogs.poisson(s, box, seed=400 + i) for i, s in enumerate(sizes)]
    cfg = api.Config(ng=ng, box=box, prec="fp32", tile_run=run)
    cells = torch.cat([api.prepare(_t(c), cfg) for c in cats])
    offs = np.concatenate([[0], np.cumsum(sizes)])
    pk, nm = api.batch_power(cells, offs, cfg, batch=3)
    for i in range(len(cats)):
        u = _ref.cellpos_to_units(cells[offs[i]:offs[i + 1]].cpu().numpy(), ng)
        ref_pk, _, ref_cnt = _ref.power_units(u, box, ng, 4)
        assert np.array_equal(nm[i].cpu().numpy(), ref_cnt)
        ok = ref_cnt > 0
        assert _ref.rel(pk[i].cpu().numpy()[ok], ref_pk[ok]) <= 1e-5, i


def test_batch_with_empty_catalogue():
    box, ng = 100.0, 16
    cfg = api.Config(ng=ng, box=box, prec="fp32")
    a = api.prepare(_t(catalogs.poisson(500, box, seed=72)), cfg)
    offs = np.array([0, 500, 500, 500])
    pk, nm = api.batch_power(a, offs, cfg, batch=3)
    single, _, _ = api.power(a, cfg)
    assert _ref.rel(pk[0].cpu().numpy(), single.cpu().numpy()) <= 1e-6
    assert torch.all(nm[1] == nm[0])


def test_batch_call_replays_from_a_cuda_graph():
    # the whole pk_batch_power call (several groups) captured once and replayed: same results, no
    # host synchronisation inside
    box, ng = 200.0, 32
    sizes = catalogs.batch_sizes(6, 500, 8000, seed=73)
    cats = [catalogs.poisson(s, box, seed=300 + i) for i, s in enumerate(sizes)]
    cfg = api.Config(ng=ng, box=box, prec="fp32")
    cells = torch.cat([api.prepare(_t(c), cfg) for c in cats])
    offs = np.concatenate([[0], np.cumsum(sizes)])
    ws = api.batch_workspace(cfg, 4, api.max_group_particles(offs, 4), cells.device)
    pk = torch.empty((len(sizes), cfg.nb), dtype=torch.float64, device=DEV)
    nm = torch.empty((len(sizes), cfg.nb), dtype=torch.int64, device=DEV)
    api.batch_power(cells, offs, cfg, batch=4, ws=ws, out=(pk, nm))  # eager call: plans and attributes
    torch.cuda.synchronize()
    ref_pk, ref_nm = pk.clone(), nm.clone()
    pk.zero_()
    nm.zero_()
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            api.batch_power(cells, offs, cfg, batch=4, ws=ws, out=(pk, nm))
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(nm, ref_nm)
    assert _ref.rel(pk.cpu().numpy(), ref_pk.cpu().numpy()) <= 1e-6


def test_autotuned_group_size_gives_the_same_spectra():
    box, ng = 200.0, 32
    sizes = catalogs.batch_sizes(9, 500, 8000, seed=74)
    cats = [catalogs.poisson(s, box, seed=400 + i) for i, s in enumerate(sizes)]
    cfg = api.Config(ng=ng, box=box, prec="fp32")
    cells = torch.cat([api.prepare(_t(c), cfg) for c in cats])
    offs = np.concatenate([[0], np.cumsum(sizes)])
    best, times = api.autotune_batch(cells, offs, cfg, candidates=(2, 4, 8), reps=2)
    assert best in (2, 4, 8) and set(times) == {2, 4, 8}
    a, na = api.batch_power(cells, offs, cfg, batch=best)
    b, nb = api.batch_power(cells, offs, cfg, batch=3)
    assert torch.equal(na, nb)
    assert _ref.rel(a.cpu().numpy(), b.cpu().numpy()) <= 1e-6


def test_one_group_of_the_largest_size():
    # 600 catalogues of 50 .. 3000 particles in groups of 512 (the largest): the tile kernels take the
    # runs of all 512 catalogues of the first group as one sequence; every spectrum equals the
    # single-catalogue path, and a sample of them the FP64 oracle
    box, ng = 200.0, 16
    sizes = catalogs.batch_sizes(600, 50, 3000, seed=72)
    cats = [catalogs.poisson(int(s), box, seed=300 + i) for i, s in enumerate(sizes)]
    cfg = api.Config(ng=ng, box=box, prec="fp32")
    cells = torch.cat([api.prepare(_t(c), cfg) for c in cats])
    offs = np.concatenate([[0], np.cumsum([len(c) for c in cats])])
    pk, nm = api.batch_power(cells, offs, cfg, batch=512)
    pk, nm = pk.cpu().numpy(), nm.cpu().numpy()
    for i in range(len(cats)):
        single, _, cnt = api.power(cells[offs[i]:offs[i + 1]].contiguous(), cfg)
        assert np.array_equal(nm[i], cnt.cpu().numpy())
        assert _ref.rel(pk[i], single.cpu().numpy()) <= 1e-6, i
    for i in (0, 255, 511, 512, 599):
        u = _ref.cellpos_to_units(cells[offs[i]:offs[i + 1]].cpu().numpy(), ng)
        ref_pk, _, ref_cnt = _ref.power_units(u, box, ng, 4)
        assert np.array_equal(nm[i], ref_cnt)
        assert _ref.rel(pk[i], ref_pk) <= 1e-5, i
