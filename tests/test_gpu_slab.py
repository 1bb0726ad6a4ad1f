"""The x-slab decomposition with the library's own assignment on every rank, simulated in one process
on one GPU: each rank's particles go through pk_assign (FP64 and the deterministic FIXED64 mode) into
grids of their own, the rank keeps its slab plus halo planes (the only non-zero ones), and the halo
planes are routed to their owners by the same message functions the distributed driver uses. The
owned planes of all ranks must assemble the single-call grids (FP64: to rounding; FIXED64: the scale
is set by the rank's own weights, so to the fixed-point step)."""

import numpy as np
import pytest
import torch

from paper_1512_07295_gb300 import api, catalogs, slab

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("prec", ["fp64", "fixed64"])
@pytest.mark.parametrize("order", [2, 3, 4])
def test_slab_shards_assemble_the_whole_grid(world, prec, order):
    box, ng = 80.0, 32
    pos = catalogs.zeldovich(24, box, rms=3.0, seed=41)
    w = catalogs.random_weights(len(pos), seed=42).astype(np.float32)
    cfg = api.Config(ng=ng, box=box, order=order, prec=prec)
    full = torch.stack(api.assign(torch.from_numpy(pos).to(DEV), cfg, weights=torch.from_numpy(w).to(DEV)))
    cx = np.floor(np.mod(pos[:, 0], box) * ng / box).astype(np.int64) % ng
    owner = slab.particle_ranks(cx, ng, world)
    plans = [slab.SlabPlan(ng, world, r, order).check() for r in range(world)]
    local, msgs = [], []
    for r, pl in enumerate(plans):
        sel = owner == r
        g = torch.stack(api.assign(torch.from_numpy(pos[sel]).to(DEV), cfg, weights=torch.from_numpy(w[sel]).to(DEV)))
        loc = slab.local_from_full(g, pl)
        # every plane outside the rank's slab and halo is empty
        keep = torch.zeros(ng, dtype=torch.bool)
        keep[torch.as_tensor(pl.local_planes())] = True
        assert torch.count_nonzero(g[:, ~keep.to(DEV)]) == 0
        local.append(loc)
        msgs.append(slab.halo_messages(loc, pl))
    out = torch.empty_like(full)
    for r, pl in enumerate(plans):
        above = [t for dst, tag, t in msgs[(r + 1) % world] if dst == r and tag == slab.TAG_LOW][0]
        below = [t for dst, tag, t in msgs[(r - 1) % world] if dst == r and tag == slab.TAG_HIGH][0]
        out[:, pl.x0:pl.x1] = slab.owned_with_halos(local[r], pl, above, below)
    scale = torch.max(torch.abs(full)).item()
    tol = 1e-12 if prec == "fp64" else 1e-9
    assert torch.max(torch.abs(out - full)).item() <= tol * scale
