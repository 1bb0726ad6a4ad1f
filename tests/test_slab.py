"""The x-slab decomposition of one catalogue over several ranks (paper_1512_07295_gb300.slab), on CPU
gloo ranks: each rank assigns its particles (deterministic 64-bit fixed point, as PK_FIXED64) into its
slab plus halo, exchanges the halo planes with its neighbours, transforms its planes over (y, z),
transposes to k_y slabs, completes the transform over x, bins its modes and all-reduces the bin partials.
The shard grids must equal the single-rank grid bit for bit (int64), and P(k) the FP64 oracle's."""

import math
import os
import socket

import numpy as np
import pytest
import torch

import oracle
from paper_1512_07295_gb300 import catalogs, slab


# --- decomposition facts, no processes --------------------------------------------------------------

@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_reach_covers_every_node_the_oracle_assigns(p):
    # every node the oracle's assignment gives weight to, on grid 1 and grid 2, lies in c - lo .. c + hi
    ng = 16
    lo, hi = slab.reach(p)
    u = np.random.default_rng(p).uniform(0.0, ng, (3000, 1))
    u = np.concatenate([u, np.full((3000, 2), 8.3)], axis=1)
    u[:4, 0] = [0.0, 0.5, 0.9999999, 7.5]
    for shift in (False, True):
        for i in range(0, len(u), 600):
            rho = oracle.assign.assign_units(u[i:i + 1], ng, p, shift=shift)
            xs = np.nonzero(rho.sum(axis=(1, 2)))[0]
            c = int(np.floor(u[i, 0]))
            d = (xs - c + ng // 2) % ng - ng // 2
            assert d.min() >= -lo and d.max() <= hi, (p, shift, u[i, 0], d)
    # and the bound is attained on some grid (no wasted halo plane)
    assert lo + hi == p


def test_slab_bounds_and_ownership():
    assert slab.slab_bounds(10, 3) == [(0, 3), (3, 6), (6, 10)]
    r = slab.particle_ranks([0, 2, 3, 9, 5], 10, 3)
    assert r.tolist() == [0, 0, 1, 2, 1]
    with pytest.raises(ValueError):
        slab.SlabPlan(16, 8, 0, 4).check()  # slabs of 2 planes, halo (1, 3)


@pytest.mark.parametrize("world", [1, 3])
def test_halo_messages_route_to_the_owning_planes(world):
    # in-process routing of every rank's halo messages: a buffer whose planes carry their global x index
    ng, p = 12, 4
    plans = [slab.SlabPlan(ng, world, r, p).check() for r in range(world)]
    locs = [torch.as_tensor(pl.local_planes(), dtype=torch.int64)[:, None, None].expand(-1, 2, 2).clone()
            for pl in plans]
    msgs = {r: slab.halo_messages(locs[r], plans[r]) for r in range(world)}
    total = torch.zeros(ng, dtype=torch.int64)
    for r, pl in enumerate(plans):
        above = [t for rr in range(world) for dst, tag, t in msgs[rr] if dst == r and tag == slab.TAG_LOW and rr == (r + 1) % world][0]
        below = [t for rr in range(world) for dst, tag, t in msgs[rr] if dst == r and tag == slab.TAG_HIGH and rr == (r - 1) % world][0]
        own = slab.owned_with_halos(locs[r], pl, above, below)
        total[pl.x0:pl.x1] += own[:, 0, 0]
    # each plane x receives its own copy plus one copy from every rank whose halo reaches it: x itself
    # counted (1 + number of halo copies) times, all carrying the value x
    mult = np.zeros(ng, dtype=np.int64)
    for pl in plans:
        np.add.at(mult, pl.local_planes(), 1)
    mult = torch.from_numpy(mult)
    assert torch.equal(total, torch.arange(ng) * mult)


# --- the per-rank arithmetic of the test (plain NumPy, FP64 / int64) ----------------------------------

def _fixed_scale(wabs_total):
    return 62 - math.ceil(math.log2(max(wabs_total, 1.0)))


def _assign_fixed(u, w, ng, p, shift, F, plane0, nplanes):
    """int64 grid [nplanes, N, N] of the particles u (grid units): every contribution w W_x W_y W_z at the
    nodes within the kernel support, rounded to an integer at scale 2^F (the rule of PK_FIXED64), at
    plane (x - plane0) mod N."""
    out = np.zeros((nplanes, ng, ng), dtype=np.int64)
    uu = u + (0.5 if shift else 0.0)
    offs = np.arange(p + 1)
    j = np.ceil(uu - 0.5 * p).astype(np.int64)[:, :, None] + offs
    wt = oracle.bspline.weight(p, j - uu[:, :, None])
    jm = np.mod(j, ng)
    xi = (jm[:, 0, :] - plane0) % ng
    val = w[:, None, None, None] * wt[:, 0, :, None, None] * wt[:, 1, None, :, None] * wt[:, 2, None, None, :]
    q = np.rint(val * 2.0 ** F).astype(np.int64)
    xs = np.broadcast_to(xi[:, :, None, None], q.shape)
    ys = np.broadcast_to(jm[:, 1, None, :, None], q.shape)
    zs = np.broadcast_to(jm[:, 2, None, None, :], q.shape)
    keep = (q != 0)
    assert np.all(xs[keep] < nplanes), "a contribution outside the rank's planes"
    np.add.at(out, (xs[keep], ys[keep], zs[keep]), q[keep])
    return out


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, box, ng, p, seed, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pos = catalogs.zeldovich(12, box, rms=3.0, seed=seed)
        w = catalogs.random_weights(len(pos), seed=seed + 1)
        u = oracle.assign.grid_units(pos, box, ng)
        cx = np.floor(u[:, 0]).astype(np.int64) % ng
        plan = slab.SlabPlan(ng, world, rank, p).check()
        mine = slab.particle_ranks(cx, ng, world) == rank
        comm = slab.TorchComm()
        wabs = comm.all_reduce(torch.tensor([np.abs(w[mine]).sum()], dtype=torch.float64))
        F = _fixed_scale(float(wabs[0]))
        lo, _ = plan.halo
        nloc = plan.width + sum(plan.halo)

        def assign_local(pl):
            g = [_assign_fixed(u[mine], w[mine], ng, p, s, F, pl.x0 - lo, nloc) for s in (False, True)]
            return torch.from_numpy(np.stack(g))

        nc = ng ** 3

        def transform_yz(own, wsum):
            rho = own.numpy().astype(np.float64) / 2.0 ** F
            delta = rho / (wsum / nc) - 1.0
            return torch.from_numpy(np.fft.fft2(delta, axes=(-2, -1)))

        def transform_x(yslab):
            return torch.from_numpy(np.fft.fft(yslab.numpy(), axis=-3) / nc)

        def partials(modes, pl, wsum, w2sum):
            y0, y1 = pl.bounds[pl.rank]
            g = modes.numpy()
            phase = oracle.fourier.interlace_phase(ng)[:, y0:y1, :]
            win = oracle.fourier.window_3d(p, ng)[:, y0:y1, :]
            delta = 0.5 * (g[0] + phase * g[1]) / win
            b = oracle.power.bin_index(ng, oracle.power.default_edges(ng))[:, y0:y1, :].ravel()
            sel = b >= 0
            kf = 2.0 * np.pi / box
            kmag = kf * np.sqrt(oracle.power.mode_norm2_x4(ng)[:, y0:y1, :].ravel()[sel] / 4.0)
            nb = ng // 2
            out = np.stack([np.bincount(b[sel], weights=box ** 3 * np.abs(delta.ravel()[sel]) ** 2, minlength=nb),
                            np.bincount(b[sel], weights=kmag, minlength=nb),
                            np.bincount(b[sel], minlength=nb).astype(np.float64)])
            return torch.from_numpy(out)

        ws = torch.tensor([w[mine].sum(), (w[mine] ** 2).sum()], dtype=torch.float64)
        pk, km, cnt = slab.slab_power(cx[mine], plan, comm, assign_local, transform_yz, transform_x, partials, ws)
        # shard grid: this rank's own planes after the halo exchange, against the single-rank grid
        own = slab.exchange_halos(assign_local(plan), plan, comm).numpy()
        full = np.stack([_assign_fixed(u, w, ng, p, s, F, 0, ng) for s in (False, True)])
        own_ok = bool(np.array_equal(own, full[:, plan.x0:plan.x1]))
        q.put((rank, own_ok, pk.numpy(), km.numpy(), cnt.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("p", [2, 4])
def test_slab_split_over_gloo_ranks(world, p):
    import torch.multiprocessing as mp

    box, ng, seed = 60.0, 16, 31
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, box, ng, p, seed, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    pos = catalogs.zeldovich(12, box, rms=3.0, seed=seed)
    w = catalogs.random_weights(len(pos), seed=seed + 1)
    r1 = oracle.assign.assign(pos, box, ng, p, weights=w)
    r2 = oracle.assign.assign(pos, box, ng, p, weights=w, shift=True)
    ref_pk, ref_k, ref_cnt = oracle.power.power_spectrum(oracle.fourier.density_modes(r1, p, r2), box)
    for rank, own_ok, pk, km, cnt in res:
        assert own_ok, f"rank {rank}: shard planes differ from the single-rank int64 grid"
        assert np.array_equal(cnt, ref_cnt)
        assert np.max(np.abs(pk / ref_pk - 1.0)) < 1e-10
        assert np.max(np.abs(km / ref_k - 1.0)) < 1e-12
