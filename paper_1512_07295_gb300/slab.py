"""One catalogue split across ranks by x-slab: the multi-GPU decomposition of the estimator path.

The mass assignment (eq:delgrid, Sec. 2.3) is a sum over particles, so the grids of a catalogue are the
sums of the grids of any partition of its particles. Rank r owns the x-planes [x0_r, x1_r) of both grids
and the particles whose cell lies in them. Such a particle reaches the planes c - lo .. c + hi of either
grid (``reach``), so a rank assigns its particles into its slab plus lo planes below and hi planes above,
and sends each halo plane to the rank that owns it, which adds it (one point-to-point message to each
neighbour). The transform is slab-decomposed: each rank transforms its own planes over (y, z), a
transpose (an all-to-all built from point-to-point messages) gives every rank all x planes of its range
of k_y, and the transform over x completes the modes. The fused estimate (window division, interlacing
phase, binning: Sec. 2.2, eq:windowcorrection, eq:intdelta) then covers the rank's modes, and an
all-reduce of the FP64 bin partials (sum of V|delta|^2, sum of |k|, count) gives P(k) on every rank.

This module holds the decomposition: slab bounds, particle ownership, the halo messages and their
addition, the transpose and the reductions, over a communicator with point-to-point messages and a sum
all-reduce (``TorchComm``: torch.distributed, gloo on CPU ranks, NCCL between GPUs). The per-rank
arithmetic (assignment into the local planes, the transforms, the estimate of a range of modes) is passed
in by the caller: on GPUs it is the library's kernels, one GPU per rank.
"""

from dataclasses import dataclass

import numpy as np
import torch

TAG_LOW, TAG_HIGH, TAG_T = 11, 12, 20


def slab_bounds(ng, world):
    """[x0, x1) of the planes owned by each rank: ng planes in world slabs of near-equal thickness."""
    if world < 1 or world > ng:
        raise ValueError(f"world size {world} must be in 1 .. N ({ng})")
    edges = [(r * ng) // world for r in range(world + 1)]
    return [(edges[r], edges[r + 1]) for r in range(world)]


def reach(order):
    """Planes (lo, hi) below and above its cell c = floor(u_x) that a particle reaches on either grid.

    Grid 1 (Sec. 2.3): even p takes nodes c - p/2 + 1 .. c + p/2, odd p the nearest node m in {c, c + 1}
    and (p - 1)/2 on each side. Grid 2 (Sec. 3.1) samples u + 1/2, whose cell (even p) or nearest node
    (odd p) is at most one above; so lo = p/2 - 1, hi = p/2 + 1 for even p and lo = (p - 1)/2,
    hi = (p + 1)/2 for odd p."""
    if order < 1:
        raise ValueError("order must be >= 1")
    if order % 2 == 0:
        return order // 2 - 1, order // 2 + 1
    return (order - 1) // 2, (order + 1) // 2


@dataclass(frozen=True)
class SlabPlan:
    ng: int
    world: int
    rank: int
    order: int

    @property
    def bounds(self):
        return slab_bounds(self.ng, self.world)

    @property
    def x0(self):
        return self.bounds[self.rank][0]

    @property
    def x1(self):
        return self.bounds[self.rank][1]

    @property
    def width(self):
        return self.x1 - self.x0

    @property
    def halo(self):
        return reach(self.order)

    def local_planes(self):
        """Global x index of each plane of the rank's local buffer: x0 - lo .. x1 + hi - 1 (periodic)."""
        lo, hi = self.halo
        return np.arange(self.x0 - lo, self.x1 + hi) % self.ng

    def check(self):
        """The halo of a rank must fall on its two neighbours only: every slab at least as thick as the
        halo on either side (world 1 wraps onto itself)."""
        lo, hi = self.halo
        thin = min(x1 - x0 for x0, x1 in self.bounds)
        if self.world > 1 and thin < max(lo, hi):
            raise ValueError(f"slabs of {thin} planes are thinner than the halo ({lo}, {hi}) of order {self.order}")
        return self


def particle_ranks(cell_x, ng, world):
    """Owning rank of each particle: the rank whose planes hold its cell (cell_x in 0 .. N - 1)."""
    owner = np.empty(ng, dtype=np.int64)
    for r, (x0, x1) in enumerate(slab_bounds(ng, world)):
        owner[x0:x1] = r
    return owner[np.asarray(cell_x, dtype=np.int64)]


def halo_messages(local, plan):
    """The planes a rank sends after assigning into its local buffer: (dst, tag, planes).

    local: tensor [..., lo + width + hi, ...] with the plane axis at dim -3 (grids, planes, y, z). The lo
    planes below the slab belong to the top of rank r - 1, the hi planes above it to the bottom of rank
    r + 1 (periodic)."""
    lo, hi = plan.halo
    w = plan.width
    low = local[..., :lo, :, :]
    high = local[..., lo + w:, :, :]
    return [((plan.rank - 1) % plan.world, TAG_LOW, low), ((plan.rank + 1) % plan.world, TAG_HIGH, high)]


def owned_with_halos(local, plan, from_above, from_below):
    """The rank's own planes plus the halo planes received: from_above is rank r + 1's low halo (added
    to the top lo planes), from_below rank r - 1's high halo (added to the bottom hi planes)."""
    lo, hi = plan.halo
    w = plan.width
    own = local[..., lo:lo + w, :, :].clone()
    if lo:
        own[..., w - lo:, :, :] += from_above
    if hi:
        own[..., :hi, :, :] += from_below
    return own


class TorchComm:
    """Point-to-point messages and sum all-reduce over torch.distributed (complex tensors travel as
    their real view)."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def exchange(self, sends, recvs):
        """sends: [(dst, tag, tensor)], recvs: [(src, tag, tensor to fill)]; all posted, then awaited."""
        d = self.dist
        ops = []
        for dst, tag, t in sends:
            ops.append(d.isend(_wire(t.contiguous()), dst, group=self.group, tag=tag))
        bufs = []
        for src, tag, t in recvs:
            w = torch.empty_like(_wire(t))
            bufs.append((t, w))
            ops.append(d.irecv(w, src, group=self.group, tag=tag))
        for op in ops:
            op.wait()
        for t, w in bufs:
            t.copy_(_unwire(w, t))

    def all_reduce(self, t):
        self.dist.all_reduce(t, group=self.group)
        return t


def _wire(t):
    return torch.view_as_real(t) if t.is_complex() else t


def _unwire(w, like):
    return torch.view_as_complex(w) if like.is_complex() else w


def exchange_halos(local, plan, comm):
    """Sends the rank's halo planes to its neighbours and returns its own planes with theirs added."""
    lo, hi = plan.halo
    if plan.world == 1:
        (_, _, low), (_, _, high) = halo_messages(local, plan)
        return owned_with_halos(local, plan, low, high)
    shape = list(local.shape)
    shape_lo, shape_hi = shape.copy(), shape.copy()
    shape_lo[-3], shape_hi[-3] = lo, hi
    from_above = torch.empty(shape_lo, dtype=local.dtype, device=local.device)
    from_below = torch.empty(shape_hi, dtype=local.dtype, device=local.device)
    sends = [(dst, tag, t) for dst, tag, t in halo_messages(local, plan) if t.shape[-3] > 0]
    recvs = []
    if lo:
        recvs.append(((plan.rank + 1) % plan.world, TAG_LOW, from_above))
    if hi:
        recvs.append(((plan.rank - 1) % plan.world, TAG_HIGH, from_below))
    comm.exchange(sends, recvs)
    return owned_with_halos(local, plan, from_above, from_below)


def transpose_to_y(planes, plan, comm):
    """x-slab -> y-slab: planes [..., width, N, nz] (the rank's x planes, all k_y) become
    [..., N, h, nz] (all x, the rank's range of k_y, same bounds as the x slabs)."""
    bounds = plan.bounds
    y0, y1 = bounds[plan.rank]
    lead = list(planes.shape[:-3])
    nz = planes.shape[-1]
    out = torch.empty(lead + [plan.ng, y1 - y0, nz], dtype=planes.dtype, device=planes.device)
    out[..., plan.x0:plan.x1, :, :] = planes[..., :, y0:y1, :]
    if plan.world == 1:
        return out
    sends, recvs, parts = [], [], []
    for j, (a, b) in enumerate(bounds):
        if j == plan.rank:
            continue
        sends.append((j, TAG_T + plan.rank, planes[..., :, a:b, :]))
        part = torch.empty(lead + [bounds[j][1] - bounds[j][0], y1 - y0, nz], dtype=planes.dtype, device=planes.device)
        recvs.append((j, TAG_T + j, part))
        parts.append((j, part))
    comm.exchange(sends, recvs)
    for j, part in parts:
        out[..., bounds[j][0]:bounds[j][1], :, :] = part
    return out


def slab_power(particles_cell_x, plan, comm, assign_local, transform_yz, transform_x, partials, weight_sums):
    """P(k) of a catalogue split by x-slab, on every rank.

    particles_cell_x: cell x index of the rank's particles (used to check ownership);
    assign_local(plan) -> local grids [ngrid, lo + width + hi, N, N] (the rank's particles);
    transform_yz(own, wsum) -> the rank's planes transformed over (y, z) [ngrid, width, N, nz];
    transform_x(yslab) -> all modes of the rank's k_y range [ngrid, N, h, nz];
    partials(modes, plan, wsum, w2sum) -> FP64 tensor [3, nbins] (sum V|delta|^2, sum |k|, count) over
    the rank's modes; weight_sums -> FP64 tensor [2] (sum w, sum w^2) of the rank's particles.
    Returns (P_b, k_eff_b, count_b) with NaN for empty bins, identical on every rank."""
    plan.check()
    owner = particle_ranks(particles_cell_x, plan.ng, plan.world)
    if owner.size and not np.all(owner == plan.rank):
        raise ValueError("every particle given to a rank must lie in its slab")
    ws = comm.all_reduce(weight_sums.clone())
    local = assign_local(plan)
    own = exchange_halos(local, plan, comm)
    yslab = transpose_to_y(transform_yz(own, float(ws[0])), plan, comm)
    modes = transform_x(yslab)
    part = comm.all_reduce(partials(modes, plan, float(ws[0]), float(ws[1])).clone())
    s, k, c = part[0], part[1], part[2]
    pk = torch.where(c > 0, s / torch.clamp(c, min=1.0), torch.full_like(s, float("nan")))
    kmean = torch.where(c > 0, k / torch.clamp(c, min=1.0), torch.full_like(k, float("nan")))
    return pk, kmean, torch.round(c).to(torch.int64)


def local_from_full(grids, plan):
    """The rank's local buffer cut from full periodic grids [..., N, N, N] (x slowest): the planes
    x0 - lo .. x1 + hi - 1. A rank that assigns its particles into a whole grid of its own (one GPU per
    rank, the library's assignment on the rank's particles) sends and keeps exactly these planes; every
    other plane of that grid is zero."""
    idx = torch.as_tensor(plan.local_planes(), device=grids.device)
    return torch.index_select(grids, grids.dim() - 3, idx)
