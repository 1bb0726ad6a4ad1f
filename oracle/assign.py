"""Mass assignment of particles to a periodic grid, eq:delgrid (Sec. 2.3) and the interlaced
second grid of Sec. 3.1.

Test infrastructure (see ``oracle/__init__``); never imported by the product path.

For particle i at x_i and grid node j (periodic, spacing H = L/N_G), the node receives
w_i * prod_axis W^(p)((x_j - x_i)/H). The sum over all particles of W is the interpolated density
of eq:delgrid up to the constant (2 pi)^3 nbar; this module returns the mass grid
rho_j = sum_i w_i W(x_j - x_i), whose sum equals sum_i w_i because the B-splines are a partition of
unity. The interlaced grid of Sec. 3.1 samples the field at the nodes shifted by H/2; it is built
here, equivalently, by shifting every particle by +H/2 on each axis onto the same nodes.
"""

import numpy as np

from .bspline import weight


def grid_units(pos, box, ng):
    """Positions in units of the grid spacing, wrapped into [0, N_G) (periodic box of side L)."""
    u = np.mod(np.asarray(pos, dtype=np.float64), box) * (ng / box)
    u[u >= ng] -= ng  # x equal to L (after rounding) wraps to 0
    return u


def assign_units(u, ng, p, weights=None, shift=False, chunk=1 << 16):
    """rho_j = sum_i w_i prod_axis W^(p)(j_axis - u_i,axis), eq:delgrid, u in grid units.

    Every node j whose distance to the particle lies inside the kernel support (|s| < p/2) is
    visited: the candidates on one axis are j = ceil(u - p/2) + a, a = 0..p, and the distance
    s = j - u is the minimum-image separation. shift=True adds 1/2 to u (grid 2 of Sec. 3.1); a
    3-vector adds that shift (grid units) per axis, for the grids of multi-grid interlacing.
    """
    u = np.asarray(u, dtype=np.float64)
    if isinstance(shift, (bool, np.bool_)):
        shift = 0.5 if shift else 0.0
    shift = np.broadcast_to(np.asarray(shift, dtype=np.float64), (3,))
    n = u.shape[0]
    w_all = np.ones(n) if weights is None else np.asarray(weights, dtype=np.float64)
    rho = np.zeros(ng * ng * ng)
    offs = np.arange(p + 1)
    for lo in range(0, n, chunk):
        uu = u[lo:lo + chunk] + shift[None, :]
        ww = w_all[lo:lo + chunk]
        j = np.ceil(uu - 0.5 * p).astype(np.int64)[:, :, None] + offs[None, None, :]  # (m,3,p+1)
        wt = weight(p, j - uu[:, :, None])                                              # (m,3,p+1)
        jm = np.mod(j, ng)
        idx = (jm[:, 0, :, None, None] * ng + jm[:, 1, None, :, None]) * ng + jm[:, 2, None, None, :]
        val = ww[:, None, None, None] * wt[:, 0, :, None, None] * wt[:, 1, None, :, None] * wt[:, 2, None, None, :]
        rho += np.bincount(idx.ravel(), weights=val.ravel(), minlength=ng ** 3)
    return rho.reshape(ng, ng, ng)


def assign(pos, box, ng, p, weights=None, shift=False):
    """Mass grid of eq:delgrid from positions in length units (see ``assign_units``)."""
    return assign_units(grid_units(pos, box, ng), ng, p, weights=weights, shift=shift)


def node_value(u, ng, p, node, weights=None, shift=False):
    """rho_j of eq:delgrid at one node j = (jx, jy, jz): sum_i w_i prod_axis W^(p)(s_axis), with s the
    minimum-image separation j - u_i (u + 1/2 for shift=True, grid 2 of Sec. 3.1). Particles outside
    the support contribute W = 0, so u may hold any subset that contains every particle near j."""
    u = np.asarray(u, dtype=np.float64) + (0.5 if shift else 0.0)
    w = np.ones(u.shape[0]) if weights is None else np.asarray(weights, dtype=np.float64)
    s = np.asarray(node, dtype=np.float64)[None, :] - u
    s -= ng * np.round(s / ng)  # minimum image
    return float(np.sum(w * weight(p, s[:, 0]) * weight(p, s[:, 1]) * weight(p, s[:, 2])))
