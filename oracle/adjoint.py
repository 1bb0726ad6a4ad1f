"""Analytic gradient of a loss on the binned power spectrum with respect to particle positions.

Test infrastructure (see ``oracle/__init__``); never imported by the product path.

The paper has no adjoint; this is the chain rule through the forward steps of ``assign``,
``fourier`` and ``power`` written out plainly:

  P_b = (V/M_b) sum_{n in b} |delta(n)|^2,    delta(n) = [d_1(n) + e^{i pi sum n/N} d_2(n)] / (2 W(n))
  d_g(n) = (1/N_c) sum_j (rho_g[j]/rhobar - 1) e^{-2 pi i n.j/N},   rhobar = sum_i w_i / N_c
  rho_g[j] = sum_i w_i prod_axis W^(p)(j_axis - u_i,axis - shift_g),   u = x/H, shift_1 = 0, shift_2 = 1/2

(without interlacing delta = d_1/W). rhobar does not depend on the positions (mass conservation), so

  dL/drho_1[j] = Re sum_n A(n) e^{-2 pi i n.j/N},   dL/drho_2[j] = Re sum_n A(n) e^{i pi sum n/N} e^{-2 pi i n.j/N}
  A(n) = (dL/dP_b) (V/M_b) 2 a conj(delta(n)) / (W(n) sum_i w_i),   a = 1/2 interlaced, 1 otherwise,

and dL/dx_{i,a} = w_i sum_g sum_j dL/drho_g[j] (-1/H) W'(s_a) prod_{c != a} W(s_c), s = j - u_i - shift_g.
"""

import numpy as np

from .assign import assign_units, grid_units
from .bspline import dweight, weight
from .fourier import density_modes, interlace_phase, window_3d
from .power import bin_index, default_edges


def grid_gradient(pos, box, ng, p, dl_dpk, interlace=True, weights=None, edges=None):
    """dL/drho_g on the grid(s) for dL/dP_b given per bin. Returns (g1, g2 or None)."""
    u = grid_units(pos, box, ng)
    rho1 = assign_units(u, ng, p, weights)
    rho2 = assign_units(u, ng, p, weights, shift=True) if interlace else None
    delta = density_modes(rho1, p, rho2)
    if edges is None:
        edges = default_edges(ng)
    b = bin_index(ng, edges)
    cnt = np.bincount(b[b >= 0], minlength=len(edges) - 1)
    dl = np.asarray(dl_dpk, dtype=np.float64)
    coef = np.zeros(delta.shape)
    sel = b >= 0
    coef[sel] = dl[b[sel]] * float(box) ** 3 / cnt[b[sel]]
    wsum = float(len(u)) if weights is None else float(np.sum(weights))
    a = 0.5 if interlace else 1.0
    amp = coef * 2.0 * a * np.conj(delta) / (window_3d(p, ng) * wsum)
    g1 = np.real(np.fft.fftn(amp))
    g2 = np.real(np.fft.fftn(amp * interlace_phase(ng))) if interlace else None
    return g1, g2


def _gather(u, g, p, shift, ng, weights):
    """sum_j g[j] dW/du over the stencil of each particle (per axis), in grid units."""
    n = u.shape[0]
    out = np.zeros((n, 3))
    uu = u + (0.5 if shift else 0.0)
    offs = np.arange(p + 1)
    j = np.ceil(uu - 0.5 * p).astype(np.int64)[:, :, None] + offs[None, None, :]
    s = j - uu[:, :, None]
    w = weight(p, s)
    dw = -dweight(p, s)  # d/du of W(j - u)
    jm = np.mod(j, ng)
    gv = g[jm[:, 0, :, None, None], jm[:, 1, None, :, None], jm[:, 2, None, None, :]]
    out[:, 0] = np.einsum("nabc,na,nb,nc->n", gv, dw[:, 0], w[:, 1], w[:, 2])
    out[:, 1] = np.einsum("nabc,na,nb,nc->n", gv, w[:, 0], dw[:, 1], w[:, 2])
    out[:, 2] = np.einsum("nabc,na,nb,nc->n", gv, w[:, 0], w[:, 1], dw[:, 2])
    if weights is not None:
        out *= np.asarray(weights, dtype=np.float64)[:, None]
    return out


def position_gradient(pos, box, ng, p, dl_dpk, interlace=True, weights=None, edges=None):
    """dL/dx (N_P x 3, length units) for a loss L(P_b) with the given dL/dP_b."""
    g1, g2 = grid_gradient(pos, box, ng, p, dl_dpk, interlace, weights, edges)
    u = grid_units(pos, box, ng)
    grad = _gather(u, g1, p, False, ng, weights)
    if interlace:
        grad += _gather(u, g2, p, True, ng, weights)
    return grad * (ng / float(box))
