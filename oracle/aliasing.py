"""Aliasing sums of Secs. 2.3 and 3.1 for B-spline windows.

Test infrastructure (see ``oracle/__init__``); never imported by the product path.

- ``shot_noise_expectation``: eq:Pknoint and its interlaced form with P = 0, i.e. the expected
  window-corrected power of a uniform random (Poisson) catalogue, the aliasing sum over images m of
  theta_m |W(k - m k_s)|^2 P_tot / |W(k)|^2 with P_tot = 1/nbar and theta_m = 1 (no interlacing) or
  [1 + (-1)^(m_x+m_y+m_z)]/2 (interlacing). With x = n/N_G, |W(k - m k_s)| = |sinc(pi (x - m))|^p.
- ``fres_1d`` / ``fres_1d_hurwitz``: the one-dimensional residual factor of eq:res1Di and
  eq:res1Dnoi as a truncated image sum and in its Hurwitz-zeta closed form.
- ``fres_3d``: the residual factor F_res(k) = sum_{m != 0} theta_m |w_m(k)|^2 of eq:res (reading:
  |w_m|, not |w_2m|) on three-dimensional modes, from the one-dimensional forms.
"""

import numpy as np
import scipy.special

from .bspline import sinc
from .fourier import signed_index
from .power import bin_index, default_edges


def _image_sums(x, p, mmax):
    """Per axis: sum_m sinc^{2p}(pi (x - m)) and sum_m (-1)^m sinc^{2p}(pi (x - m)), |m| <= mmax."""
    m = np.arange(-mmax, mmax + 1, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    t = sinc(np.pi * (x[:, None] - m[None, :])) ** (2 * p)
    sgn = np.where(np.abs(m) % 2 == 0, 1.0, -1.0)
    return t.sum(axis=1), (t * sgn[None, :]).sum(axis=1)


def _parities(interlace, shifts):
    """Per grid and axis, whether the shift is an odd number of half cells (None: 1 or 2 grids)."""
    if shifts is None:
        shifts = [(0.0, 0.0, 0.0), (0.5, 0.5, 0.5)] if interlace else [(0.0, 0.0, 0.0)]
    return [[int(round(2 * d)) % 2 == 1 for d in sh] for sh in shifts]


def shot_noise_expectation(n, ng, p, interlace, shot, mmax=2000, shifts=None):
    """E[P(n)] for a uniform random catalogue (n: (..., 3) integer modes, n != 0). With ``shifts`` (grid
    units, multiples of 1/2) the grids of multi-grid interlacing: image m is kept with weight
    (1/J) sum_j (-1)^{m.(2 d_j)}, so per grid each axis contributes its plain image sum (even shift)
    or its alternating one (odd number of half cells)."""
    n = np.asarray(n, dtype=np.float64)
    x = n / ng
    sums, alts = [], []
    win = np.ones(x.shape[:-1])
    for a in range(3):
        s, sa = _image_sums(x[..., a].ravel(), p, mmax)
        sums.append(s.reshape(x.shape[:-1]))
        alts.append(sa.reshape(x.shape[:-1]))
        win = win * (sinc(np.pi * x[..., a]) ** (2 * p))
    par = _parities(interlace, shifts)
    num = np.zeros(x.shape[:-1])
    for odd in par:
        term = np.ones(x.shape[:-1])
        for a in range(3):
            term = term * (alts[a] if odd[a] else sums[a])
        num += term
    return shot * num / len(par) / win


def fres_1d(x, p, interlace, mmax=100000):
    """eq:res1Di / eq:res1Dnoi as the truncated image sum over n != 0, x = k/k_s."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = np.arange(1, mmax + 1, dtype=np.float64)
    step = 2.0 if interlace else 1.0
    t = (x[:, None] / (x[:, None] - step * n[None, :])) ** (2 * p) + (x[:, None] / (x[:, None] + step * n[None, :])) ** (2 * p)
    return t.sum(axis=1)


def fres_1d_hurwitz(x, p, interlace):
    """Closed forms of eq:res1Dnoi, x^{2p}[zeta(2p, x) + zeta(2p, -x)] - 2, written with
    zeta(2p, 1 - x) + zeta(2p, 1 + x) (same series without the n = 0 terms); the interlaced form
    follows from eq:res_comp, F_int(x) = F_noint(x/2)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    y = x / 2.0 if interlace else x
    return y ** (2 * p) * (scipy.special.zeta(2 * p, 1.0 - y) + scipy.special.zeta(2 * p, 1.0 + y))


def fres_3d(n, ng, p, interlace, shifts=None):
    """F_res(n) = sum_{m != 0} theta_m prod_i (x_i / (x_i - m_i))^{2p}, x = n / N_G (eq:res with
    |w_m(k)|^2 = |W(k - m k_s)|^2 / |W(k)|^2 and |W| = sinc^p).

    The sum over all m factorises per axis: with f(x) = sum_{m != 0} (x/(x-m))^{2p} (eq:res1Dnoi) and
    the alternating f'(x) = sum_{m != 0} (-1)^m (x/(x-m))^{2p} = 2 F_int(x) - f(x) (F_int of eq:res1Di
    keeps the even images), theta_m = 1 gives prod(1 + f_i) - 1 and theta_m = [1 + (-1)^{sum m}]/2
    gives [prod(1 + f_i) + prod(1 + f'_i)]/2 - 1. The products are expanded so that no 1 is
    subtracted from a sum close to 1 (F_res is tiny at small k).

    With ``shifts`` (multi-grid interlacing, grid units) theta_m = (1/J) sum_j (-1)^{m.(2 d_j)} and
    F_res = (1/J) sum_j [prod_i (1 + g_ji) - 1], g_ji = f'(x_i) where d_ji is an odd number of half
    cells, else f(x_i)."""
    n = np.asarray(n, dtype=np.float64)
    x = n / ng
    f = [fres_1d_hurwitz(x[..., a].ravel(), p, False).reshape(x.shape[:-1]) for a in range(3)]
    fi = [fres_1d_hurwitz(x[..., a].ravel(), p, True).reshape(x.shape[:-1]) for a in range(3)]
    fa = [2.0 * fi[a] - f[a] for a in range(3)]

    def excess(g):  # prod(1 + g_i) - 1
        return g[0] + g[1] + g[2] + g[0] * g[1] + g[0] * g[2] + g[1] * g[2] + g[0] * g[1] * g[2]

    par = _parities(interlace, shifts)
    total = np.zeros(x.shape[:-1])
    for odd in par:
        total += excess([fa[a] if odd[a] else f[a] for a in range(3)])
    return total / len(par)


def fres_binned(ng, p, interlace, edges=None):
    """Mean and maximum of F_res(n) over the modes of each bin of the full N_G^3 grid (bins as in
    ``power.power_spectrum``), with the integer mode counts; NaN for empty bins."""
    if edges is None:
        edges = default_edges(ng)
    nb = len(edges) - 1
    s = signed_index(ng)
    n = np.stack(np.meshgrid(s, s, s, indexing="ij"), -1).reshape(-1, 3)
    b = bin_index(ng, edges).ravel()
    sel = b >= 0
    f = fres_3d(n[sel], ng, p, interlace)
    cnt = np.bincount(b[sel], minlength=nb).astype(np.int64)
    with np.errstate(invalid="ignore", divide="ignore"):
        mean = np.bincount(b[sel], weights=f, minlength=nb) / cnt
    mx = np.full(nb, np.nan)
    for k in range(nb):
        if cnt[k]:
            mx[k] = f[b[sel] == k].max()
    return mean, mx, cnt
