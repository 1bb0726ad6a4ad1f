"""Aliasing sums of Secs. 2.3 and 3.1 for B-spline windows.

Test infrastructure (see ``oracle/__init__``); never imported by the product path.

- ``shot_noise_expectation``: eq:Pknoint and its interlaced form with P = 0, i.e. the expected
  window-corrected power of a uniform random (Poisson) catalogue, the aliasing sum over images m of
  theta_m |W(k - m k_s)|^2 P_tot / |W(k)|^2 with P_tot = 1/nbar and theta_m = 1 (no interlacing) or
  [1 + (-1)^(m_x+m_y+m_z)]/2 (interlacing). With x = n/N_G, |W(k - m k_s)| = |sinc(pi (x - m))|^p.
- ``fres_1d`` / ``fres_1d_hurwitz``: the one-dimensional residual factor of eq:res1Di and
  eq:res1Dnoi as a truncated image sum and in its Hurwitz-zeta closed form.
"""

import numpy as np
import scipy.special

from .bspline import sinc


def _image_sums(x, p, mmax):
    """Per axis: sum_m sinc^{2p}(pi (x - m)) and sum_m (-1)^m sinc^{2p}(pi (x - m)), |m| <= mmax."""
    m = np.arange(-mmax, mmax + 1, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    t = sinc(np.pi * (x[:, None] - m[None, :])) ** (2 * p)
    sgn = np.where(np.abs(m) % 2 == 0, 1.0, -1.0)
    return t.sum(axis=1), (t * sgn[None, :]).sum(axis=1)


def shot_noise_expectation(n, ng, p, interlace, shot, mmax=2000):
    """E[P(n)] for a uniform random catalogue (n: (..., 3) integer modes, n != 0)."""
    n = np.asarray(n, dtype=np.float64)
    x = n / ng
    even = np.ones(x.shape[:-1])
    alt = np.ones(x.shape[:-1])
    win = np.ones(x.shape[:-1])
    for a in range(3):
        s, sa = _image_sums(x[..., a].ravel(), p, mmax)
        even = even * s.reshape(x.shape[:-1])
        alt = alt * sa.reshape(x.shape[:-1])
        win = win * (sinc(np.pi * x[..., a]) ** (2 * p))
    num = 0.5 * (even + alt) if interlace else even
    return shot * num / win


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
