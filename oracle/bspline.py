"""B-spline mass-assignment kernels, Sec. 2.3 ("Mass Assignment and Aliasing").

Test infrastructure (see ``oracle/__init__``); never imported by the product path.

The one-dimensional weights W^(p)(s), s = (x_j^G - x)/H, for p = 1 (NGP), 2 (CIC), 3 (TSC) and
4 (PCS), written piece by piece as the paper lists them, and the Fourier window
W^(p)(k) = [sin(kH/2)/(kH/2)]^p of eq:intkerFT.

Reading taken for NGP: the cell is half-open, -1/2 <= s < 1/2, so that a particle exactly half-way
between two nodes still gives its whole mass to one of them (the paper's |s| < 1/2 gives none).

Reading taken for CIC: the paper prints the support of 1-|s| as |s| < 1/2, which contradicts the
two grid points per axis of a p = 2 scheme and the sinc^2 window; the support used is |s| < 1.

Orders p = 5, 6 (beyond the paper's PCS; Sec. 2.3 defines W^(p) as the top hat convolved with itself
p - 1 times): the centred B-spline in its truncated-power form,
W^(p)(s) = (1/(p-1)!) sum_{k=0}^{p} (-1)^k C(p, k) (s + p/2 - k)_+^{p-1}.
"""

from math import comb, factorial

import numpy as np


def weight(p, s):
    """W^(p)(s), Sec. 2.3: NGP, CIC, TSC and PCS piecewise polynomials (array in, array out)."""
    s = np.asarray(s, dtype=np.float64)
    a = np.abs(s)
    w = np.zeros_like(a)
    if p == 1:  # NGP: 1 for |s| < 1/2, with the tie s = -1/2 included (reading: half-open cell)
        w[(s >= -0.5) & (s < 0.5)] = 1.0
    elif p == 2:  # CIC: 1 - |s| for |s| < 1 (support reading, see module docstring)
        m = a < 1.0
        w[m] = 1.0 - a[m]
    elif p == 3:  # TSC: 3/4 - s^2 for |s| < 1/2; (3/2 - |s|)^2 / 2 for 1/2 <= |s| < 3/2
        m0 = a < 0.5
        m1 = (a >= 0.5) & (a < 1.5)
        w[m0] = 0.75 - a[m0] ** 2
        w[m1] = 0.5 * (1.5 - a[m1]) ** 2
    elif p == 4:  # PCS: (4 - 6 s^2 + 3|s|^3)/6 for |s| < 1; (2 - |s|)^3 / 6 for 1 <= |s| < 2
        m0 = a < 1.0
        m1 = (a >= 1.0) & (a < 2.0)
        w[m0] = (4.0 - 6.0 * a[m0] ** 2 + 3.0 * a[m0] ** 3) / 6.0
        w[m1] = (2.0 - a[m1]) ** 3 / 6.0
    elif p in (5, 6):
        for k in range(p + 1):
            t = s + 0.5 * p - k
            w += (-1) ** k * comb(p, k) * np.where(t > 0.0, t, 0.0) ** (p - 1)
        w /= factorial(p - 1)
        w[a >= 0.5 * p] = 0.0
    else:
        raise ValueError("order p must be 1..6")
    return w


def dweight(p, s):
    """dW^(p)/ds, the derivative of the Sec. 2.3 polynomials piece by piece (zero for NGP)."""
    s = np.asarray(s, dtype=np.float64)
    a = np.abs(s)
    sg = np.sign(s)
    d = np.zeros_like(a)
    if p == 1:
        pass
    elif p == 2:
        m = a < 1.0
        d[m] = -sg[m]
    elif p == 3:
        m0 = a < 0.5
        m1 = (a >= 0.5) & (a < 1.5)
        d[m0] = -2.0 * s[m0]
        d[m1] = -(1.5 - a[m1]) * sg[m1]
    elif p == 4:
        m0 = a < 1.0
        m1 = (a >= 1.0) & (a < 2.0)
        d[m0] = (-12.0 * a[m0] + 9.0 * a[m0] ** 2) / 6.0 * sg[m0]
        d[m1] = -0.5 * (2.0 - a[m1]) ** 2 * sg[m1]
    elif p in (5, 6):
        for k in range(p + 1):
            t = s + 0.5 * p - k
            d += (-1) ** k * comb(p, k) * np.where(t > 0.0, t, 0.0) ** (p - 2)
        d /= factorial(p - 2)
        d[a >= 0.5 * p] = 0.0
    else:
        raise ValueError("order p must be 1..6")
    return d


def sinc(x):
    """sin(x)/x with sinc(0) = 1 (argument in radians)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x != 0.0
    out[nz] = np.sin(x[nz]) / x[nz]
    return out


def window_k(p, n, ng):
    """Fourier window of one axis, eq:intkerFT: [sin(pi n/N_G)/(pi n/N_G)]^p for integer mode n.

    kH/2 = (2 pi n / L)(L / N_G)/2 = pi n / N_G.
    """
    return sinc(np.pi * np.asarray(n, dtype=np.float64) / ng) ** p
