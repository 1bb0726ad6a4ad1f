"""Direct-summation Fourier coefficients of a particle set, eq:deltaDS (Sec. 2.2): alias-free and
window-free, at cost N_P x (number of modes).

Test infrastructure (see ``oracle/__init__``); never imported by the product path.

In the dimensionless convention used throughout the oracle, eq:deltaDS reads
delta(n) = (1/sum_i w_i) sum_i w_i exp(-2 pi i n.u_i/N_G) - Kronecker(n), with u = x/H.

Unlike a grid transform, the sum is defined for every integer vector n and is not periodic in n:
n and n + N_G e_x differ by the factor exp(-2 pi i u_x) per particle. It is exactly Hermitian,
delta(-n) = conj(delta(n)), for every n.
"""

import numpy as np

from .assign import grid_units
from .fourier import signed_index


def direct_modes(pos, box, ng, weights=None):
    """delta(n) by direct summation on every mode of the full N_G^3 grid (FFT slot order)."""
    u = grid_units(pos, box, ng)
    n = signed_index(ng)
    w = np.ones(len(u)) if weights is None else np.asarray(weights, dtype=np.float64)
    ph = [np.exp(-2j * np.pi * np.outer(u[:, a], n) / ng) for a in range(3)]  # (N_P, N_G) per axis
    d = np.einsum("i,ia,ib,ic->abc", w, ph[0], ph[1], ph[2], optimize=True) / np.sum(w)
    d[0, 0, 0] -= 1.0
    return d


def direct_modes_at(pos, box, nvec, weights=None):
    """delta(n) of eq:deltaDS at arbitrary integer mode vectors nvec (M, 3); k = k_f n, so the phase
    of particle i is k.x_i = 2 pi n.x_i / L. The Kronecker term is removed where n = 0."""
    x = np.asarray(pos, dtype=np.float64)
    nvec = np.asarray(nvec, dtype=np.int64)
    w = np.ones(len(x)) if weights is None else np.asarray(weights, dtype=np.float64)
    out = np.empty(len(nvec), dtype=np.complex128)
    for s in range(0, len(nvec), 256):
        ph = np.exp(-2j * np.pi * (nvec[s:s + 256].astype(np.float64) @ x.T) / box)  # (m, N_P)
        out[s:s + 256] = ph @ w / np.sum(w)
    out[np.all(nvec == 0, axis=1)] -= 1.0
    return out
