"""Grid density in Fourier space: FFT, interlacing combine (eq:intdelta) and window deconvolution
(eq:windowcorrection, eq:intkerFT), evaluated on every mode of the full N_G^3 grid.

Test infrastructure (see ``oracle/__init__``); never imported by the product path.

Conventions: delta_j = rho_j / rhobar - 1 (Sec. 2.1, with rhobar the mean of the mass grid);
delta(n) = (1/N_c) sum_j delta_j exp(-2 pi i n.j / N_G) with the signed mode index
n_i in [-N_G/2, N_G/2). The interlaced grid samples the field at x_j - H/2 (particles shifted by
+H/2), so by the shift theorem its alias images carry (-1)^(n_x+n_y+n_z) once it is multiplied by
exp(+i k.(H/2)(1,1,1)) = exp(+i pi (n_x+n_y+n_z)/N_G); the average of the two grids (eq:intdelta)
then cancels the odd images.
"""

import os

import numpy as np
import scipy.fft

from .bspline import window_k

_WORKERS = os.cpu_count() or 1


def signed_index(ng):
    """Signed mode index of each FFT slot: i for i < N_G/2, else i - N_G (so N_G/2 -> -N_G/2)."""
    i = np.arange(ng)
    return np.where(i < ng // 2, i, i - ng)


def overdensity(rho):
    """delta_j = rho_j / rhobar - 1, Sec. 2.1."""
    rho = np.asarray(rho, dtype=np.float64)
    return rho / rho.mean() - 1.0


def fourier_coefficients(field):
    """delta(n) = (1/N_c) sum_j field_j exp(-2 pi i n.j/N_G) on the full grid (FFT slot order)."""
    return scipy.fft.fftn(field, workers=_WORKERS) / field.size


def window_3d(p, ng):
    """W(n) = prod_i [sin(pi n_i/N_G)/(pi n_i/N_G)]^p, eq:intkerFT, separable in 3-D."""
    w1 = window_k(p, signed_index(ng), ng)
    return w1[:, None, None] * w1[None, :, None] * w1[None, None, :]


def interlace_phase(ng):
    """exp(+i pi (n_x+n_y+n_z)/N_G) on the full grid with the signed index (Sec. 3.1)."""
    n = signed_index(ng)
    s = n[:, None, None] + n[None, :, None] + n[None, None, :]
    return np.exp(1j * np.pi * s / ng)


def density_modes(rho1, p, rho2=None):
    """Window-corrected grid density delta^G(n) on every mode of the full grid.

    Without rho2: delta^G = delta~_1^G / W (eq:windowcorrection).
    With rho2 (the grid of the particles shifted by +H/2): delta~^G = (delta~_1^G + e^{+i pi sum n/N}
    delta~_2^G)/2 (eq:intdelta), then delta^G = delta~^G / W.
    The n = 0 mode is zero by construction (delta_j has zero mean).
    """
    ng = rho1.shape[0]
    d1 = fourier_coefficients(overdensity(rho1))
    if rho2 is None:
        dt = d1
    else:
        d2 = fourier_coefficients(overdensity(rho2))
        dt = 0.5 * (d1 + interlace_phase(ng) * d2)
    return dt / window_3d(p, ng)


def density_modes_multi(rhos, shifts, p):
    """Window-corrected density from J grids, grid j holding the particles shifted by d_j (grid
    units): delta^G = (1/J) sum_j e^{+2 pi i n.d_j/N_G} delta~_j^G / W, the phase that undoes each
    shift (Sec. 3.1 for J = 2, d = {0, (1,1,1)/2}). Image m of grid j then carries e^{+2 pi i m.d_j},
    so the average keeps images with weight (1/J) sum_j e^{2 pi i m.d_j}."""
    ng = rhos[0].shape[0]
    n = signed_index(ng)
    acc = np.zeros((ng, ng, ng), dtype=np.complex128)
    for rho, d in zip(rhos, shifts):
        d = np.asarray(d, dtype=np.float64)
        ph = np.exp(2j * np.pi * (n[:, None, None] * d[0] + n[None, :, None] * d[1] + n[None, None, :] * d[2]) / ng)
        acc += ph * fourier_coefficients(overdensity(rho))
    return acc / len(rhos) / window_3d(p, ng)


def multigrid_shifts(ngrids):
    """Shift sets of multi-grid interlacing (grid units): 1 grid {0}; 2 grids {0, (1,1,1)/2} (Sec. 3.1);
    4 grids {0, (1,1,0)/2, (1,0,1)/2, (0,1,1)/2}; 8 grids {0, 1/2}^3."""
    if ngrids == 1:
        return [(0.0, 0.0, 0.0)]
    if ngrids == 2:
        return [(0.0, 0.0, 0.0), (0.5, 0.5, 0.5)]
    if ngrids == 4:
        return [(0.0, 0.0, 0.0), (0.5, 0.5, 0.0), (0.5, 0.0, 0.5), (0.0, 0.5, 0.5)]
    if ngrids == 8:
        return [(a, b, c) for a in (0.0, 0.5) for b in (0.0, 0.5) for c in (0.0, 0.5)]
    raise ValueError("ngrids must be 1, 2, 4 or 8")
