"""Power spectrum from the grid density: shell binning of V |delta(n)|^2 (Sec. 2.2, eq:ps and the
estimator P^ = k_f^3 |delta(k)|^2 in the paper's normalisation).

Test infrastructure (see ``oracle/__init__``); never imported by the product path.

Normalisation: with delta(n) the dimensionless Fourier coefficient of ``fourier``, the estimator is
P(n) = V |delta(n)|^2 (the paper's P differs by the constant (2 pi)^3 of its transform convention).
Bins: edges e_0 < e_1 < ... in units of k_f/2 (integers); a mode n != 0 belongs to bin b when
e_b^2 <= 4|n|^2 < e_{b+1}^2, an exact integer test. The default bins are centred on b k_f,
b = 1..N_G/2 (edges 2b -/+ 1). Every mode of the full N_G^3 grid is visited once.
"""

import numpy as np

from .fourier import signed_index


def default_edges(ng):
    """Edges (units of k_f/2) of the bins (b - 1/2) k_f <= |k| < (b + 1/2) k_f, b = 1..N_G/2."""
    return 1 + 2 * np.arange(ng // 2 + 1, dtype=np.int64)


def mode_norm2_x4(ng):
    """4 |n|^2 on the full grid, int64 (signed convention)."""
    n = signed_index(ng).astype(np.int64)
    n2 = n * n
    return 4 * (n2[:, None, None] + n2[None, :, None] + n2[None, None, :])


def bin_index(ng, edges):
    """Bin of every mode (-1 outside the edges, and for n = 0), from the exact integer test."""
    e2 = np.asarray(edges, dtype=np.int64) ** 2
    v = mode_norm2_x4(ng)
    b = np.searchsorted(e2, v, side="right") - 1
    b[(b >= len(edges) - 1) | (v == 0)] = -1
    return b


def power_spectrum(delta, box, edges=None, subtract=0.0):
    """Bin averages of V|delta(n)|^2, mean |k| and the integer mode count per bin.

    Returns (P_b, k_eff_b, count_b); empty bins give NaN for P and k_eff. ``subtract`` is removed
    from every non-empty bin (the shot noise 1/nbar when requested).
    """
    ng = delta.shape[0]
    if edges is None:
        edges = default_edges(ng)
    nb = len(edges) - 1
    b = bin_index(ng, edges).ravel()
    sel = b >= 0
    vol = float(box) ** 3
    pk_modes = vol * np.abs(delta.ravel()[sel]) ** 2
    kf = 2.0 * np.pi / box
    kmag = kf * np.sqrt(mode_norm2_x4(ng).ravel()[sel] / 4.0)
    cnt = np.bincount(b[sel], minlength=nb).astype(np.int64)
    ssum = np.bincount(b[sel], weights=pk_modes, minlength=nb)
    ksum = np.bincount(b[sel], weights=kmag, minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        pk = ssum / cnt - subtract
        keff = ksum / cnt
    return pk, keff, cnt


def shot_noise(box, weights=None, n=None):
    """1/nbar = V/N_P for equal masses (Sec. 2.2, eq:ds2pcf); V sum w^2 / (sum w)^2 with weights."""
    vol = float(box) ** 3
    if weights is None:
        return vol / n
    w = np.asarray(weights, dtype=np.float64)
    return vol * np.sum(w * w) / np.sum(w) ** 2


def half_complex_weights(ng):
    """Multiplicity of each stored mode of the half-complex layout [N][N][N/2+1] (i_z <= N/2, i_z = N/2
    meaning n_z = -N/2): 2 where 0 < i_z < N/2 (the stored mode and its partner -n, whose n_z lies
    in (-N/2, 0) and is not stored), 1 on the planes i_z = 0 and i_z = N/2, where every mode of the
    full grid is stored itself."""
    m = np.full((ng, ng, ng // 2 + 1), 2.0)
    m[:, :, 0] = 1.0
    m[:, :, ng // 2] = 1.0
    return m


def cross_power_half(da, db, box, edges=None):
    """Binned cross power V Re[delta_a(n) conj(delta_b(n))] of two fields given on the half-complex
    layout, each stored mode counted with the multiplicity of ``half_complex_weights`` (its partner
    -n contributing the conjugate product, which has the same real part). With da = db this is the
    auto power over the stored modes and their partners: the N_G^3 vectors of the full grid, except
    that a partner with a component +N_G/2 stands for the grid's -N_G/2 (the two are the same mode of
    a periodic grid transform, and different modes of the direct sum of eq:deltaDS).

    Bins as in ``power_spectrum`` (same integer test; counts equal those of the full grid).
    Returns (P_b, k_eff_b, count_b), NaN for empty bins; no shot noise is subtracted.
    """
    ng = da.shape[0]
    if edges is None:
        edges = default_edges(ng)
    nb = len(edges) - 1
    b = bin_index(ng, edges)[:, :, : ng // 2 + 1].ravel()
    mult = half_complex_weights(ng).ravel()
    sel = b >= 0
    vol = float(box) ** 3
    prod = vol * np.real(np.asarray(da).ravel() * np.conj(np.asarray(db).ravel()))
    kf = 2.0 * np.pi / box
    kmag = kf * np.sqrt(mode_norm2_x4(ng)[:, :, : ng // 2 + 1].ravel() / 4.0)
    cnt = np.bincount(b[sel], weights=mult[sel], minlength=nb)
    ssum = np.bincount(b[sel], weights=(mult * prod)[sel], minlength=nb)
    ksum = np.bincount(b[sel], weights=(mult * kmag)[sel], minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        pk = ssum / cnt
        keff = ksum / cnt
    return pk, keff, np.rint(cnt).astype(np.int64)
