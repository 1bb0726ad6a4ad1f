"""Bispectrum estimator of Sec. 4.1: the shell definition (eq:Best, eq:VBest) by brute force, and the
fast form (eq:Best2, eq:IntI) that filters the density into k-shells, inverse-transforms each shell
and sums the triple product over the grid.

Test infrastructure (see ``oracle/__init__``); never imported by the product path.

Readings (the shell integral of the paper is garbled): shell s (0-based) holds the modes n != 0 with
(lo + s w) <= |n| < (lo + (s+1) w) in units of k_f (exact integer test on |n|^2). Triangles are all
shell triples s1 >= s2 >= s3 with s1 <= s2 + s3 + 1 (the closure test of the shell centres with one
shell of slack), listed with s1 slowest and s3 fastest. V_B is the exact number N_tri of mode triplets
(q1, q2, q3) with q_i in shell s_i and q1 + q2 + q3 = 0, so that
B = V^2 <delta_q1 delta_q2 delta_q3> = V^2 S / (N_c N_tri) with S = sum_x I_1 I_2 I_3.
The largest usable |q| is below N_G/3 (Sec. 4.1); the shells must end below that.
"""

import os

import numpy as np
import scipy.fft

from .fourier import signed_index

_WORKERS = os.cpu_count() or 1


def mode_norm2(ng):
    n = signed_index(ng).astype(np.int64)
    n2 = n * n
    return n2[:, None, None] + n2[None, :, None] + n2[None, None, :]


def shell_masks(ng, lo, w, nshells):
    """Boolean mask of each shell on the full mode grid (n = 0 excluded)."""
    kmax = lo + nshells * w
    if 3 * (kmax - 1) >= ng:
        raise ValueError("shells must stay below k_max = k_f N_G/3 (Sec. 4.1): need 3 (kmax - 1) < N_G")
    m2 = mode_norm2(ng)
    out = []
    for s in range(nshells):
        a, b = lo + s * w, lo + (s + 1) * w
        out.append((m2 >= a * a) & (m2 < b * b) & (m2 > 0))
    return out


def triangles(nshells):
    """(s1, s2, s3) with s1 >= s2 >= s3 and s1 <= s2 + s3 + 1, s1 slowest."""
    return [(a, b, c) for a in range(nshells) for b in range(a + 1) for c in range(b + 1) if a <= b + c + 1]


def shell_fields(delta, masks):
    """I_s(x) = sum_{n in shell s} delta(n) exp(+2 pi i n.x/N_G) (eq:IntI), real by Hermitian symmetry."""
    nc = delta.size
    return [np.real(scipy.fft.ifftn(np.where(m, delta, 0.0), workers=_WORKERS)) * nc for m in masks]


def triangle_counts(ng, lo, w, nshells):
    """Exact N_tri per triangle: C12(m) = #{(q1, q2): q1 in s1, q2 in s2, q1 + q2 = m}, obtained by an
    FP64 circular convolution of the two shell indicators and rounded (the values are integers far
    below 2^52), then N_tri = sum_{m in s3} C12(m) in int64."""
    masks = shell_masks(ng, lo, w, nshells)
    ft = [scipy.fft.fftn(m.astype(np.float64), workers=_WORKERS) for m in masks]
    out = []
    for a, b, c in triangles(nshells):
        c12 = np.rint(np.real(scipy.fft.ifftn(ft[a] * ft[b], workers=_WORKERS))).astype(np.int64)
        out.append(int(c12[masks[c]].sum()))
    return np.array(out, dtype=np.int64)


def bispectrum_fft(delta, box, lo, w, nshells):
    """B per triangle from eq:Best2: V^2 sum_x I_1 I_2 I_3 / (N_c N_tri); NaN where N_tri = 0."""
    ng = delta.shape[0]
    masks = shell_masks(ng, lo, w, nshells)
    fields = shell_fields(delta, masks)
    counts = triangle_counts(ng, lo, w, nshells)
    vol2 = float(box) ** 6
    out = np.empty(len(counts))
    for t, (a, b, c) in enumerate(triangles(nshells)):
        s = np.sum(fields[a] * fields[b] * fields[c])
        out[t] = vol2 * s / (delta.size * counts[t]) if counts[t] > 0 else np.nan
    return out, counts


def bispectrum_brute(delta, box, lo, w, nshells):
    """eq:Best by enumeration: V^2 sum_{q1 in s1, q2 in s2, q3 = -q1-q2 in s3} delta delta delta / N_tri.

    Plain enumeration of q1 and q2 over the shells; for tiny grids only."""
    ng = delta.shape[0]
    n = signed_index(ng)
    m2 = mode_norm2(ng)
    lists = []
    for s in range(nshells):
        a, b = lo + s * w, lo + (s + 1) * w
        idx = np.argwhere((m2 >= a * a) & (m2 < b * b) & (m2 > 0))
        lists.append(n[idx])  # signed mode vectors of the shell
    vol2 = float(box) ** 6
    res, cnts = [], []
    for a, b, c in triangles(nshells):
        lo3, hi3 = (lo + c * w) ** 2, (lo + (c + 1) * w) ** 2
        acc = 0.0 + 0.0j
        cnt = 0
        for q1 in lists[a]:
            q3 = -(q1[None, :] + lists[b])
            r2 = np.sum(q3 * q3, axis=1)
            ok = (r2 >= lo3) & (r2 < hi3) & (r2 > 0)
            if not ok.any():
                continue
            q2 = lists[b][ok]
            q3 = q3[ok]
            acc += np.sum(delta[tuple(q1 % ng)] * delta[tuple((q2 % ng).T)] * delta[tuple((q3 % ng).T)])
            cnt += int(ok.sum())
        cnts.append(cnt)
        res.append(vol2 * acc.real / cnt if cnt > 0 else np.nan)
    return np.array(res), np.array(cnts, dtype=np.int64)
