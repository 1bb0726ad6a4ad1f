"""Seeded synthetic particle catalogues (test and benchmark inputs).

This module generates inputs only; it holds none of the estimator's arithmetic and imports neither
the CUDA library nor the oracle, so both sides of a parity test can take their inputs from it.

Catalogues (positions in a periodic cube of side ``box``, FP64 unless stated):

- ``poisson``: uniform random positions (the Poisson / shot-noise workload).
- ``lattice``: particles on a regular lattice (exact-cancellation checks).
- ``zeldovich``: a lattice displaced by a Gaussian random displacement field whose density has the
  power spectrum P(k) = A k^slope exp(-(k/kcut)^2), A fixed by the rms displacement
  (Zel'dovich approximation: psi(k) = i k delta(k)/k^2, x = q + psi). The paper's tests use
  N-body and Zel'dovich catalogues of this kind (Sec. 3.2); these synthetic ones stand in for them.
- ``batch_sizes``: per-catalogue particle counts drawn log-uniform in [lo, hi].
"""

import numpy as np


def poisson(n, box, seed):
    """n uniform random positions in [0, box)^3 (FP64)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, box, size=(int(n), 3))


def lattice(nside, box, offset=0.5):
    """Particles at (i + offset) box/nside on every axis, C order (x slowest)."""
    q = (np.arange(nside, dtype=np.float64) + offset) * (box / nside)
    g = np.meshgrid(q, q, q, indexing="ij")
    return np.stack([a.ravel() for a in g], axis=1)


def random_weights(n, seed, lo=0.5, hi=1.5):
    """Positive per-particle weights, uniform in [lo, hi)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=int(n))


def _displacement_numpy(nside, box, rms, seed, kcut, slope):
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((nside, nside, nside))
    wk = np.fft.rfftn(white)
    kf = 2.0 * np.pi / box
    k1 = np.fft.fftfreq(nside, d=1.0 / nside) * kf
    kz = np.fft.rfftfreq(nside, d=1.0 / nside) * kf
    kx, ky, kzz = np.meshgrid(k1, k1, kz, indexing="ij")
    k2 = kx * kx + ky * ky + kzz * kzz
    k = np.sqrt(k2)
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = np.sqrt(k[nz] ** slope * np.exp(-(k[nz] / kcut) ** 2))
    dk = wk * amp
    nyq = nside // 2
    dk[nyq, :, :] = 0.0
    dk[:, nyq, :] = 0.0
    dk[:, :, nyq] = 0.0
    dk[0, 0, 0] = 0.0
    psi = []
    for kc in (kx, ky, kzz):
        comp = np.zeros_like(dk)
        comp[nz] = 1j * kc[nz] * dk[nz] / k2[nz]
        psi.append(np.fft.irfftn(comp, s=(nside, nside, nside), axes=(0, 1, 2)))
    psi = np.stack([p.ravel() for p in psi], axis=1)
    cur = np.sqrt(np.mean(np.sum(psi * psi, axis=1)))
    return psi * (rms / cur)


def zeldovich(nside, box, rms, seed, kcut=0.5, slope=-1.5):
    """Lattice of nside^3 particles displaced by a Gaussian random field (CPU, FP64).

    The field: white noise -> FFT -> times sqrt(k^slope exp(-(k/kcut)^2)) (k in units of 2 pi/box
    per box length, i.e. h/Mpc for box in Mpc/h) -> psi(k) = i k delta(k)/k^2 with k = 0 and the
    Nyquist planes zeroed -> inverse FFT -> rescaled so that the rms |psi| equals ``rms``.
    Positions are wrapped into [0, box)."""
    q = lattice(nside, box)
    psi = _displacement_numpy(nside, box, rms, seed, kcut, slope)
    x = np.mod(q + psi, box)
    x[x >= box] -= box
    return x


def zeldovich_torch(nside, box, rms, seed, device, kcut=0.5, slope=-1.5, out_dtype=None):
    """Same recipe as ``zeldovich`` on a torch device (for catalogues too large for the host).

    Returns an (nside^3, 3) FP64 tensor on ``device`` (or ``out_dtype``). Generation is staged one
    displacement component at a time to bound peak memory."""
    import torch

    out_dtype = out_dtype or torch.float64
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    white = torch.randn((nside, nside, nside), generator=gen, device=device, dtype=torch.float32)
    dk = torch.fft.rfftn(white)
    del white
    kf = 2.0 * np.pi / box
    k1 = torch.fft.fftfreq(nside, d=1.0 / nside, device=device, dtype=torch.float32) * kf
    kz = torch.fft.rfftfreq(nside, d=1.0 / nside, device=device, dtype=torch.float32) * kf
    k2 = k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kz[None, None, :] ** 2
    k2[0, 0, 0] = 1.0
    amp = torch.sqrt(k2 ** (0.5 * slope) * torch.exp(-k2 / (kcut * kcut)))
    amp[0, 0, 0] = 0.0
    dk *= amp
    del amp
    nyq = nside // 2
    dk[nyq, :, :] = 0
    dk[:, nyq, :] = 0
    dk[:, :, nyq] = 0
    n = nside ** 3
    out = torch.empty((n, 3), device=device, dtype=out_dtype)
    sumsq = 0.0
    comps = (k1[:, None, None], k1[None, :, None], kz[None, None, :])
    for a in range(3):
        comp = dk * (1j * comps[a] / k2)
        psi = torch.fft.irfftn(comp, s=(nside, nside, nside)).reshape(-1)
        del comp
        sumsq += float(torch.sum(psi.double() ** 2))
        out[:, a] = psi.to(out_dtype)
        del psi
    del dk
    scale = rms / np.sqrt(sumsq / n)
    q1 = (torch.arange(nside, device=device, dtype=torch.float64) + 0.5) * (box / nside)
    for a in range(3):
        shape = [1, 1, 1]
        shape[a] = nside
        qa = q1.view(shape).expand(nside, nside, nside).reshape(-1)
        col = torch.remainder(qa + out[:, a].double() * scale, box)
        col[col >= box] -= box
        out[:, a] = col.to(out_dtype)
    return out


def batch_sizes(n_cat, lo, hi, seed):
    """Particle counts floor(exp(U[ln lo, ln hi])) per catalogue."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), size=int(n_cat)))).astype(np.int64)
