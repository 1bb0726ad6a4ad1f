"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics, independent of
the oracle's own code: closed forms, invariants, brute force on tiny inputs and a statistical
expectation. Each test names the passage it pins."""

import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import adjoint, aliasing, assign, bispectrum, bspline, direct, fourier, power
from paper_1512_07295_gb300 import catalogs


# --- Sec. 2.3 kernels against eq:intkerFT -----------------------------------------------------------

def _ft_numeric(p, nu):
    """int W^(p)(s) exp(-2 pi i nu s) ds by Gauss-Legendre on every unit-half piece (exact for the
    piecewise polynomials, whatever their coefficients)."""
    xg, wg = np.polynomial.legendre.leggauss(12)
    total = 0.0
    for a in np.arange(-p / 2.0, p / 2.0, 0.5):
        s = a + 0.25 * (xg + 1.0)
        total += 0.25 * np.sum(wg * bspline.weight(p, s) * np.cos(2 * np.pi * nu * s))
    return total


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_kernel_fourier_transform_is_sinc_power(p):
    # eq:intkerFT: the FT of the order-p B-spline of unit spacing is sinc^p(pi nu); this pins the
    # piece-wise coefficients of Sec. 2.3 (and the CIC support reading |s| < 1).
    for nu in [0.0, 0.1, 0.25, 0.37, 0.5, 0.8, 1.3]:
        expect = bspline.sinc(np.pi * nu) ** p
        assert abs(_ft_numeric(p, nu) - expect) < 1e-12


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_kernel_derivative_matches_finite_difference(p):
    s = np.linspace(-3.3, 3.3, 661) + 1e-3
    h = 1e-6
    fd = (bspline.weight(p, s + h) - bspline.weight(p, s - h)) / (2 * h)
    assert np.max(np.abs(fd - bspline.dweight(p, s))) < 1e-6


# --- eq:delgrid: partition of unity, single particle, lattices -------------------------------------

@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("shift", [False, True])
def test_mass_conservation(p, shift):
    pos = catalogs.poisson(500, 100.0, seed=11)
    w = catalogs.random_weights(500, seed=12)
    rho = assign.assign(pos, 100.0, 12, p, weights=w, shift=shift)
    assert abs(rho.sum() - w.sum()) < 1e-11 * w.sum()
    assert rho.min() >= 0.0


def _poisson_sum_1d(u, ng, p, mmax):
    """sum_j W^(p)(j - u) e^{-2 pi i n j/N} for all n, by Poisson summation of the continuous
    transform: sum_m e^{-2 pi i (nu+m) u} sinc^p(pi (nu+m)), nu = n/N (eq:tdelG2 with eq:intkerFT)."""
    nu = np.arange(ng) / ng
    m = np.arange(-mmax, mmax + 1)
    f = nu[:, None] + m[None, :]
    return np.sum(np.exp(-2j * np.pi * f * u) * bspline.sinc(np.pi * f) ** p, axis=1)


@pytest.mark.parametrize("p,tol", [(2, 2e-6), (3, 1e-9), (4, 1e-11), (5, 1e-11), (6, 1e-11)])
@pytest.mark.parametrize("shift", [False, True])
def test_single_particle_grid_transform(p, tol, shift):
    # One particle: the DFT of its mass grid is the product over axes of the aliased window sums.
    ng, box = 8, 10.0
    x = np.array([[1.234, 5.678, 9.012]])
    rho = assign.assign(x, box, ng, p, shift=shift)
    g = np.fft.fftn(rho)
    u = x[0] * ng / box + (0.5 if shift else 0.0)
    ax = [_poisson_sum_1d(u[a], ng, p, 200000 if p == 2 else 4000) for a in range(3)]
    expect = ax[0][:, None, None] * ax[1][None, :, None] * ax[2][None, None, :]
    assert np.max(np.abs(g - expect)) < tol


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_full_lattice_has_no_power(p):
    # Particles on every node: the partition of unity makes the grid uniform, so delta = 0 (both
    # the plain and the shifted grid), and P vanishes in every bin.
    ng, box = 8, 50.0
    pos = catalogs.lattice(ng, box, offset=0.0)
    rho1 = assign.assign(pos, box, ng, p)
    rho2 = assign.assign(pos, box, ng, p, shift=True)
    assert np.max(np.abs(rho1 - 1.0)) < 1e-12
    assert np.max(np.abs(rho2 - 1.0)) < 1e-12
    pk, _, cnt = power.power_spectrum(fourier.density_modes(rho1, p, rho2), box)
    assert np.all(cnt > 0)
    assert np.max(np.abs(pk)) < 1e-20 * box ** 3 / ng ** 3


def test_second_lattice_pcs_pattern():
    # Particles on every second node, PCS: node weights 2/3 (own node) and 1/6 (neighbours) give the
    # per-axis pattern (2/3, 1/3); its DFT is N/2 at n = 0 and N/2 (2/3 - 1/3) at n = N/2, so the only
    # non-zero modes have every n_i in {0, -N/2}.
    ng, box = 8, 16.0
    pos = catalogs.lattice(ng // 2, box, offset=0.0)
    rho = assign.assign(pos, box, ng, 4)
    d = fourier.fourier_coefficients(fourier.overdensity(rho))
    a = {0: 1.0, ng // 2: 1.0 / 3.0}  # per-axis DFT normalised by its n = 0 value
    for idx in itertools.product(range(ng), repeat=3):
        if all(i in a for i in idx) and idx != (0, 0, 0):
            assert abs(d[idx] - a[idx[0]] * a[idx[1]] * a[idx[2]]) < 1e-13
        else:
            assert abs(d[idx]) < 1e-13


# --- FFT conventions ---------------------------------------------------------------------------------

def test_fft_matches_direct_dft():
    ng = 5
    rng = np.random.default_rng(3)
    f = rng.standard_normal((ng, ng, ng))
    out = np.zeros((ng, ng, ng), dtype=complex)
    j = np.array(list(itertools.product(range(ng), repeat=3)))
    for n in itertools.product(range(ng), repeat=3):
        ph = np.exp(-2j * np.pi * (j @ np.array(n)) / ng)
        out[n] = np.sum(f.ravel() * ph) / ng ** 3
    assert np.max(np.abs(fourier.fourier_coefficients(f) - out)) < 1e-14


def test_parseval_full_grid():
    rng = np.random.default_rng(4)
    f = rng.standard_normal((6, 6, 6))
    d = fourier.fourier_coefficients(f)
    assert abs(np.sum(np.abs(d) ** 2) * f.size - np.sum(f * f)) < 1e-10


def test_interlace_phase_nyquist_convention():
    # Signed index: slot N/2 is -N/2, so the phase there is exp(-i pi/2) per axis.
    ph = fourier.interlace_phase(8)
    assert abs(ph[4, 0, 0] - np.exp(-1j * np.pi / 2)) < 1e-15
    assert abs(ph[1, 2, 3] - np.exp(1j * np.pi * 6 / 8)) < 1e-15


# --- binning: exact integer counts --------------------------------------------------------------------

@pytest.mark.parametrize("ng", [6, 8, 12])
def test_mode_counts_brute_force(ng):
    edges = power.default_edges(ng)
    _, _, cnt = power.power_spectrum(np.ones((ng, ng, ng), dtype=complex), 1.0, edges)
    ref = np.zeros(len(edges) - 1, dtype=np.int64)
    half = ng // 2
    for n in itertools.product(range(-half, half), repeat=3):
        r = math.sqrt(n[0] ** 2 + n[1] ** 2 + n[2] ** 2)
        if r == 0:
            continue
        b = int(math.floor(r + 0.5))  # (b - 1/2) <= |n| < (b + 1/2)
        if 1 <= b <= half:
            ref[b - 1] += 1
    assert np.array_equal(cnt, ref)


# --- shot-noise aliasing sums (eq:Pknoint and its interlaced form with P = 0) --------------------------

def _bspline_autocorr(p, m):
    """int W^(p)(s) W^(p)(s + m) ds, Gauss-Legendre per half-unit piece (exact for polynomials)."""
    xg, wg = np.polynomial.legendre.leggauss(16)
    tot = 0.0
    for a in np.arange(-p / 2.0 - abs(m), p / 2.0 + abs(m), 0.5):
        s = a + 0.25 * (xg + 1.0)
        tot += 0.25 * np.sum(wg * bspline.weight(p, s) * bspline.weight(p, s + m))
    return tot


@pytest.mark.parametrize("p", [2, 4])
def test_alias_sum_equals_autocorrelation_series(p):
    # sum_m sinc^{2p}(pi (x - m)) = sum_m M_{2p}(m) cos(2 pi m x), M the kernel autocorrelation; for
    # CIC the coefficients are the rationals 2/3 and 1/6.
    xs = np.array([0.05, 0.2, 0.33, 0.5])
    series = np.zeros_like(xs)
    coeffs = [_bspline_autocorr(p, m) for m in range(p)]
    for m, c in enumerate(coeffs):
        series += c * (1.0 if m == 0 else 2.0 * np.cos(2 * np.pi * m * xs))
    imgs, _ = aliasing._image_sums(xs, p, 4000)
    assert np.max(np.abs(series - imgs)) < (1e-9 if p == 2 else 1e-12)
    if p == 2:
        assert abs(coeffs[0] - float(Fraction(2, 3))) < 1e-14
        assert abs(coeffs[1] - float(Fraction(1, 6))) < 1e-14


@pytest.mark.parametrize("p,interlace", [(2, False), (2, True), (4, True)])
def test_poisson_power_matches_alias_expectation(p, interlace):
    # A uniform random catalogue has P = 0, so the window-corrected estimator averages to the aliased
    # shot noise (eq:Pknoint; with interlacing only the even images survive, eq:intdelta). A wrong
    # interlacing phase sign or a wrong window fails this by many sigma near the Nyquist frequency.
    ng, box, npart, nseeds = 8, 100.0, 400, 300
    shot = box ** 3 / npart
    edges = power.default_edges(ng)
    b = power.bin_index(ng, edges)
    half = ng // 2
    sn = fourier.signed_index(ng)
    nvec = np.stack(np.meshgrid(sn, sn, sn, indexing="ij"), axis=-1)
    sel = b >= 0
    e_mode = aliasing.shot_noise_expectation(nvec[sel], ng, p, interlace, shot, mmax=3000)
    cnt = np.bincount(b[sel], minlength=half)
    expect = np.bincount(b[sel], weights=e_mode, minlength=half) / cnt
    # per-mode variance: |delta|^2 of a sum of many particles is exponential (variance = mean^2);
    # modes n and -n are identical except on Nyquist planes, so use half the count.
    var_mode = np.bincount(b[sel], weights=e_mode ** 2, minlength=half) / cnt
    acc = np.zeros(half)
    for s in range(nseeds):
        pos = catalogs.poisson(npart, box, seed=1000 + s)
        r1 = assign.assign(pos, box, ng, p)
        r2 = assign.assign(pos, box, ng, p, shift=True) if interlace else None
        pk, _, _ = power.power_spectrum(fourier.density_modes(r1, p, r2), box, edges)
        acc += pk
    mean = acc / nseeds
    sigma = np.sqrt(var_mode / (cnt / 2.0) / nseeds)
    z = (mean - expect) / sigma
    assert np.max(np.abs(z)) < 4.5, z


@pytest.mark.parametrize("ngrids", [4, 8])
def test_multigrid_poisson_power_matches_alias_expectation(ngrids):
    # Multi-grid interlacing (the extension of Sec. 3.1): each grid's shift phase must cancel exactly
    # the images whose weight (1/J) sum_j e^{2 pi i m.d_j} vanishes; the realised power of uniform random
    # catalogues averages to the aliasing sum with those weights. A wrong phase sign or shift direction
    # on any grid leaves odd images in and fails by many sigma near the Nyquist frequency.
    p, ng, box, npart, nseeds = 2, 8, 100.0, 400, 150
    shifts = fourier.multigrid_shifts(ngrids)
    shot = box ** 3 / npart
    edges = power.default_edges(ng)
    b = power.bin_index(ng, edges)
    half = ng // 2
    sn = fourier.signed_index(ng)
    nvec = np.stack(np.meshgrid(sn, sn, sn, indexing="ij"), axis=-1)
    sel = b >= 0
    e_mode = aliasing.shot_noise_expectation(nvec[sel], ng, p, False, shot, mmax=3000, shifts=shifts)
    cnt = np.bincount(b[sel], minlength=half)
    expect = np.bincount(b[sel], weights=e_mode, minlength=half) / cnt
    var_mode = np.bincount(b[sel], weights=e_mode ** 2, minlength=half) / cnt
    acc = np.zeros(half)
    for s in range(nseeds):
        pos = catalogs.poisson(npart, box, seed=3000 + s)
        u = assign.grid_units(pos, box, ng)
        rhos = [assign.assign_units(u, ng, p, shift=d) for d in shifts]
        pk, _, _ = power.power_spectrum(fourier.density_modes_multi(rhos, shifts, p), box, edges)
        acc += pk
    mean = acc / nseeds
    sigma = np.sqrt(var_mode / (cnt / 2.0) / nseeds)
    z = (mean - expect) / sigma
    assert np.max(np.abs(z)) < 4.5, z
    # more grids leave less aliasing: the expectation approaches 1/nbar bin by bin near Nyquist
    e2 = aliasing.shot_noise_expectation(nvec[sel], ng, p, True, shot, mmax=3000)
    exp2 = np.bincount(b[sel], weights=e2, minlength=half) / cnt
    assert abs(expect[-1] / shot - 1.0) < abs(exp2[-1] / shot - 1.0)


@pytest.mark.parametrize("ngrids", [1, 2, 4, 8])
def test_multigrid_fres_is_the_shot_noise_excess(ngrids):
    # the Hurwitz-zeta F_res with the multi-grid weights against the sinc^{2p} image sums
    shifts = fourier.multigrid_shifts(ngrids)
    rng = np.random.default_rng(62)
    n = rng.integers(-16, 16, (50, 3))
    n = n[np.abs(n).max(axis=1) >= 6]
    for p in (2, 4):
        e = aliasing.shot_noise_expectation(n, 32, p, False, 1.0, mmax=4000, shifts=shifts)
        f = aliasing.fres_3d(n, 32, p, False, shifts=shifts)
        assert np.max(np.abs(e - 1.0 - f) / (1.0 + f)) < 2e-10


def test_two_grid_combine_is_the_interlaced_estimate():
    pos = catalogs.zeldovich(8, 50.0, rms=2.0, seed=63)
    u = assign.grid_units(pos, 50.0, 12)
    r1, r2 = assign.assign_units(u, 12, 3), assign.assign_units(u, 12, 3, shift=True)
    a = fourier.density_modes(r1, 3, r2)
    b = fourier.density_modes_multi([r1, r2], fourier.multigrid_shifts(2), 3)
    assert np.max(np.abs(a - b)) < 1e-14


def test_interlacing_removes_odd_images_in_expectation():
    # With interlacing the expected PCS shot noise is much closer to 1/nbar near Nyquist.
    shot = 1.0
    n = np.array([[4, 0, 0], [3, 3, 0], [4, 4, 4]])
    e_no = aliasing.shot_noise_expectation(n, 8, 4, False, shot)
    e_in = aliasing.shot_noise_expectation(n, 8, 4, True, shot)
    assert np.all(np.abs(e_in - 1.0) < np.abs(e_no - 1.0))


# --- direct summation (eq:deltaDS) and the accuracy ordering of Sec. 3.2 ------------------------------

def test_direct_sum_single_particle_is_plane_wave():
    x = np.array([[1.0, 2.0, 3.0]])
    d = direct.direct_modes(x, 8.0, 4)
    n = fourier.signed_index(4)
    u = x[0] * 4 / 8.0
    exp = np.exp(-2j * np.pi * (n[:, None, None] * u[0] + n[None, :, None] * u[1] + n[None, None, :] * u[2]) / 4)
    exp[0, 0, 0] -= 1.0
    assert np.max(np.abs(d - exp)) < 1e-14


def test_accuracy_ordering_against_direct_summation():
    # Sec. 3.2: relative to the alias-free direct summation, PCS+interlacing beats CIC+interlacing,
    # which beats plain CIC (power spectrum up to the Nyquist frequency).
    box, ng = 100.0, 16
    pos = catalogs.zeldovich(16, box, rms=2.0, seed=5)
    ds = direct.direct_modes(pos, box, ng)
    pk_ds, _, _ = power.power_spectrum(ds, box)

    def err(p, inter):
        r1 = assign.assign(pos, box, ng, p)
        r2 = assign.assign(pos, box, ng, p, shift=True) if inter else None
        pk, _, _ = power.power_spectrum(fourier.density_modes(r1, p, r2), box)
        return np.max(np.abs(pk / pk_ds - 1.0))

    e_cic, e_cic_i, e_pcs_i = err(2, False), err(2, True), err(4, True)
    assert e_pcs_i < e_cic_i < e_cic


def test_direct_sum_of_lattice_particles_is_the_dft_of_their_counts():
    # eq:deltaDS with every particle on a grid node (x = j H) is the discrete Fourier transform of the
    # node counts, computed here by numpy's FFT: pins the sign, the 2 pi / L scale and the signed index.
    rng = np.random.default_rng(31)
    ng, box = 8, 40.0
    nodes = rng.integers(0, ng, size=(300, 3))
    w = rng.uniform(0.5, 2.0, 300)
    counts = np.zeros((ng, ng, ng))
    np.add.at(counts, tuple(nodes.T), w)
    expect = np.fft.fftn(counts) / w.sum()
    expect[0, 0, 0] -= 1.0
    d = direct.direct_modes(nodes * (box / ng), box, ng, weights=w)
    assert np.max(np.abs(d - expect)) < 1e-13


def test_direct_sum_translation_and_hermitian_symmetry():
    # A rigid shift s of every particle multiplies delta(n != 0) by exp(-i k.s); delta(-n) = conj
    # delta(n) for any integer n, inside the grid or not (eq:deltaDS is not periodic in n).
    box = 50.0
    pos = catalogs.poisson(200, box, seed=33)
    nv = np.array([[1, 2, 3], [-4, 0, 5], [8, -8, 1], [13, 7, -9], [0, 0, 16]])
    s = np.array([3.3, -1.25, 7.0])
    d0 = direct.direct_modes_at(pos, box, nv)
    d1 = direct.direct_modes_at(np.mod(pos + s, box), box, nv)
    assert np.max(np.abs(d1 - d0 * np.exp(-2j * np.pi * (nv @ s) / box))) < 1e-13
    assert np.max(np.abs(direct.direct_modes_at(pos, box, -nv) - np.conj(d0))) < 1e-14


def test_direct_sum_poisson_expectation():
    # eq:ds2pcf with P = 0: for N iid uniform particles E|delta(n)|^2 = 1/N at every n != 0.
    box, npart = 100.0, 400
    nv = np.stack(np.meshgrid(np.arange(1, 9), np.arange(-4, 4), np.arange(0, 8), indexing="ij"), -1).reshape(-1, 3)
    acc = 0.0
    for seed in range(6):
        acc += np.mean(np.abs(direct.direct_modes_at(catalogs.poisson(npart, box, seed=40 + seed), box, nv)) ** 2)
    assert abs(acc / 6 * npart - 1.0) < 0.1  # 3072 exponential variates: std 1.8 %


def test_half_complex_cross_power_equals_full_grid_power_for_a_real_grid():
    # Without interlacing the window-corrected grid density is exactly Hermitian on the signed full
    # grid (G periodic, W even), so the half-complex sum with multiplicities reproduces the full-grid
    # bins of the Sec. 2.2 estimator, mode counts included.
    box, ng = 80.0, 12
    pos = catalogs.zeldovich(12, box, rms=3.0, seed=34)
    d = fourier.density_modes(assign.assign(pos, box, ng, 3), 3)
    pk, ke, cnt = power.power_spectrum(d, box)
    pk2, ke2, cnt2 = power.cross_power_half(d[:, :, : ng // 2 + 1], d[:, :, : ng // 2 + 1], box)
    assert np.array_equal(cnt, cnt2)
    assert np.max(np.abs(pk2 - pk) / pk) < 1e-12
    assert np.max(np.abs(ke2 - ke) / ke) < 1e-13


def test_half_complex_direct_power_by_enumerating_the_mode_set():
    # The direct-summation power over the stored modes and their partners -n, by brute force: list the
    # vectors, evaluate eq:deltaDS at each, bin by rounding |n| to the nearest integer in floating point.
    box, ng = 60.0, 6
    pos = catalogs.zeldovich(6, box, rms=4.0, seed=35)
    full = direct.direct_modes(pos, box, ng)
    half = full[:, :, : ng // 2 + 1]
    pk, ke, cnt = power.cross_power_half(half, half, box)
    n = fourier.signed_index(ng)
    vecs = []
    for ix, iy, iz in itertools.product(range(ng), range(ng), range(ng // 2 + 1)):
        v = (n[ix], n[iy], n[iz])
        if v == (0, 0, 0):
            continue
        vecs.append(v)
        if 0 < iz < ng // 2:
            vecs.append((-v[0], -v[1], -v[2]))
    vecs = np.array(vecs)
    p_modes = box ** 3 * np.abs(direct.direct_modes_at(pos, box, vecs)) ** 2
    b = np.floor(np.sqrt(np.sum(vecs.astype(np.float64) ** 2, axis=1)) + 0.5).astype(int) - 1
    for k in range(ng // 2):
        sel = b == k
        assert cnt[k] == sel.sum()
        assert abs(pk[k] - p_modes[sel].mean()) < 1e-12 * pk[k]
    # the conjugate pair has the same |delta|^2, but a partner outside the signed grid is a new mode
    assert len(vecs) == ng ** 3 - 1


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("interlace", [False, True])
def test_fres_3d_is_the_poisson_shot_noise_excess(p, interlace):
    # eq:Pknoint with P = 0: E[P(n)] n_bar = sum_m theta_m |W(k - m k_s)|^2 / |W(k)|^2 = 1 + F_res(n); the
    # expectation is summed as truncated sinc^{2p} image sums, F_res through the Hurwitz-zeta forms
    rng = np.random.default_rng(61)
    ng = 32
    n = rng.integers(-16, 16, (60, 3))
    n = n[np.abs(n).max(axis=1) >= 6]  # away from k = 0, where 1 + F_res - 1 loses its digits
    e = aliasing.shot_noise_expectation(n, ng, p, interlace, 1.0, mmax=4000)
    f = aliasing.fres_3d(n, ng, p, interlace)
    assert np.max(np.abs(e - 1.0 - f) / (1.0 + f)) < 2e-10


def test_fres_3d_brute_force_image_sum():
    # the definition summed directly over a cube of images |m_i| <= 12 (PCS terms fall as |m|^-8: the
    # truncated tail is below 1e-6 of F_res even where the interlacing leaves only |m| >= 2 images)
    ng, p, mmax = 16, 4, 12
    m = np.arange(-mmax, mmax + 1)
    M = np.stack(np.meshgrid(m, m, m, indexing="ij"), -1).reshape(-1, 3)
    M = M[np.any(M != 0, axis=1)]
    for n in ([1, 0, 0], [3, 2, 1], [8, -8, 5], [-8, -8, -8], [5, 0, -7]):
        x = np.array(n, dtype=np.float64) / ng
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.where(M == 0, 1.0, (x[None, :] / (x[None, :] - M)) ** (2 * p))
        terms = np.prod(g, axis=1)
        theta = (M.sum(axis=1) % 2 == 0).astype(float)
        for inter, th in ((False, 1.0), (True, theta)):
            ref = np.sum(th * terms)
            got = aliasing.fres_3d(np.array([n]), ng, p, inter)[0]
            assert abs(got - ref) <= 1e-6 * ref


def test_fres_3d_on_an_axis_is_the_one_dimensional_form():
    # eq:res1Dnoi / eq:res1Di are F_res along a grid axis
    ng = 64
    k = np.arange(1, 33)
    n = np.stack([k, 0 * k, 0 * k], 1)
    for p in (1, 2, 4):
        for inter in (False, True):
            got = aliasing.fres_3d(n, ng, p, inter)
            ref = aliasing.fres_1d(k / ng, p, inter, mmax=200000)
            assert np.max(np.abs(got - ref) / ref) < (2e-5 if p == 1 else 1e-10)


# --- bispectrum (eq:Best, eq:Best2, eq:VBest) ----------------------------------------------------------

def test_bispectrum_fft_form_equals_brute_force():
    box, ng = 50.0, 12
    pos = catalogs.zeldovich(12, box, rms=3.0, seed=8)
    r1 = assign.assign(pos, box, ng, 4)
    r2 = assign.assign(pos, box, ng, 4, shift=True)
    delta = fourier.density_modes(r1, 4, r2)
    b_fft, c_fft = bispectrum.bispectrum_fft(delta, box, 1, 1, 3)
    b_bf, c_bf = bispectrum.bispectrum_brute(delta, box, 1, 1, 3)
    assert np.array_equal(c_fft, c_bf)
    ok = c_bf > 0
    assert ok.sum() >= 6
    assert np.max(np.abs(b_fft[ok] / b_bf[ok] - 1.0)) < 1e-10


def test_bispectrum_single_triangle():
    # A field with only the modes q1, q2, q3 = -q1 - q2 (and their partners) of unit amplitude:
    # the triple product picks exactly the closed triangle.
    ng, box = 12, 1.0
    delta = np.zeros((ng, ng, ng), dtype=complex)
    for q in ([1, 0, 0], [0, 2, 0], [-1, -2, 0]):
        delta[tuple(np.mod(q, ng))] = 1.0
        delta[tuple(np.mod(-np.array(q), ng))] = 1.0
    b, c = bispectrum.bispectrum_fft(delta, box, 0, 1, 3)
    tri = bispectrum.triangles(3)
    t = tri.index((2, 2, 1))  # |q| = 1, 2, sqrt(5): shells 1, 2, 2 in 0-based shells of width 1
    # triplets in that bin: (q2, q3) ordered pairs from the two |q| in [2,3) modes and their partners
    assert c[t] > 0
    # sum over triplets of delta delta delta = number of closed triplets using our modes
    s_expected = 2 * 2  # (q1,q2,q3) and the negated triangle, each counted with the 2 orderings of s2=s3
    assert abs(b[t] * c[t] - s_expected) < 1e-9


def test_triangle_list_size():
    # 16 shells of width 4 k_f (up to k_N/2 at N_G = 256): the reading s1 <= s2 + s3 + 1 gives 508.
    assert len(bispectrum.triangles(16)) == 508


# --- adjoint -----------------------------------------------------------------------------------------

def test_adjoint_matches_central_differences():
    box, ng, p = 20.0, 8, 4
    pos = catalogs.poisson(24, box, seed=21)
    rng = np.random.default_rng(22)
    dl = rng.standard_normal(ng // 2)

    def loss(x):
        r1 = assign.assign(x, box, ng, p)
        r2 = assign.assign(x, box, ng, p, shift=True)
        pk, _, _ = power.power_spectrum(fourier.density_modes(r1, p, r2), box)
        return float(np.dot(dl, pk))

    g = adjoint.position_gradient(pos, box, ng, p, dl)
    h = 1e-4
    for i in range(0, 24, 5):
        for a in range(3):
            xp = pos.copy(); xp[i, a] += h
            xm = pos.copy(); xm[i, a] -= h
            fd = (loss(xp) - loss(xm)) / (2 * h)
            assert abs(fd - g[i, a]) <= 1e-5 * max(1.0, np.max(np.abs(g))), (i, a, fd, g[i, a])


# --- residual factor (eq:res1Di, eq:res1Dnoi, eq:res_comp) ---------------------------------------------

@pytest.mark.parametrize("p", [2, 3, 4])
def test_fres_hurwitz_forms(p):
    x = np.array([0.1, 0.25, 0.4, 0.5])
    for inter in (False, True):
        assert np.max(np.abs(aliasing.fres_1d(x, p, inter) - aliasing.fres_1d_hurwitz(x, p, inter))) < 1e-9
    # eq:res_comp from the two truncated sums directly
    assert np.max(np.abs(aliasing.fres_1d(x, p, True) - aliasing.fres_1d(x / 2, p, False))) < 1e-12


def test_oracle_header_marks_test_infrastructure():
    assert "TEST INFRASTRUCTURE" in oracle.__doc__


def test_mode_counts_with_edges_from_zero_exclude_k0():
    # Bins whose lower edge is 0 must still leave out the n = 0 mode (delta(0) is not a fluctuation).
    ng = 6
    edges = np.array([0, 2, 4], dtype=np.int64)  # |n| in [0, 1) and [1, 2)
    _, _, cnt = power.power_spectrum(np.ones((ng, ng, ng), dtype=complex), 1.0, edges)
    assert cnt[0] == 0
    assert cnt[1] == 6 + 12 + 8  # |n| = 1, sqrt(2), sqrt(3)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("shift", [False, True])
def test_single_node_value_equals_the_scattered_grid(p, shift):
    # gather at one node (used for sampled full-size checks) against the scatter over all nodes,
    # including nodes whose stencils wrap around the periodic box
    ng = 10
    u = np.random.default_rng(90 + p).uniform(0.0, ng, size=(400, 3))
    w = np.random.default_rng(91).uniform(0.5, 1.5, size=400)
    rho = assign.assign_units(u, ng, p, weights=w, shift=shift)
    for node in [(0, 0, 0), (9, 0, 5), (3, 9, 9), (5, 5, 5), (9, 9, 9)]:
        assert assign.node_value(u, ng, p, node, weights=w, shift=shift) == pytest.approx(rho[node], rel=1e-12, abs=1e-14)


def test_single_node_value_closed_forms():
    # a particle on a node: W(0)^3 (PCS 2/3, TSC 3/4, CIC 1); half-way between nodes on x: PCS W(1/2) = 23/48
    u = np.array([[2.0, 3.0, 4.0]])
    assert assign.node_value(u, 8, 4, (2, 3, 4)) == pytest.approx((2.0 / 3.0) ** 3, rel=1e-15)
    assert assign.node_value(u, 8, 3, (2, 3, 4)) == pytest.approx(0.75 ** 3, rel=1e-15)
    assert assign.node_value(u, 8, 2, (2, 3, 4)) == pytest.approx(1.0, rel=1e-15)
    v = np.array([[2.5, 3.0, 4.0]])
    assert assign.node_value(v, 8, 4, (2, 3, 4)) == pytest.approx(23.0 / 48.0 * (2.0 / 3.0) ** 2, rel=1e-15)


# --- k_eff, the weighted shot noise and the bispectrum normalisation ---------------------------------

def test_keff_is_the_mean_wavenumber_of_the_enumerated_modes():
    # k_eff of a bin is the mean |k| of its modes, with k = k_f n and k_f = 2 pi / L (Sec. 2.2). Every
    # integer vector of the grid is listed one at a time, its |n| taken in floating point and its bin
    # found by rounding |n| to the nearest integer (the default bins are centred on b k_f); the mean of
    # 2 pi |n| / L per bin must equal the oracle's k_eff. The first two bins also have closed forms from
    # the number of ways r3(m) to write m as a sum of three squares (r3 = 6, 12, 8, 6, 24, 24 for
    # m = 1..6). Planted mistakes this fails: k_f = 1/L or pi/L, |k| from 4|n|^2 without the 1/4, a mode
    # set that leaves out the Nyquist planes.
    ng, box = 8, 7.3
    kf = 2.0 * math.pi / box
    sums, cnts = {}, {}
    rng_n = range(-ng // 2, ng // 2)
    for nx, ny, nz in itertools.product(rng_n, rng_n, rng_n):
        m2 = nx * nx + ny * ny + nz * nz
        if m2 == 0:
            continue
        r = math.sqrt(m2)
        b = int(math.floor(r + 0.5))
        if 1 <= b <= ng // 2:
            sums[b] = sums.get(b, 0.0) + kf * r
            cnts[b] = cnts.get(b, 0) + 1
    delta = np.random.default_rng(5).standard_normal((ng, ng, ng)) + 0j
    _, keff, cnt = power.power_spectrum(delta, box)
    for b in range(1, ng // 2 + 1):
        assert cnt[b - 1] == cnts[b]
        assert keff[b - 1] == pytest.approx(sums[b] / cnts[b], rel=1e-14)
    assert keff[0] == pytest.approx(kf * (6 * 1.0 + 12 * math.sqrt(2.0)) / 18, rel=1e-14)
    k2 = kf * (8 * math.sqrt(3.0) + 6 * 2.0 + 24 * math.sqrt(5.0) + 24 * math.sqrt(6.0)) / 62
    assert keff[1] == pytest.approx(k2, rel=1e-14)


def test_weighted_poisson_power_matches_weighted_shot_noise():
    # With fixed weights w_i on independent uniform positions, E|sum_i w_i e^{-i k.x_i}|^2 = sum_i w_i^2
    # for k != 0 (the cross terms average to zero), so after the division by sum w the window-corrected
    # power averages to V sum w^2 / (sum w)^2 times the same aliasing sum as the unweighted Poisson case
    # (eq:Pknoint, interlaced form). The level is taken from power.shot_noise(box, weights). The weights
    # are spread (coefficient of variation about 0.8), so V/N_P differs from the weighted level by
    # about 60 %. Planted mistakes this fails (each by many sigma): 1/nbar = V/N_P with the weights
    # ignored, sum w in place of (sum w)^2, (sum w^2)^2 in the numerator, a missing V.
    p, ng, box, npart, nseeds = 4, 8, 100.0, 400, 300
    w = np.random.default_rng(77).lognormal(0.0, 0.7, size=npart)
    shot_w = power.shot_noise(box, w)
    assert abs(shot_w / (box ** 3 / npart) - 1.0) > 0.3
    edges = power.default_edges(ng)
    b = power.bin_index(ng, edges)
    half = ng // 2
    sn = fourier.signed_index(ng)
    nvec = np.stack(np.meshgrid(sn, sn, sn, indexing="ij"), axis=-1)
    sel = b >= 0
    e_mode = aliasing.shot_noise_expectation(nvec[sel], ng, p, True, 1.0, mmax=3000) * shot_w
    cnt = np.bincount(b[sel], minlength=half)
    expect = np.bincount(b[sel], weights=e_mode, minlength=half) / cnt
    var_mode = np.bincount(b[sel], weights=e_mode ** 2, minlength=half) / cnt
    acc = np.zeros(half)
    for s in range(nseeds):
        pos = catalogs.poisson(npart, box, seed=5000 + s)
        r1 = assign.assign(pos, box, ng, p, weights=w)
        r2 = assign.assign(pos, box, ng, p, weights=w, shift=True)
        pk, _, _ = power.power_spectrum(fourier.density_modes(r1, p, r2), box, edges)
        acc += pk
    mean = acc / nseeds
    sigma = np.sqrt(var_mode / (cnt / 2.0) / nseeds)
    z = (mean - expect) / sigma
    assert np.max(np.abs(z)) < 4.5, z
    # subtracting the weighted shot noise leaves only the aliasing excess, a small fraction of it
    pk_sub, _, _ = power.power_spectrum(fourier.density_modes(r1, p, r2), box, edges, subtract=shot_w)
    assert np.allclose(pk_sub, pk - shot_w, rtol=0, atol=1e-9 * shot_w)


def test_poisson_bispectrum_is_the_squared_shot_noise():
    # For independent uniform positions (P = B = 0) only the shot-noise terms of B_tot (Sec. 4.1)
    # remain: with delta_q = (1/N) sum_i e^{-i q.x_i}, a closed triplet q1 + q2 + q3 = 0 of non-zero
    # modes averages to E[delta_q1 delta_q2 delta_q3] = N / N^3 (only i = j = l survives), so the
    # estimator of eq:Best, V^2 times the mean over the triplets, averages to (V/N)^2 = 1/nbar^2 at
    # low k (the grid's images change it by far less than the statistical error here). Planted
    # mistakes this fails: V in place of V^2 (box = 37, a factor 5e4), a missing or squared N_c, a
    # triplet count off by a factor, a sign flip of the triple product.
    ng, box, npart, nseeds, p = 12, 37.0, 200, 200, 4
    nbar_inv2 = (box ** 3 / npart) ** 2
    tri = bispectrum.triangles(3)
    acc = np.zeros(len(tri))
    acc2 = np.zeros(len(tri))
    counts = None
    for s in range(nseeds):
        pos = catalogs.poisson(npart, box, seed=9000 + s)
        r1 = assign.assign(pos, box, ng, p)
        r2 = assign.assign(pos, box, ng, p, shift=True)
        delta = fourier.density_modes(r1, p, r2)
        bk, counts = bispectrum.bispectrum_fft(delta, box, 1, 1, 3)
        acc += bk / nbar_inv2
        acc2 += (bk / nbar_inv2) ** 2
    ok = counts > 0
    assert ok.sum() >= 6
    mean = acc / nseeds
    err = np.sqrt(np.maximum(acc2 / nseeds - mean ** 2, 0.0) / nseeds)
    z = (mean[ok] - 1.0) / err[ok]
    assert np.max(np.abs(z)) < 4.5, (mean, err)
    assert np.all(np.abs(mean[ok] - 1.0) < 0.25)
