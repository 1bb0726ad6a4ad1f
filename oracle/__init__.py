"""FP64 CPU oracle for the Fourier-space estimators of Sefusatti, Crocce, Scoccimarro & Couchman,
"Accurate Estimators of Correlation Functions in Fourier Space" (arXiv:1512.07295).

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct restatement of what the
estimator pipeline computes, written in NumPy/SciPy in double precision. It shares no code with the
CUDA library in ``paper_1512_07295_gb300`` and imports nothing from it. Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may
import it; the product path never does.

Modules (each function cites the section / equation of the paper it follows):

- ``bspline``   : real-space B-spline kernels W^(p) (Sec. 2.3) and their Fourier windows (eq:intkerFT).
- ``assign``    : mass assignment of particles to a periodic grid, optionally shifted by H/2
                  (eq:delgrid; interlaced grid of Sec. 3.1).
- ``fourier``   : grid FFT, window deconvolution (eq:windowcorrection) and the interlacing combine
                  (eq:intdelta) over every mode of the full N_G^3 grid.
- ``power``     : k-shell binning of V|delta(n)|^2 into P(k) with exact integer mode counts (Sec. 2.2).
- ``bispectrum``: shell-filter / inverse-FFT / triple-product estimator (eq:Best2, eq:IntI), its
                  brute-force definition (eq:Best) and exact triangle counts (eq:VBest).
- ``adjoint``   : analytic gradient of a loss on P(k) with respect to particle positions.
- ``direct``    : direct-summation (alias-free) Fourier coefficients (eq:deltaDS).
- ``aliasing``  : aliasing sums of the Poisson shot noise (eq:Pknoint and its interlaced form) and
                  the residual factor F_res (eq:Fres, eq:res1Di, eq:res1Dnoi).

Conventions (where the paper is silent or inconsistent, each module states the reading it takes):
delta_n = (1/N_c) sum_j delta_j exp(-2 pi i n.j/N_G); P = V |delta_n|^2; mode vector n in signed
convention n_i in [-N_G/2, N_G/2); grid 2 samples the particles shifted by +H/2 on every axis and is
combined with phase exp(+i pi (n_x+n_y+n_z)/N_G).
"""

from . import bspline, assign, fourier, power, bispectrum, adjoint, direct, aliasing  # noqa: F401
