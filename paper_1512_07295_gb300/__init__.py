"""GB300-native Fourier-space estimators of arXiv:1512.07295 (Sefusatti, Crocce, Scoccimarro &
Couchman): B-spline mass assignment with interlacing, FFT, window deconvolution, P(k) shell binning
and the FFT bispectrum, as hand-written CUDA kernels for sm_103a behind a C ABI (``include/pk.h``).

``catalogs`` (seeded synthetic inputs) imports without the CUDA library; ``api`` loads it.
"""

__all__ = ["catalogs", "api"]
