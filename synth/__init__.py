"""Seeded synthetic inputs for the FFT EnKF analysis step.

This package draws the forecast ensembles, truths, data, data perturbations and
spectral data variances that both the CUDA path and the CPU oracle consume.  It
holds none of the filter's arithmetic (no covariance estimate, no gain, no
update): it only synthesises stationary Gaussian random fields by spectral
filtering of white noise, the way the paper generates its random smooth
perturbations (Sec. 2.2, Fourier series with fast-decaying random coefficients).
"""

from .fields import (  # noqa: F401
    Problem,
    bf16_bits_to_f32,
    f32_to_bf16_bits,
    folded_wavenumbers,
    gaussian_field,
    make_config1,
    make_config2,
    make_config3,
    make_batched_items,
    make_problem,
    matern32_spectrum,
    powerlaw_spectrum,
    radial_wavenumber_half,
    se_spectrum,
)
