"""Pin of the FFT-step oracle (oracle/enkf_fft.py) to the explicit-DFT oracle (oracle/enkf.py).

The full-size whole-array GPU check uses oracle/enkf_fft.py (numpy's FP64 real FFT as the transform
step, members streamed one field at a time).  On small grids it must give the explicit-DFT oracle's
covariance tables and analysis to FP64 rounding, for 1-4 blocks with 1-2 observed, odd and even
widths, flat and 1/|k| rhat, and a zero denominator (rhat = 0 with equal members of an observed
block), so that a dropped term, a wrong conjugate or a transposed table would fail here.
"""

import numpy as np
import pytest

from oracle import enkf, enkf_fft
from synth import fields


@pytest.mark.parametrize("ny,nx,N,observed", [(16, 24, 5, [1]), (12, 16, 4, [1, 0, 0]),
                                              (16, 16, 6, [1, 1, 0, 0]), (24, 12, 3, [0, 1, 1])])
def test_fft_path_matches_explicit_dft(ny, nx, N, observed):
    M = len(observed)
    spectra = [fields.matern32_spectrum(ny, nx, 1.5 + b, 1.0) for b in range(M)]
    n_obs = int(np.sum(observed))
    kk = fields.radial_wavenumber_half(ny, nx)
    rh = np.stack([(0.1 + 0.05 * i) / np.maximum(kk, 1.0) for i in range(n_obs)])
    p = fields.make_problem(ny, nx, N, spectra, observed, rh, seed=900 + ny + nx, rho=0.5)
    ens = p.ensemble.astype(np.float64)
    mean, auto, cross = enkf_fft.covariance_sums(lambda j, k: ens[j, k], M, N, observed)
    tab = enkf.spectrum_to_tables(enkf.estimate_spectrum(ens, observed), observed)
    obs = [int(i) for i in np.flatnonzero(observed)]
    un = [int(i) for i in np.flatnonzero(np.logical_not(observed))]
    parts = [auto[o].ravel() for o in obs]
    for o in obs:
        for j in un:
            h = cross[(j, o)]
            parts.append(np.stack([h.real, h.imag], axis=-1).ravel())
    got = np.concatenate(parts)
    assert np.abs(got - tab).max() <= 1e-12 * np.abs(tab).max()
    g = enkf_fft.gains(auto, cross, {o: p.rhat[i] for i, o in enumerate(obs)})
    ref = enkf.analyze(p.ensemble, p.data, p.perturbations, p.rhat, observed)
    for k in range(N):
        ua = enkf_fft.analysis_of_member(k, lambda j, kk_: ens[j, kk_], M, observed, p.data,
                                         lambda kk_, i: p.perturbations[kk_, i], g)
        assert np.abs(ua - ref[:, k]).max() <= 1e-11 * np.abs(ref[:, k]).max()


def test_fft_path_zero_denominator_keeps_forecast():
    p = fields.make_config2(ny=16, nx=16, N=4)
    o = int(np.flatnonzero(p.observed)[0])
    p.ensemble[o, :] = p.ensemble[o, 0]
    p.rhat[:] = 0.0
    ens = p.ensemble.astype(np.float64)
    _, auto, cross = enkf_fft.covariance_sums(lambda j, k: ens[j, k], p.M, p.N, p.observed)
    g = enkf_fft.gains(auto, cross, {o: p.rhat[0]})
    for k in range(p.N):
        ua = enkf_fft.analysis_of_member(k, lambda j, kk: ens[j, kk], p.M, p.observed, p.data,
                                         lambda kk, i: p.perturbations[kk, i], g)
        np.testing.assert_array_equal(ua, ens[:, k])
