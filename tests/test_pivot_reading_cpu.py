"""CPU checks of the pivot form of eq. (dii) that the GPU uses (no mean field): with d_k = u_k - u_0,
s = (1/sqrt N) sum_{k>=1} d_k and D = F d, S = F s,

    sum_{k>=1} D_k D'_k* - S S'*  =  sum_k A_k A'_k*,   A_k = F(u_k - ubar),

for auto and cross spectra, and in FP32 the pivot form keeps the covariance of anomalies riding on a
large common mean to a few rounding errors.  numpy only: the identity is the reading, checked against
the oracle's spectrum estimate."""

import numpy as np

from oracle import enkf
from synth import fields


def _pivot_tables(u, dtype):
    """auto and cross sums of blocks 0 (observed) and 1 by the pivot form, in `dtype`."""
    M, N = u.shape[:2]
    u = u.astype(dtype)
    d = u[:, 1:] - u[:, :1]                                   # [M][N-1]
    s = d.sum(axis=1) / np.sqrt(N).astype(dtype)              # [M]
    D = np.fft.fft2(d, norm="ortho")
    S = np.fft.fft2(s, norm="ortho")
    auto = (np.abs(D[0]) ** 2).sum(axis=0) - np.abs(S[0]) ** 2
    cross = (D[1] * np.conj(D[0])).sum(axis=0) - S[1] * np.conj(S[0])
    return auto / (N - 1), cross / (N - 1)


def test_pivot_identity_matches_the_oracle_estimate():
    ny, nx, N = 16, 24, 6
    spectra = [fields.matern32_spectrum(ny, nx, 2.0, 1.0), fields.matern32_spectrum(ny, nx, 4.0, 1.0)]
    p = fields.make_problem(ny, nx, N, spectra, [1, 0], np.full((1, ny, nx // 2 + 1), 0.1), seed=31, rho=0.5)
    u = p.ensemble.astype(np.float64)
    auto, cross = _pivot_tables(u, np.float64)
    spec = enkf.estimate_spectrum(u, p.observed)
    tab = enkf.spectrum_to_tables(spec, p.observed)
    K = ny * (nx // 2 + 1)
    half = (slice(None), slice(0, nx // 2 + 1))
    np.testing.assert_allclose(auto[half].ravel(), tab[:K], rtol=0, atol=1e-12 * np.abs(tab[:K]).max())
    x = tab[K:].reshape(-1, 2)
    np.testing.assert_allclose(cross[half].ravel(), x[:, 0] + 1j * x[:, 1], rtol=0, atol=1e-12 * np.abs(x).max())


def test_pivot_form_keeps_digits_under_a_large_common_mean():
    """FP32, common mean 300, unit anomalies: the pivot form's auto and cross tables stay within 1e-6
    (relative L2) of the FP64 estimate of the same FP32 members."""
    ny, nx, N = 32, 32, 8
    S = fields.se_spectrum(ny, nx, 3.0, 1.0)
    p = fields.make_problem(ny, nx, N, [S, S], [1, 0], np.full((1, ny, nx // 2 + 1), 0.1), seed=5, rho=0.6,
                            mean=[300.0, 300.0])
    u = p.ensemble.astype(np.float64)                         # the FP32 members, exactly
    exact_a, exact_x = _pivot_tables(u, np.float64)
    piv_a, piv_x = _pivot_tables(u, np.float32)
    assert np.linalg.norm(piv_a - exact_a) / np.linalg.norm(exact_a) <= 1e-6
    assert np.linalg.norm(piv_x - exact_x) / np.linalg.norm(exact_x) <= 1e-6
