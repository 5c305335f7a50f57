"""Pins of the seeded spectral perturbations (oracle/perturb.py): the generator's words are
uniform and stream-distinct, the normals have the right moments, e is real, and its
frequency-space covariance is diag(rhat) (e ~ N(0, F* diag(rhat) F), eq. enkf)."""

import numpy as np

from oracle import dft, enkf, perturb


def test_philox_words_uniform_and_distinct():
    n = 1 << 15
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n)
    key = np.tile(np.array([7, 0], dtype=np.uint32), (n, 1))
    w = perturb.philox4x32_10(ctr, key)
    assert len(np.unique(w[:, 0])) > n - 4            # no collisions beyond chance
    hist = np.bincount((w.ravel() >> 28).astype(np.int64), minlength=16)
    expected = w.size / 16
    chi2 = np.sum((hist - expected) ** 2 / expected)
    assert chi2 < 45.0                                 # 15 dof, p ~ 1e-4
    # another key gives other words; the same counter and key the same words
    w2 = perturb.philox4x32_10(ctr[:8], np.tile(np.array([8, 0], dtype=np.uint32), (8, 1)))
    assert not np.array_equal(w2, w[:8])
    np.testing.assert_array_equal(perturb.philox4x32_10(ctr[:8], key[:8]), w[:8])


def test_spectral_white_moments_and_hermitian_edges():
    ny, nx = 64, 48
    z = np.stack([perturb.spectral_white(ny, nx, 3, s) for s in range(64)])
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.02
    assert abs(np.mean(z)) < 0.02
    L = nx // 2
    for kx in (0, L):
        col = z[:, :, kx]
        np.testing.assert_array_equal(col[:, 1:ny // 2], np.conj(col[:, ny - 1:ny // 2:-1]))
        assert np.all(col[:, 0].imag == 0) and np.all(col[:, ny // 2].imag == 0)
    inner = z[:, :, 1:L]
    assert abs(np.mean(inner.real ** 2) - 0.5) < 0.02 and abs(np.mean(inner.real * inner.imag)) < 0.01


def test_perturbations_are_real_with_spectral_variance_rhat():
    ny, nx, N = 16, 24, 400
    kk = np.sqrt(np.minimum(np.arange(ny), ny - np.arange(ny))[:, None] ** 2 + np.arange(nx // 2 + 1)[None] ** 2)
    rhat = (0.1 / np.maximum(kk, 1.0))[None]
    e = perturb.perturbations(ny, nx, rhat, 99, N)
    assert e.shape == (N, 1, ny, nx)
    # e real by construction: the unitary inverse of the Hermitian spectrum has no imaginary part
    eh = np.sqrt(rhat[0]) * perturb.spectral_white(ny, nx, 99, 0)
    assert np.max(np.abs(dft.ifft2(enkf.half_to_full(eh, nx, hermitian=True)).imag)) < 1e-12
    # frequency-space variance of the draws equals rhat (relative standard error ~ 1/sqrt(N))
    spec = np.mean(np.abs(dft.fft2(e[:, 0])) ** 2, axis=0)
    ratio = enkf.full_to_half(spec) / rhat[0]
    assert abs(np.mean(ratio) - 1.0) < 0.02
    assert np.max(np.abs(ratio - 1.0)) < 6.0 / np.sqrt(N) * 2
    # point variance = mean of rhat over the full grid (Parseval)
    assert abs(np.var(e) / np.mean(enkf.half_to_full(rhat[0], nx, hermitian=False)) - 1.0) < 0.05


def test_streams_differ_and_repeat():
    a = perturb.perturbations(8, 8, np.full((2, 8, 5), 0.2), 5, 3)
    b = perturb.perturbations(8, 8, np.full((2, 8, 5), 0.2), 5, 3)
    np.testing.assert_array_equal(a, b)
    assert not np.allclose(a[0, 0], a[0, 1]) and not np.allclose(a[0, 0], a[1, 0])
    c = perturb.perturbations(8, 8, np.full((2, 8, 5), 0.2), 6, 3)
    assert not np.allclose(a, c)
