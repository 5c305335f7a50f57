"""Pins of the sine-transform oracle (oracle/sine.py, Sec. 4's real sine FFT variant): the DST-I
matrix against its closed forms and SciPy's orthonormal DST-I, the spectra against the dense
sample covariance, the update against the dense EnKF solve of eq. (enkf) with the sine-diagonal
covariance, and against the periodic oracle on the odd extension of the grid."""

import numpy as np
import pytest

from oracle import dense, enkf, sine


def _problem(ny, nx, M, N, observed, seed, rhat=None):
    rng = np.random.default_rng(seed)
    ens = rng.standard_normal((M, N, ny, nx)) * np.arange(1, M + 1)[:, None, None, None] + 0.3
    ens = ens + 0.7 * ens[:1]
    n_obs = int(np.sum(observed))
    data = rng.standard_normal((n_obs, ny, nx)) + 0.5
    pert = 0.3 * rng.standard_normal((N, n_obs, ny, nx))
    if rhat is None:
        rhat = np.full((n_obs, ny - 2, nx - 2), 0.2)
    return ens, data, pert, rhat


def test_dst1_matrix_closed_forms():
    for m in (1, 2, 5, 16, 31):
        S = sine.dst1_matrix(m)
        np.testing.assert_allclose(S, S.T, atol=1e-15)
        np.testing.assert_allclose(S @ S, np.eye(m), atol=1e-13)
        # a sine mode with k0 half-periods is a spike of height sqrt((m+1)/2) at coefficient k0-1
        for k0 in (1, m):
            x = np.sin(np.pi * k0 * np.arange(1, m + 1) / (m + 1))
            ref = np.zeros(m)
            ref[k0 - 1] = np.sqrt((m + 1) / 2)
            np.testing.assert_allclose(S @ x, ref, atol=1e-12)


def test_dst1_matches_library_routine():
    scipy_fft = pytest.importorskip("scipy.fft")
    rng = np.random.default_rng(1)
    v = rng.standard_normal((7, 12))
    ref = scipy_fft.dst(scipy_fft.dst(v, type=1, norm="ortho", axis=0), type=1, norm="ortho", axis=1)
    np.testing.assert_allclose(sine.sine2(v), ref, atol=1e-12)


def _kron_sine(my, mx):
    return np.kron(sine.dst1_matrix(my), sine.dst1_matrix(mx))


def test_spectra_equal_dense_sample_covariance_diagonal():
    ny, nx, M, N = 6, 7, 3, 5
    observed = [1, 0, 1]
    ens, _, _, _ = _problem(ny, nx, M, N, observed, 3)
    auto, cross = sine.estimate(ens, observed)
    S = _kron_sine(ny - 2, nx - 2)
    inner = sine.interior(ens)
    for o in (0, 2):
        C = dense.sample_covariance(inner[o], inner[o])
        np.testing.assert_allclose(auto[o].ravel(), np.diag(S @ C @ S.T), atol=1e-12)
        C = dense.sample_covariance(inner[1], inner[o])
        np.testing.assert_allclose(cross[(1, o)].ravel(), np.diag(S @ C @ S.T), atol=1e-12)


@pytest.mark.parametrize("ny,nx,M,N,observed", [(5, 6, 1, 4, [1]), (6, 5, 3, 4, [1, 0, 0]),
                                                (5, 5, 3, 5, [1, 0, 1]), (6, 6, 4, 3, [0, 1, 1, 0])])
def test_update_equals_dense_enkf_solve(ny, nx, M, N, observed):
    """eq. (enkf) solved densely with C^(ab) = S diag(chat^(ab)) S (chat from the dense sample
    covariance), C^(o'o) = 0 between distinct observed blocks (Sec. 2.2) and R = S diag(rhat) S
    equals the per-wavenumber sine update; the boundary keeps the forecast."""
    my, mx = ny - 2, nx - 2
    rng = np.random.default_rng(ny * 10 + M)
    n_obs = int(np.sum(observed))
    ens, data, pert, _ = _problem(ny, nx, M, N, observed, 50 + M)
    rhat = 0.05 + rng.random((n_obs, my, mx))
    ua = sine.analyze(ens, data, pert, rhat, observed)
    S = _kron_sine(my, mx)
    inner = sine.interior(ens).reshape(M, N, -1)
    n = my * mx
    obs = [j for j in range(M) if observed[j]]

    def chat(a, b):
        return np.diag(S @ dense.sample_covariance(inner[a].reshape(N, my, mx), inner[b].reshape(N, my, mx)) @ S.T)

    C = np.zeros((M * n, M * n))
    for a in range(M):
        for b in range(M):
            if a != b and observed[a] and observed[b]:
                continue
            C[a * n:(a + 1) * n, b * n:(b + 1) * n] = S.T @ np.diag(chat(a, b)) @ S
    H = np.zeros((n_obs * n, M * n))
    for i, o in enumerate(obs):
        H[i * n:(i + 1) * n, o * n:(o + 1) * n] = np.eye(n)
    R = np.zeros((n_obs * n, n_obs * n))
    for i in range(n_obs):
        R[i * n:(i + 1) * n, i * n:(i + 1) * n] = S.T @ np.diag(rhat[i].ravel()) @ S
    K = C @ H.T @ np.linalg.inv(H @ C @ H.T + R)
    d = sine.interior(data).reshape(-1)
    for k in range(N):
        u = inner[:, k].reshape(-1)
        e = sine.interior(pert[k]).reshape(-1)
        ref = u + K @ (d + e - H @ u)
        np.testing.assert_allclose(sine.interior(ua[:, k]).reshape(-1), ref, atol=1e-10)
    np.testing.assert_array_equal(ua[..., 0, :], ens[..., 0, :])
    np.testing.assert_array_equal(ua[..., -1, :], ens[..., -1, :])
    np.testing.assert_array_equal(ua[..., :, 0], ens[..., :, 0])
    np.testing.assert_array_equal(ua[..., :, -1], ens[..., :, -1])


def _odd_extension(u):
    """Odd extension of the interior of u [..., ny, nx] to the period 2(ny-1) x 2(nx-1); the
    boundary nodes become the zero nodes of the extension."""
    ny, nx = u.shape[-2:]
    inner = u[..., 1:-1, 1:-1]
    col = np.concatenate([np.zeros(inner.shape[:-1] + (1,)), inner, np.zeros(inner.shape[:-1] + (1,)),
                          -inner[..., ::-1]], axis=-1)
    z = np.zeros(col.shape[:-2] + (1, col.shape[-1]))
    return np.concatenate([z, col, z, -col[..., ::-1, :]], axis=-2)


def _rhat_extension(rhat, ny, nx, fill=1.0):
    Py, Px = 2 * (ny - 1), 2 * (nx - 1)
    out = np.full(rhat.shape[:-2] + (Py, Px // 2 + 1), fill)
    for ky in range(Py):
        a = min(ky, Py - ky)
        if 1 <= a <= ny - 2:
            out[..., ky, 1:nx - 1] = rhat[..., a - 1, :]
    return out


@pytest.mark.parametrize("ny,nx,M,N,observed", [(5, 7, 1, 4, [1]), (7, 6, 3, 5, [1, 0, 1])])
def test_periodic_update_on_odd_extension(ny, nx, M, N, observed):
    """The periodic FFT EnKF applied to the odd extension of the grid, restricted to the interior,
    is the sine-transform EnKF: the DFT of an odd field is -S of its interior at the matching
    wavenumbers (zero on the lines k = 0, period/2), the gains are even, and the update stays odd."""
    ens, data, pert, _ = _problem(ny, nx, M, N, observed, 9)
    n_obs = int(np.sum(observed))
    rhat = 0.1 + np.random.default_rng(2).random((n_obs, ny - 2, nx - 2))
    ua = sine.analyze(ens, data, pert, rhat, observed)
    ext = enkf.analyze(_odd_extension(ens), _odd_extension(data), _odd_extension(pert),
                       _rhat_extension(rhat, ny, nx), observed)
    np.testing.assert_allclose(ext[..., 1:ny - 1, 1:nx - 1], sine.interior(ua), atol=1e-11)
    np.testing.assert_allclose(ext, _odd_extension(ext[..., :ny, :nx]), atol=1e-11)


def test_exact_data_and_infinite_noise_limits():
    ny, nx = 6, 8
    ens, data, pert, _ = _problem(ny, nx, 2, 4, [1, 0], 13)
    # rhat -> 0, e = 0: the observed interior equals the data where chat > 0 (all, for N >= 2 draws)
    ua = sine.analyze(ens, data, np.zeros_like(pert), np.zeros((1, ny - 2, nx - 2)), [1, 0])
    np.testing.assert_allclose(sine.interior(ua[0]), np.broadcast_to(sine.interior(data[0]), ua[0, :, 1:-1, 1:-1].shape),
                               atol=1e-10)
    # rhat -> infinity: the forecast is kept
    ua = sine.analyze(ens, data, pert, np.full((1, ny - 2, nx - 2), 1e30), [1, 0])
    assert np.max(np.abs(ua - ens)) < 1e-25
    # constant members: chat = 0 and rhat = 0 give gain 0 (0/0 rule)
    flat = np.repeat(ens[:, :1], 4, axis=1)
    ua = sine.analyze(flat, data, pert, np.zeros((1, ny - 2, nx - 2)), [1, 0])
    np.testing.assert_array_equal(ua, flat)
