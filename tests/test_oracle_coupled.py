"""Pins of the coupled-observed-blocks oracle (oracle/coupled.py) against the dense EnKF
solve with the full stationary covariance, the neglect rule and closed forms."""

import numpy as np
import pytest

from oracle import coupled, dense, enkf
from synth import fields


def _problem(ny, nx, M, N, observed, seed, rhat=None):
    rng = np.random.default_rng(seed)
    ens = rng.standard_normal((M, N, ny, nx)) * np.arange(1, M + 1)[:, None, None, None]
    # correlate the blocks so that the observed cross-covariances matter
    ens = ens + 0.8 * ens[:1]
    n_obs = int(np.sum(observed))
    data = rng.standard_normal((n_obs, ny, nx)) + 0.5
    pert = 0.3 * rng.standard_normal((N, n_obs, ny, nx))
    if rhat is None:
        rhat = np.full((n_obs, ny, nx // 2 + 1), 0.2)
    return ens, data, pert, rhat


@pytest.mark.parametrize(
    "ny,nx,M,N,observed,kinv",
    [
        (4, 4, 2, 4, [1, 1], False),
        (4, 6, 3, 5, [1, 0, 1], False),
        (4, 4, 4, 5, [1, 1, 0, 0], True),
        (6, 4, 3, 3, [0, 1, 1], True),
    ],
)
def test_coupled_equals_dense_full_covariance(ny, nx, M, N, observed, kinv):
    """eq. (multi-enkf) with the full block covariance, solved densely, equals the
    per-wavenumber coupled update."""
    rhat = None
    if kinv:
        kk = fields.radial_wavenumber_half(ny, nx)
        rhat = np.repeat((0.1 / np.maximum(kk, 1.0))[None], int(np.sum(observed)), axis=0)
    ens, data, pert, rhat = _problem(ny, nx, M, N, observed, 31 + ny + M, rhat)
    ua, parts = coupled.analyze(ens, data, pert, rhat, observed, return_parts=True)
    obs = [i for i in range(M) if observed[i]]
    r_full = {o: enkf.half_to_full(rhat[i], nx, False) for i, o in enumerate(obs)}
    ref = dense.dense_analyze(ens, data, pert, parts["auto"], parts["cross"], r_full, observed,
                              neglect_observed_cross=False)
    np.testing.assert_allclose(ua, ref, atol=1e-10)
    # and it differs from the neglect rule when two blocks are observed and correlated
    if len(obs) == 2:
        assert np.max(np.abs(ua - enkf.analyze(ens, data, pert, rhat, observed))) > 1e-3


def test_bruteforce_covariance_tables():
    """The observed-pair cross tables equal diag(F C_N^(o'o) F*) of the dense sample covariance."""
    ny, nx, M, N = 4, 4, 3, 4
    observed = [1, 0, 1]
    ens, _, _, _ = _problem(ny, nx, M, N, observed, 5)
    auto, cross = coupled.estimate(ens, observed)
    for (a, o), c in cross.items():
        ref = dense.freq_diagonal(dense.sample_covariance(ens[a], ens[o]), ny, nx)
        np.testing.assert_allclose(c, ref, atol=1e-12)


def test_single_observed_block_reduces_to_spectral_enkf():
    ens, data, pert, rhat = _problem(6, 8, 3, 4, [0, 1, 0], 7)
    np.testing.assert_allclose(coupled.analyze(ens, data, pert, rhat, [0, 1, 0]),
                               enkf.analyze(ens, data, pert, rhat, [0, 1, 0]), atol=1e-12)


def test_zero_observed_cross_gives_the_neglect_rule():
    ens, data, pert, rhat = _problem(4, 6, 3, 4, [1, 1, 0], 9)
    observed = [1, 1, 0]
    auto, cross = coupled.estimate(ens, observed)
    cross[(0, 1)] = np.zeros_like(cross[(0, 1)])
    cross[(1, 0)] = np.zeros_like(cross[(1, 0)])
    r_full = {o: enkf.half_to_full(rhat[i], 6, False) for i, o in enumerate((0, 1))}
    K = coupled.gains(auto, cross, r_full, observed)
    spec = enkf.estimate_spectrum(ens, observed)
    g = enkf.gains(spec, r_full, observed)
    for o in (0, 1):
        np.testing.assert_allclose(K[(o, o)], g[(o, o)], atol=1e-14)
        np.testing.assert_allclose(K[(2, o)], g[(2, o)], atol=1e-14)
        np.testing.assert_allclose(K[(1 - o, o)], 0, atol=1e-14)


def test_bracket_inverse_regular_and_singular():
    rng = np.random.default_rng(3)
    B = rng.standard_normal((50, 2, 2)) + 1j * rng.standard_normal((50, 2, 2))
    A = B @ np.conj(np.swapaxes(B, -1, -2)) + 0.1 * np.eye(2)        # Hermitian positive definite
    np.testing.assert_allclose(coupled.bracket_inverse(A), np.linalg.inv(A), rtol=1e-10, atol=1e-12)
    v = rng.standard_normal((50, 2)) + 1j * rng.standard_normal((50, 2))
    R1 = v[:, :, None] * np.conj(v[:, None, :])                        # rank 1: pseudo-inverse
    np.testing.assert_allclose(coupled.bracket_inverse(R1), np.linalg.pinv(R1, rcond=1e-8), rtol=1e-8, atol=1e-12)
    np.testing.assert_array_equal(coupled.bracket_inverse(np.zeros((3, 2, 2), complex)), 0)


def test_rank_one_members_with_zero_rhat():
    """N = 2, rhat = 0: the bracket is rank 1 at every wavenumber; the pseudo-inverse rule
    keeps the update finite."""
    ens, data, pert, _ = _problem(4, 4, 2, 2, [1, 1], 11)
    rhat = np.zeros((2, 4, 3))
    ua = coupled.analyze(ens, data, np.zeros_like(pert), rhat, [1, 1])
    assert np.all(np.isfinite(ua))


def test_rhat_infinite_keeps_forecast():
    ens, data, pert, _ = _problem(4, 6, 3, 4, [1, 1, 0], 13)
    ua = coupled.analyze(ens, data, pert, np.full((2, 4, 4), 1e30), [1, 1, 0])
    assert np.max(np.abs(ua - ens)) < 1e-20 * np.max(np.abs(ens)) * 1e12
