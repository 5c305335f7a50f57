"""Pins of the FP64 oracle against closed forms, brute force and invariants (CPU only).

Each test ties the oracle to something other than itself: the DFT's closed
forms and a library FFT, the dense sample covariance (Sec. 2), the dense EnKF
solve of eq. (enkf)/(multi-enkf), a hand-derived worked example, statistical
convergence of eq. (dii) to the generating spectrum, and invariances.
"""

import json
import os

import numpy as np
import pytest

from oracle import dense, dft, enkf
from synth import fields

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(s):
    return np.random.default_rng(s)


# ---------------------------------------------------------------- the DFT
def test_dft_closed_forms():
    ny, nx = 6, 8
    u = np.zeros((ny, nx))
    u[0, 0] = 1.0
    np.testing.assert_allclose(dft.fft2(u), np.full((ny, nx), 1 / np.sqrt(ny * nx)), atol=1e-15)
    k0 = 3
    x = np.arange(nx)
    u = np.tile(np.cos(2 * np.pi * k0 * x / nx), (ny, 1))
    U = dft.fft2(u)
    ref = np.zeros((ny, nx), complex)
    ref[0, k0] = ref[0, nx - k0] = np.sqrt(ny * nx) / 2
    np.testing.assert_allclose(U, ref, atol=1e-13)


@pytest.mark.parametrize("n", [4, 6, 12, 16])
def test_dft_unitary_and_library(n):
    F = dft.dft_matrix(n)
    np.testing.assert_allclose(F @ F.conj().T, np.eye(n), atol=1e-13)
    u = _rng(n).standard_normal((3, n, 2 * n))
    np.testing.assert_allclose(dft.fft2(u), np.fft.fft2(u, norm="ortho"), atol=1e-12)
    np.testing.assert_allclose(dft.ifft2(dft.fft2(u)).real, u, atol=1e-12)


def test_dft_coefficients_sampling():
    u = _rng(1).standard_normal((2, 12, 16))
    full = np.fft.fft2(u, norm="ortho")
    ks = [(0, 0), (3, 5), (11, 15), (6, 8), (1, 0)]
    got = dft.coefficients(u, ks)
    ref = np.stack([full[..., a, b] for a, b in ks], axis=-1)
    np.testing.assert_allclose(got, ref, atol=1e-12)


# ------------------------------------------------------- eq. (dii) / cross
@pytest.mark.parametrize("ny,nx,N", [(4, 4, 3), (8, 8, 5), (6, 12, 4)])
def test_chat_equals_diag_FCnF(ny, nx, N):
    rng = _rng(ny * 100 + nx)
    ens = rng.standard_normal((3, N, ny, nx)) + 5.0
    spec = enkf.estimate_spectrum(ens, [1, 0, 1])
    for o in (0, 2):
        C = dense.sample_covariance(ens[o], ens[o])
        np.testing.assert_allclose(spec.auto[o], dense.freq_diagonal(C, ny, nx).real, atol=1e-12)
        C1 = dense.sample_covariance(ens[1], ens[o])
        np.testing.assert_allclose(spec.cross[(1, o)], dense.freq_diagonal(C1, ny, nx), atol=1e-12)


def test_printed_conjugation_is_the_transposed_block():
    """The formula as printed gives diag(F C^(oj) F*), not diag(F C^(jo) F*)."""
    ny, nx, N = 4, 6, 4
    ens = _rng(7).standard_normal((2, N, ny, nx))
    printed = enkf.estimate_spectrum(ens, [1, 0], printed_form=True).cross[(1, 0)]
    C10 = dense.sample_covariance(ens[1], ens[0])
    assert np.max(np.abs(printed - dense.freq_diagonal(C10, ny, nx))) > 1e-3
    np.testing.assert_allclose(printed, dense.freq_diagonal(C10.T, ny, nx), atol=1e-12)


def test_parseval_and_constant_invariance():
    ny, nx, N = 8, 10, 6
    ens = _rng(3).standard_normal((1, N, ny, nx))
    c = enkf.estimate_spectrum(ens, [1]).auto[0]
    var = ens[0].var(axis=0, ddof=1)
    np.testing.assert_allclose(c.sum(), var.sum(), rtol=1e-12)
    c2 = enkf.estimate_spectrum(ens + 123.0, [1]).auto[0]
    np.testing.assert_allclose(c2, c, rtol=1e-9, atol=1e-12)


def test_chat_converges_to_generating_spectrum():
    """E chat = S and Var chat = S^2/(N-1) for complex modes: a chi-square check at N=400."""
    ny = nx = 16
    S = fields.se_spectrum(ny, nx, 2.0, 1.0)
    rng = _rng(11)
    N = 400
    ens = np.stack([fields.gaussian_field(S, rng.standard_normal((ny, nx))) for _ in range(N)])[None]
    c = enkf.estimate_spectrum(ens, [1]).auto[0]
    ratio = c / S
    # modes whose negative is a different wavenumber are complex: Var(ratio) = 1/(N-1)
    ky, kx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    self_conj = ((2 * ky) % ny == 0) & ((2 * kx) % nx == 0)
    r = ratio[~self_conj]
    assert abs(r.mean() - 1.0) < 4.0 / np.sqrt((N - 1) * r.size / 2)
    assert abs(r.std() * np.sqrt(N - 1) - 1.0) < 0.15
    # and the spread shrinks like 1/sqrt(N-1)
    small = enkf.estimate_spectrum(ens[:, :26], [1]).auto[0] / S
    assert 3.0 < small[~self_conj].std() / r.std() < 5.5


# -------------------------------------------- update vs dense eq. (enkf)
def _problem(ny, nx, M, N, observed, seed, rhat=None):
    rng = _rng(seed)
    ens = rng.standard_normal((M, N, ny, nx)) * np.arange(1, M + 1)[:, None, None, None]
    n_obs = int(np.sum(observed))
    data = rng.standard_normal((n_obs, ny, nx)) + 0.5
    pert = 0.3 * rng.standard_normal((N, n_obs, ny, nx))
    if rhat is None:
        rhat = np.full((n_obs, ny, nx // 2 + 1), 0.2)
    return ens, data, pert, rhat


@pytest.mark.parametrize(
    "ny,nx,M,N,observed,kinv",
    [
        (4, 4, 1, 3, [1], False),
        (4, 6, 3, 4, [1, 0, 0], False),
        (4, 4, 4, 5, [1, 1, 0, 0], True),
        (6, 4, 3, 3, [0, 1, 1], True),
    ],
)
def test_update_equals_dense_enkf(ny, nx, M, N, observed, kinv):
    rhat = None
    if kinv:
        kk = fields.radial_wavenumber_half(ny, nx)
        rhat = np.repeat((0.1 / np.maximum(kk, 1.0))[None], int(np.sum(observed)), axis=0)
    ens, data, pert, rhat = _problem(ny, nx, M, N, observed, 5 + ny + M, rhat)
    ua, parts = enkf.analyze(ens, data, pert, rhat, observed, return_parts=True)
    spec = parts["spectrum"]
    obs = [i for i in range(M) if observed[i]]
    r_full = {o: enkf.half_to_full(rhat[i], nx, False) for i, o in enumerate(obs)}
    ref = dense.dense_analyze(ens, data, pert, spec.auto, spec.cross, r_full, observed)
    np.testing.assert_allclose(ua, ref, atol=1e-10)
    assert parts["max_imag"] < 1e-10


def test_dense_update_with_bruteforce_covariance():
    """Feed the dense solve covariances taken from diag(F C_N F*) directly."""
    ny, nx, M, N = 4, 4, 3, 4
    observed = [1, 0, 1]
    ens, data, pert, rhat = _problem(ny, nx, M, N, observed, 21)
    auto = {o: dense.freq_diagonal(dense.sample_covariance(ens[o], ens[o]), ny, nx) for o in (0, 2)}
    cross = {(1, o): dense.freq_diagonal(dense.sample_covariance(ens[1], ens[o]), ny, nx) for o in (0, 2)}
    r_full = {o: enkf.half_to_full(rhat[i], nx, False) for i, o in enumerate((0, 2))}
    ref = dense.dense_analyze(ens, data, pert, auto, cross, r_full, observed)
    np.testing.assert_allclose(enkf.analyze(ens, data, pert, rhat, observed), ref, atol=1e-10)


def test_rhat_limits():
    ny, nx, M, N = 6, 8, 2, 4
    ens, data, pert, _ = _problem(ny, nx, M, N, [1, 0], 9)
    big = np.full((1, ny, nx // 2 + 1), 1e30)
    ua = enkf.analyze(ens, data, pert, big, [1, 0])
    assert np.max(np.abs(ua - ens)) < 1e-20 * np.max(np.abs(ens)) * 1e12
    zero = np.zeros((1, ny, nx // 2 + 1))
    ua0 = enkf.analyze(ens, data, np.zeros_like(pert), zero, [1, 0])
    for k in range(N):
        np.testing.assert_allclose(ua0[0, k], data[0], atol=1e-10)


def test_gain_zero_where_no_information():
    """chat + rhat == 0 at some wavenumber: the forecast is kept there."""
    ny, nx, N = 4, 4, 3
    ens = np.zeros((1, N, ny, nx))
    ens[0] += 2.0                               # identical members: chat == 0
    data = np.ones((1, ny, nx))
    rhat = np.zeros((1, ny, nx // 2 + 1))
    ua = enkf.analyze(ens, data, np.zeros((N, 1, ny, nx)), rhat, [1])
    np.testing.assert_allclose(ua, ens, atol=0)


def test_wiener_posterior_mean_with_true_spectrum():
    """Supplying the generating S with e = 0 gives the circulant Gaussian posterior mean."""
    ny, nx, N = 8, 8, 5
    S = fields.se_spectrum(ny, nx, 1.5, 1.0)
    rng = _rng(4)
    ens = np.stack([fields.gaussian_field(S, rng.standard_normal((ny, nx))) for _ in range(N)])[None]
    truth = fields.gaussian_field(S, rng.standard_normal((ny, nx)))
    r = 0.3
    data = (truth + np.sqrt(r) * rng.standard_normal((ny, nx)))[None]
    spec = enkf.Spectrum({0: S}, {})
    tables = enkf.spectrum_to_tables(spec, [1])
    ua = enkf.analyze(ens, data, np.zeros((N, 1, ny, nx)), np.full((1, ny, nx // 2 + 1), r), [1],
                      spectrum=tables)
    # covariance function from a library inverse FFT, dense conditioning by scipy
    import scipy.linalg as sl
    c = np.fft.ifft2(S).real                    # c(h) = (1/G) sum_k S(k) exp(2 pi i k.h)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    P = np.stack([yy.ravel(), xx.ravel()], 1)
    d = (P[:, None, :] - P[None, :, :]) % np.array([ny, nx])
    Sigma = c[d[..., 0], d[..., 1]]
    m = ens[0].mean(axis=0).ravel()
    post = m + Sigma @ sl.solve(Sigma + r * np.eye(ny * nx), data[0].ravel() - m)
    np.testing.assert_allclose(ua[0].mean(axis=0).ravel(), post, atol=1e-10)


def test_cyclic_shift_equivariance():
    ny, nx, M, N = 6, 8, 3, 4
    observed = [0, 1, 1]
    kk = fields.radial_wavenumber_half(ny, nx)
    rhat = np.repeat((0.1 / np.maximum(kk, 1.0))[None], 2, axis=0)
    ens, data, pert, rhat = _problem(ny, nx, M, N, observed, 13, rhat)
    ua = enkf.analyze(ens, data, pert, rhat, observed)
    sh = (2, 3)
    r = lambda a: np.roll(a, sh, axis=(-2, -1))  # noqa: E731
    ua_s = enkf.analyze(r(ens), r(data), r(pert), rhat, observed)
    np.testing.assert_allclose(ua_s, r(ua), atol=1e-11)


def test_half_full_tables_roundtrip():
    ny, nx = 6, 8
    ens = _rng(2).standard_normal((3, 4, ny, nx))
    spec = enkf.estimate_spectrum(ens, [1, 1, 0])
    t = enkf.spectrum_to_tables(spec, [1, 1, 0])
    K = ny * (nx // 2 + 1)
    assert t.size == 2 * K + 2 * 2 * K
    back = enkf.tables_to_spectrum(t, [1, 1, 0], ny, nx)
    for o in (0, 1):
        np.testing.assert_allclose(back.auto[o], spec.auto[o], atol=1e-13)
        np.testing.assert_allclose(back.cross[(2, o)], spec.cross[(2, o)], atol=1e-13)


# ---------------------------------------------------------- worked example
def test_golden_two_block_shift():
    g = json.load(open(os.path.join(GOLDEN, "two_block_shift.json")))
    ens = np.array(g["ensemble"], float)
    data = np.array(g["data"], float)
    pert = np.array(g["perturbations"], float)
    rhat = np.full((1, g["ny"], g["nx"] // 2 + 1), g["rhat"])
    ua, parts = enkf.analyze(ens, data, pert, rhat, g["observed"], return_parts=True)
    np.testing.assert_allclose(ua, np.array(g["analysis"], float), atol=1e-13)
    spec = parts["spectrum"]
    np.testing.assert_allclose(enkf.full_to_half(spec.auto[0]), g["chat11_half"], atol=1e-14)
    c21 = enkf.full_to_half(spec.cross[(1, 0)])
    np.testing.assert_allclose(c21.real, g["chat21_half_re"], atol=1e-14)
    np.testing.assert_allclose(c21.imag, g["chat21_half_im"], atol=1e-14)


# --------------------------------------------------- planted mistakes fail
def _mutants():
    def no_mean(ens):
        return dft.fft2(np.asarray(ens, float))

    def divide_by_N(a):
        return np.sum(np.abs(a) ** 2, axis=0) / a.shape[0]

    def transposed_cross(aj, ao, printed_form=False):
        return np.sum(np.conj(aj) * ao, axis=0) / (aj.shape[0] - 1)

    orig_gains = enkf.gains

    def gain_without_rhat(spec, r_full, observed):
        return orig_gains(spec, {o: 0.0 * r for o, r in r_full.items()}, observed)

    def gain_without_inverse(spec, r_full, observed):
        g = orig_gains(spec, r_full, observed)
        return {key: v * (spec.auto[key[1]] + r_full[key[1]]) for key, v in g.items()}

    return {
        "anomaly_spectra": no_mean,
        "spectral_variance": divide_by_N,
        "spectral_cross": transposed_cross,
        "gains:rhat": gain_without_rhat,
        "gains:inverse": gain_without_inverse,
    }


@pytest.mark.parametrize("name", sorted(_mutants()))
def test_planted_oracle_mistakes_are_caught(name, monkeypatch):
    """Each planted mistake in the oracle fails the golden example or a brute-force pin."""
    mut = _mutants()[name]
    monkeypatch.setattr(enkf, name.split(":")[0], mut)
    caught = False
    try:
        test_golden_two_block_shift()
    except AssertionError:
        caught = True
    for case in [(4, 6, 3, 4, [1, 0, 0], False), (4, 4, 4, 5, [1, 1, 0, 0], True)]:
        try:
            test_chat_equals_diag_FCnF(4, 6, 4) if name != "gains:rhat" else None
            test_update_equals_dense_enkf(*case)
        except AssertionError:
            caught = True
    ens = _rng(8).standard_normal((2, 4, 4, 6)) + 3.0
    try:
        spec = enkf.estimate_spectrum(ens, [1, 0])
        C = dense.sample_covariance(ens[0], ens[0])
        np.testing.assert_allclose(spec.auto[0], dense.freq_diagonal(C, 4, 6).real, atol=1e-10)
        C1 = dense.sample_covariance(ens[1], ens[0])
        np.testing.assert_allclose(spec.cross[(1, 0)], dense.freq_diagonal(C1, 4, 6), atol=1e-10)
    except AssertionError:
        caught = True
    assert caught, name
