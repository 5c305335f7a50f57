"""Pins of the denoiser oracle: finite-difference gradients, brute-force binning, interpolation."""

import numpy as np

from oracle import mlp


def test_param_count():
    assert mlp.param_count() == 33088


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init_params(1) + 0.05 * rng.standard_normal(mlp.param_count())
    X = rng.standard_normal((3, 256))
    Y = rng.standard_normal((3, 128))
    g = mlp.backward(theta, X, Y)
    h = 1e-6
    idx = rng.choice(theta.size, 60, replace=False)
    idx = np.concatenate([idx, [0, 256 * 64, theta.size - 1, theta.size - 128 - 5]])  # first W, first b, last b, last W
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(mlp.forward(tp, X)[0], Y) - mlp.loss(mlp.forward(tm, X)[0], Y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_gelu_closed_form():
    z = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    phi = np.array([0.0013498980, 0.1586552539, 0.5, 0.6914624613, 0.9772498681])   # normal CDF table
    np.testing.assert_allclose(mlp.gelu(z), z * phi, atol=1e-9)
    np.testing.assert_allclose(mlp.gelu_grad(0.0), 0.5, atol=1e-15)


def test_binning_bruteforce():
    ny, nx = 24, 40
    rng = np.random.default_rng(3)
    c = np.exp(rng.standard_normal((ny, nx // 2 + 1)))
    got = mlp.bin_log(c, ny, nx)
    w = np.sqrt(ny * ny + nx * nx) / 2 / 128
    sums = np.zeros(128)
    cnt = np.zeros(128)
    for y in range(ny):
        kyv = y if y <= ny // 2 else y - ny
        for x in range(nx // 2 + 1):
            b = min(127, int(np.floor(np.sqrt(kyv * kyv + x * x) / w)))
            sums[b] += np.log(c[y, x])
            cnt[b] += 1
    ref = np.where(cnt > 0, sums / np.maximum(cnt, 1), 0.0)
    np.testing.assert_allclose(got, ref, atol=1e-12)


def test_unbin_interpolates_linear_log_spectrum():
    ny = nx = 64
    kabs, _, centres = mlp.radial(ny, nx)
    out = -0.3 * centres + 1.0            # log spectrum linear in |k|
    S = mlp.unbin(out, ny, nx)
    inside = (kabs >= centres[0]) & (kabs <= centres[-1])
    np.testing.assert_allclose(np.log(S[inside]), -0.3 * kabs[inside] + 1.0, atol=1e-12)
    np.testing.assert_allclose(np.log(S[kabs < centres[0]]), out[0], atol=1e-12)


def test_adam_first_step_is_sign_times_lr():
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = mlp.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-5)


def test_bin_decisions_use_exact_integer_wavenumbers():
    """|k| on bin boundaries (|k|/w integer) must fall in the upper bin: 96 x 128 has w = 0.625."""
    kabs, b, centres = mlp.radial(96, 128)
    assert kabs[25, 0] == 25.0 and b[25, 0] == 40
    assert kabs[96 - 15, 20] == 25.0 and b[96 - 15, 20] == 40
