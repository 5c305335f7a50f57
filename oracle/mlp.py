"""FP64 oracle of the learned spectral-variance denoiser (test infrastructure).

Not part of the paper's method: the paper motivates covariance estimation from a
very small ensemble (Sec. 2.1); the denoiser maps the radially binned log of the
N=5 estimate of eq. (dii) to that of a large ensemble.  Parity of trained
weights is unpinned (there is no reference network); what is pinned here is
the arithmetic: binning against a brute-force loop, the backward pass against
central finite differences, the interpolation against closed forms.

Binning: |k| = sqrt(k_y^2 + k_x^2) in integer units on the half spectrum
[ny][nx/2+1] (k_y folded), bin width w = k_max/128 with k_max = sqrt(ny^2+nx^2)/2,
bin b = min(127, floor(|k|/w)); a bin's value is the mean over its half-spectrum
entries of log(max(chat, 1e-30 max chat)).  Features: the 128 bin values minus
their mean, then log(max(centre_b, 1/2)) at the 128 bin centres (b + 1/2) w.
Network: 256 -> 64 -> 64 -> 64 -> 128, exact (erf) GELU after the hidden layers,
the output plus the removed mean is the predicted binned log spectrum.
Per-wavenumber spectrum: exp of the piecewise-linear interpolation in |k|
between bin centres (constant beyond the first and last centre).
Loss: mean squared error over bins and samples.
"""

from __future__ import annotations

from math import erf, sqrt

import numpy as np

N_BINS = 128
LAYERS = ((256, 64), (64, 64), (64, 64), (64, N_BINS))
FLOOR = 1e-30


def param_count() -> int:
    return sum(i * o + o for i, o in LAYERS)


def unpack(theta):
    """Flat parameter vector -> [(W [out][in], b [out])] in layer order."""
    theta = np.asarray(theta, dtype=np.float64)
    out, pos = [], 0
    for i, o in LAYERS:
        W = theta[pos:pos + i * o].reshape(o, i)
        pos += i * o
        b = theta[pos:pos + o]
        pos += o
        out.append((W, b))
    return out


def radial(ny: int, nx: int):
    j = np.arange(ny)
    ky = np.where(j <= ny // 2, j, j - ny).astype(np.float64)   # exact integer wavenumbers
    kx = np.arange(nx // 2 + 1, dtype=np.float64)
    kabs = np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
    w = sqrt(ny * ny + nx * nx) / 2.0 / N_BINS
    b = np.minimum(N_BINS - 1, np.floor(kabs / w)).astype(np.int64)
    centres = (np.arange(N_BINS) + 0.5) * w
    return kabs, b, centres


def bin_log(chat_half: np.ndarray, ny: int, nx: int) -> np.ndarray:
    """Mean of log(max(chat, FLOOR max chat)) per radial bin (128 values)."""
    c = np.asarray(chat_half, dtype=np.float64).reshape(ny, nx // 2 + 1)
    _, b, _ = radial(ny, nx)
    logc = np.log(np.maximum(c, FLOOR * c.max()))
    s = np.bincount(b.ravel(), weights=logc.ravel(), minlength=N_BINS)
    n = np.bincount(b.ravel(), minlength=N_BINS)
    return s / np.maximum(n, 1)


def features(binned: np.ndarray, ny: int, nx: int):
    """256 inputs and the removed mean."""
    _, _, centres = radial(ny, nx)
    mu = float(np.mean(binned))
    return np.concatenate([binned - mu, np.log(np.maximum(centres, 0.5))]), mu


def gelu(z):
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + np.vectorize(erf)(z / sqrt(2.0)))


def gelu_grad(z):
    z = np.asarray(z, dtype=np.float64)
    cdf = 0.5 * (1.0 + np.vectorize(erf)(z / sqrt(2.0)))
    pdf = np.exp(-0.5 * z * z) / sqrt(2.0 * np.pi)
    return cdf + z * pdf


def forward(theta, X):
    """X [B][256] -> outputs [B][128] and the cache for backward."""
    layers = unpack(theta)
    a = np.asarray(X, dtype=np.float64)
    cache = [a]
    zs = []
    for li, (W, b) in enumerate(layers):
        z = a @ W.T + b
        zs.append(z)
        a = gelu(z) if li < len(layers) - 1 else z
        cache.append(a)
    return a, (cache, zs)


def loss(pred, target) -> float:
    d = np.asarray(pred) - np.asarray(target)
    return float(np.mean(d * d))


def backward(theta, X, target):
    """Gradient of `loss` with respect to the flat parameter vector (analytic)."""
    layers = unpack(theta)
    pred, (acts, zs) = forward(theta, X)
    B = pred.shape[0]
    delta = 2.0 * (pred - target) / (B * pred.shape[1])
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        gW = delta.T @ acts[li]
        gb = delta.sum(axis=0)
        grads.append((gW, gb))
        if li > 0:
            delta = (delta @ W) * gelu_grad(zs[li - 1])
    grads.reverse()
    return np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


def unbin(out_log: np.ndarray, ny: int, nx: int) -> np.ndarray:
    """Per-wavenumber spectrum [ny][nx/2+1] from 128 binned log values."""
    kabs, _, centres = radial(ny, nx)
    return np.exp(np.interp(kabs, centres, np.asarray(out_log, dtype=np.float64)))


def adam(theta, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) with bias correction; returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed: int = 0):
    """He-style uniform initialisation, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in LAYERS:
        lim = sqrt(6.0 / i)
        parts.append(rng.uniform(-lim, lim, size=(o, i)).ravel())
        parts.append(np.zeros(o))
    return np.concatenate(parts)
