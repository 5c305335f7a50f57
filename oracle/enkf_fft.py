"""FFT EnKF analysis of a few members at full size, in FP64 with a library FFT as the transform step
(oracle; test infrastructure, imported only by the tests).

The explicit-DFT oracle (enkf.py) costs O(G (nx + ny)) per field, too slow for a 4096 x 4096 state of
80 fields.  This module computes the same quantities with a library real FFT (scipy.fft / numpy.fft
rfft2 and irfft2, unitary scaling, FP64) as the step F, on the half spectrum [ny][nx/2+1], and streams the
members one field at a time so that only the covariance sums and a few spectra are held:

  1. chat^(oo) = 1/(N-1) sum_k |F(u_k^(o) - ubar^(o))|^2 and chat^(jo) = 1/(N-1) sum_k
     F(u_k^(j) - ubar^(j)) conj F(u_k^(o) - ubar^(o)) (eq. dii, eq. cov-multi-spectral, the
     conjugate on the observed block as in enkf.py), the mean taken in physical space in FP64;
  2. gains G^(oo) = chat^(oo) / (chat^(oo) + rhat_o) and G^(jo) = chat^(jo) / (chat^(oo) + rhat_o),
     0 where the denominator is 0 (eq. spectral-multi-enkf; several observed blocks as in enkf.py);
  3. for the requested members k, u_k^(j),a = u_k^(j) + F^-1 [sum_o G^(jo) F(d_o + e_{k,o} - u_k^(o))]
     (observed o: only G^(oo) times its own innovation).

On the half spectrum every table of a real field is Hermitian in the columns k_x = 0 and nx/2, so
irfft2 of the half-spectrum product equals the real part of the full inverse transform.  Pinned to
enkf.analyze on small grids in tests/test_oracle_fft_path.py.
"""

from __future__ import annotations

import os
from typing import Callable, Dict, Sequence

import numpy as np


try:   # the same transform, threaded over the host's cores where scipy is present
    import scipy.fft as _sfft

    _WORKERS = os.cpu_count() or 1

    def _rfft2(x: np.ndarray) -> np.ndarray:
        return _sfft.rfft2(np.asarray(x, dtype=np.float64), norm="ortho", workers=_WORKERS)

    def _irfft2(X: np.ndarray, shape) -> np.ndarray:
        return _sfft.irfft2(X, s=shape, norm="ortho", workers=_WORKERS)
except ImportError:  # pragma: no cover
    def _rfft2(x: np.ndarray) -> np.ndarray:
        return np.fft.rfft2(np.asarray(x, dtype=np.float64), norm="ortho")

    def _irfft2(X: np.ndarray, shape) -> np.ndarray:
        return np.fft.irfft2(X, s=shape, norm="ortho")


def covariance_sums(field: Callable[[int, int], np.ndarray], M: int, N: int, observed: Sequence[int]):
    """Step 1 streamed over the members: field(j, k) returns u_k^(j) [ny][nx].  Returns the block
    means [M][ny][nx], auto tables {o: chat^(oo)} and cross tables {(j, o): chat^(jo)} on the half
    spectrum."""
    observed = np.asarray(observed).astype(bool)
    obs = [int(i) for i in np.flatnonzero(observed)]
    un = [int(i) for i in np.flatnonzero(~observed)]
    mean = None
    for j in range(M):
        acc = None
        for k in range(N):
            f = np.asarray(field(j, k), dtype=np.float64)
            acc = f.copy() if acc is None else acc + f
        if mean is None:
            mean = np.empty((M,) + acc.shape)
        mean[j] = acc / N
    auto: Dict[int, np.ndarray] = {o: 0.0 for o in obs}
    cross: Dict = {(j, o): 0.0 for o in obs for j in un}
    for k in range(N):
        ahat = {j: _rfft2(np.asarray(field(j, k), dtype=np.float64) - mean[j]) for j in range(M)}
        for o in obs:
            auto[o] = auto[o] + np.abs(ahat[o]) ** 2
            for j in un:
                cross[(j, o)] = cross[(j, o)] + ahat[j] * np.conj(ahat[o])
    auto = {o: v / (N - 1) for o, v in auto.items()}
    cross = {p: v / (N - 1) for p, v in cross.items()}
    return mean, auto, cross


def gains(auto, cross, rhat_half: Dict[int, np.ndarray]):
    """Step 2 on the half spectrum: {(o, o): G^(oo), (j, o): G^(jo)}."""
    g = {}
    for o, c in auto.items():
        den = c + rhat_half[o]
        nz = den != 0
        g[(o, o)] = np.where(nz, c / np.where(nz, den, 1.0), 0.0)
        for (j, oo), cj in cross.items():
            if oo == o:
                g[(j, o)] = np.where(nz, cj / np.where(nz, den, 1.0), 0.0)
    return g


def analysis_of_member(k: int, field: Callable[[int, int], np.ndarray], M: int, observed: Sequence[int],
                       data: np.ndarray, pert: Callable[[int, int], np.ndarray], g) -> np.ndarray:
    """Step 3 for member k: u_k^a [M][ny][nx].  data [n_obs][ny][nx]; pert(k, i) returns e_{k,i}."""
    observed = np.asarray(observed).astype(bool)
    obs = [int(i) for i in np.flatnonzero(observed)]
    u = {j: np.asarray(field(j, k), dtype=np.float64) for j in range(M)}
    shape = u[0].shape
    what = {o: _rfft2(np.asarray(data[i], np.float64) + np.asarray(pert(k, i), np.float64) - u[o])
            for i, o in enumerate(obs)}
    out = np.empty((M,) + shape)
    for j in range(M):
        if observed[j]:
            S = g[(j, j)] * what[j]
        else:
            S = sum(g[(j, o)] * what[o] for o in obs)
        out[j] = u[j] + _irfft2(S, shape)
    return out
