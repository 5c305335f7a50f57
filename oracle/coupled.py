"""Coupled observed blocks: the spectral analysis without neglecting the mutual
cross-covariance of the observed blocks (oracle; test infrastructure).

eq. (multi-enkf) with H selecting the observed blocks O and the stationary block
covariance diagonalised by F gives, per wavenumber k, the Kalman gain

    K(k) = Chat_{:,O}(k) (Chat_{O,O}(k) + diag(rhat_O(k)))^-1          (M x n_obs)

where Chat_{a,b}(k) = 1/(N-1) sum_k ahat_k^(a) conj(ahat_k^(b)) (eq. dii and eq.
cov-multi-spectral, dense-consistent conjugation), and the update is
uhat^(j),a = uhat^(j) + sum_o K_{j,o} what_o.  Sec. 2.2 instead neglects
Chat_{o',o} for distinct observed o', o, which makes the bracket diagonal; this
module keeps it (a generalisation; the paper derives the single-observed case).

Singular brackets (possible only with rhat = 0): A = Chat_{O,O} + diag(rhat_O) is
Hermitian positive semidefinite; with det(A) <= 1e-6 a_11 a_22 (two observed
blocks) the gain uses the pseudo-inverse of the rank-1 part, A / tr(A)^2, and 0
where tr(A) = 0.  Supported for one or two observed blocks.
"""

from __future__ import annotations

from typing import Dict, Sequence, Tuple

import numpy as np

from . import dft
from .enkf import anomaly_spectra, half_to_full, spectral_cross, spectral_variance

SINGULAR_REL = 1e-6


def estimate(ens: np.ndarray, observed: Sequence[int]):
    """auto[o] (real) for o in O and cross[(a, o)] for every block a != o, o in O (full grid)."""
    observed = np.asarray(observed).astype(bool)
    M = observed.shape[0]
    ahat = anomaly_spectra(ens)
    auto: Dict[int, np.ndarray] = {}
    cross: Dict[Tuple[int, int], np.ndarray] = {}
    for o in np.flatnonzero(observed):
        o = int(o)
        auto[o] = spectral_variance(ahat[o])
        for a in range(M):
            if a != o:
                cross[(a, o)] = spectral_cross(ahat[a], ahat[o])
    return auto, cross


def bracket_inverse(A: np.ndarray) -> np.ndarray:
    """(A)^-1 per wavenumber for Hermitian PSD A [..., n, n], n <= 2, with the singular rule above."""
    n = A.shape[-1]
    if n == 1:
        a = A[..., 0, 0].real
        out = np.zeros_like(A)
        nz = a != 0
        out[..., 0, 0][nz] = 1.0 / a[nz]
        return out
    if n != 2:
        raise ValueError("coupled observed blocks: one or two supported")
    a = A[..., 0, 0].real
    d = A[..., 1, 1].real
    b = A[..., 0, 1]
    det = a * d - np.abs(b) ** 2
    tr = a + d
    regular = det > SINGULAR_REL * a * d
    out = np.zeros_like(A)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.stack([np.stack([d, -b], -1), np.stack([-np.conj(b), a], -1)], -2) / det[..., None, None]
        pinv = A / (tr ** 2)[..., None, None]
    out[regular] = inv[regular]
    sing = (~regular) & (tr > 0)
    out[sing] = pinv[sing]
    return out


def gains(auto, cross, rhat_full: Dict[int, np.ndarray], observed: Sequence[int]):
    """K[(j, o)] for every block j and observed o (full grid)."""
    observed = np.asarray(observed).astype(bool)
    M = observed.shape[0]
    obs = [int(i) for i in np.flatnonzero(observed)]
    n = len(obs)
    shape = next(iter(auto.values())).shape
    A = np.zeros(shape + (n, n), dtype=np.complex128)
    for p, o in enumerate(obs):
        for q, o2 in enumerate(obs):
            A[..., p, q] = auto[o] + rhat_full[o] if p == q else cross[(o, o2)]
    Ainv = bracket_inverse(A)
    K = {}
    for j in range(M):
        row = np.zeros(shape + (n,), dtype=np.complex128)      # Chat_{j,O}
        for q, o in enumerate(obs):
            row[..., q] = auto[o] if j == o else cross[(j, o)]
        Kj = np.einsum("...q,...qp->...p", row, Ainv)
        for p, o in enumerate(obs):
            K[(j, o)] = Kj[..., p]
    return K


def analyze(ens, data, pert, rhat_half, observed, return_parts=False):
    """Analysis ensemble [M][N][ny][nx] with the coupled gain (float64)."""
    ens = np.asarray(ens, dtype=np.float64)
    M, N, ny, nx = ens.shape
    observed = np.asarray(observed).astype(bool)
    obs = [int(i) for i in np.flatnonzero(observed)]
    auto, cross = estimate(ens, observed)
    rhat_half = np.asarray(rhat_half, dtype=np.float64).reshape(len(obs), ny, nx // 2 + 1)
    r_full = {o: half_to_full(rhat_half[i], nx, hermitian=False) for i, o in enumerate(obs)}
    K = gains(auto, cross, r_full, observed)
    data = np.asarray(data, dtype=np.float64)
    pert = np.asarray(pert, dtype=np.float64)
    ua = ens.copy()
    for k in range(N):
        w = {o: dft.fft2(data[i] + pert[k, i] - ens[o, k]) for i, o in enumerate(obs)}
        for j in range(M):
            S = np.zeros((ny, nx), dtype=np.complex128)
            for o in obs:
                S = S + K[(j, o)] * w[o]
            ua[j, k] = ens[j, k] + dft.ifft2(S).real
    if return_parts:
        return ua, {"auto": auto, "cross": cross, "gains": K}
    return ua
