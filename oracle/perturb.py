"""Perturbations drawn by the method itself, e_{k,o} ~ N(0, R_o) with R_o = F* diag(rhat_o) F
(eq. enkf: the data perturbations of the EnKF), generated in frequency space from a seed
(oracle; test infrastructure).

    ehat_{k,o}(kappa) = sqrt(rhat_o(kappa)) zhat_{k,o}(kappa),     e_{k,o} = F^-1 ehat_{k,o}

with zhat the unitary DFT of a white N(0, 1) field: Hermitian (zhat(-kappa) = conj zhat(kappa)),
E |zhat|^2 = 1, real at the self-conjugate wavenumbers.  On the half spectrum [ny][nx/2+1]:
columns 0 < k_x < nx/2 hold independent complex values (real and imaginary parts N(0, 1/2));
in the columns k_x = 0 and k_x = nx/2 the value at k_y > ny/2 is the conjugate of the one at
ny - k_y, and k_y = 0, ny/2 are real N(0, 1).

The normals come from the counter-based generator Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC 2011), key (seed mod 2^32, seed div 2^32),
stream s = k n_obs + o.  In the columns 0 < k_x < nx/2 one counter (k_y mod ny/2, k_x, s, 0)
serves k_y and k_y + ny/2: words (0, 1) for k_y < ny/2, words (2, 3) for the other; in the
columns k_x = 0, nx/2 the counter is (min(k_y, ny - k_y), k_x, s, 0) with words (0, 1).  A word
pair (w_a, w_b) gives u = (floor(w / 2^8) + 1/2) / 2^24 and Box-Muller
n_1 + i n_2 = sqrt(-2 ln u_a) exp(2 pi i u_b).  Complex entries are (n_1 + i n_2) / sqrt(2),
real ones n_1.  The GPU implements the same definition independently.
"""

from __future__ import annotations

import numpy as np

from . import dft
from .enkf import half_to_full

M0, M1 = 0xD2511F53, 0xCD9E8D57      # round multipliers
W0, W1 = 0x9E3779B9, 0xBB67AE85      # key increments (golden ratio, sqrt(3) - 1)
MASK = 0xFFFFFFFF


def philox4x32_10(counter, key):
    """Philox4x32 with 10 rounds; counter (..., 4), key (..., 2) uint32 arrays -> (..., 4) uint32."""
    c = [np.asarray(counter[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64)
    k1 = np.asarray(key[..., 1], dtype=np.uint64)
    for _ in range(10):
        p0 = c[0] * np.uint64(M0)
        p1 = c[2] * np.uint64(M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        k0 = (k0 + np.uint64(W0)) & np.uint64(MASK)
        k1 = (k1 + np.uint64(W1)) & np.uint64(MASK)
    return np.stack([x.astype(np.uint32) for x in c], axis=-1)


def spectral_white(ny: int, nx: int, seed: int, stream: int) -> np.ndarray:
    """zhat on the half spectrum [ny][nx/2+1] (complex128) for one (member, observed block) stream."""
    L = nx // 2
    ky = np.arange(ny)[:, None] * np.ones((1, L + 1), dtype=np.int64)
    kx = np.ones((ny, 1), dtype=np.int64) * np.arange(L + 1)[None, :]
    edge = (kx == 0) | (kx == L)
    high = (~edge) & (2 * ky >= ny)                    # interior entries taking words (2, 3)
    kyc = np.where(edge, np.minimum(ky, (ny - ky) % ny), ky % (ny // 2))
    ctr = np.stack([kyc, kx, np.full_like(ky, stream), np.zeros_like(ky)], axis=-1).astype(np.uint32)
    key = np.broadcast_to(np.array([seed & MASK, (seed >> 32) & MASK], dtype=np.uint32), ctr.shape[:-1] + (2,))
    w = philox4x32_10(ctr, key)
    wa = np.where(high, w[..., 2], w[..., 0])
    wb = np.where(high, w[..., 3], w[..., 1])
    u1 = ((wa >> np.uint32(8)).astype(np.float64) + 0.5) / 2.0 ** 24
    u2 = ((wb >> np.uint32(8)).astype(np.float64) + 0.5) / 2.0 ** 24
    r = np.sqrt(-2.0 * np.log(u1))
    n1, n2 = r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)
    z = (n1 + 1j * n2) / np.sqrt(2.0)
    self_conj = edge & ((ky == 0) | (2 * ky == ny))
    z = np.where(self_conj, n1 + 0j, z)
    upper = edge & (2 * ky > ny)
    return np.where(upper, np.conj(z), z)


def perturbations(ny: int, nx: int, rhat_half: np.ndarray, seed: int, N: int) -> np.ndarray:
    """e [N][n_obs][ny][nx] = F^-1 (sqrt(rhat_o) zhat_{k,o}), zhat from stream k n_obs + o."""
    rhat_half = np.asarray(rhat_half, dtype=np.float64)
    n_obs = rhat_half.shape[0]
    out = np.empty((N, n_obs, ny, nx))
    for k in range(N):
        for o in range(n_obs):
            eh = np.sqrt(rhat_half[o]) * spectral_white(ny, nx, seed, k * n_obs + o)
            full = half_to_full(eh, nx, hermitian=True)
            e = dft.ifft2(full)
            out[k, o] = e.real
    return out
