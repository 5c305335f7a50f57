"""Explicit unitary discrete Fourier transform in FP64 (oracle; test infrastructure).

The paper's step 1 (Sec. 2.1, "apply a FFT operator F to each member") only
needs F to be the DFT; the scale is not fixed.  The oracle uses the unitary
DFT, F u(k) = G^(-1/2) sum_x u(x) exp(-2 pi i (k_y y/ny + k_x x/nx)), so that
R = rI in physical space is rI in frequency space (Sec. 2.1, eq. spectral-enkf)
and Parseval holds without factors.  It is applied separably as dense DFT-matrix
products, O(ny nx (ny + nx)) per field: the definition, not a fast algorithm.
"""

from __future__ import annotations

import numpy as np


def dft_matrix(n: int, inverse: bool = False) -> np.ndarray:
    """Unitary 1-D DFT matrix W[k, x] = n^(-1/2) exp(-+2 pi i k x / n)."""
    j = np.arange(n, dtype=np.int64)
    e = np.outer(j, j) % n                    # exact integer phase index
    ang = 2.0 * np.pi * e.astype(np.float64) / n
    s = 1.0 if inverse else -1.0
    return (np.cos(ang) + 1j * s * np.sin(ang)) / np.sqrt(n)


def fft2(u: np.ndarray) -> np.ndarray:
    """Unitary 2-D DFT over the last two axes (full complex spectrum)."""
    ny, nx = u.shape[-2:]
    Fy = dft_matrix(ny)
    Fx = dft_matrix(nx)
    return Fy @ np.asarray(u, dtype=np.complex128) @ Fx.T


def ifft2(U: np.ndarray) -> np.ndarray:
    """Inverse of :func:`fft2` (complex result)."""
    ny, nx = U.shape[-2:]
    Gy = dft_matrix(ny, inverse=True)
    Gx = dft_matrix(nx, inverse=True)
    return Gy @ np.asarray(U, dtype=np.complex128) @ Gx.T


def dft2_matrix(ny: int, nx: int) -> np.ndarray:
    """The unitary 2-D DFT as one dense G x G matrix acting on row-major fields."""
    return np.kron(dft_matrix(ny), dft_matrix(nx))


def coefficients(u: np.ndarray, ks) -> np.ndarray:
    """Selected unitary DFT coefficients of u (last two axes) at wavenumbers ks.

    ``ks`` is a sequence of (k_y, k_x).  Cost O(G) per field per distinct k_x
    column, so it can sample full-size fields one coefficient at a time.
    """
    ny, nx = u.shape[-2:]
    ks = [(int(a) % ny, int(b) % nx) for a, b in ks]
    kxs = sorted({b for _, b in ks})
    x = np.arange(nx)
    y = np.arange(ny)
    Ex = np.exp(-2j * np.pi * ((np.outer(x, kxs) % nx) / nx))          # [nx][n_kx]
    part = np.asarray(u, dtype=np.float64) @ Ex                        # [..., ny, n_kx]
    out = np.empty(u.shape[:-2] + (len(ks),), dtype=np.complex128)
    col = {b: i for i, b in enumerate(kxs)}
    for i, (a, b) in enumerate(ks):
        ey = np.exp(-2j * np.pi * ((y * a) % ny) / ny)
        out[..., i] = np.tensordot(part[..., :, col[b]], ey, axes=([-1], [0]))
    return out / np.sqrt(ny * nx)
