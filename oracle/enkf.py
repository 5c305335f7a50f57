"""FFT EnKF analysis step in FP64, written from the paper (oracle; test infrastructure).

Notation follows Sec. 2: M blocks (physical fields), N members, block j of
member k is u_k^(j) on an ny x nx periodic grid; O is the set of observed blocks
(H^(o) = I for o in O, H^(j) = 0 otherwise) and the data error of block o has
spectral variance rhat_o (R = rI gives rhat_o = r).

Steps, in the paper's order:
  1. uhat_k = F u_k for every member (Sec. 2.1, step 1).
  2. chat_i = 1/(N-1) sum_k |uhat_ik - mean_k uhat_ik|^2, eq. (dii); the
     spectral cross-covariance of eq. (cov-multi-spectral) for block pairs.
     The mean is removed in physical space before F; by linearity this is the
     same as removing mean_k uhat_ik in frequency space.
  3. uhat_k^(j),a = uhat_k^(j) + chat^(jo) . (chat^(oo) + rhat_o)^-1 .
     (dhat_o + ehat_{k,o} - uhat_k^(o)), eq. (spectral-enkf) for one block and
     eq. (spectral-multi-enkf) for a block state, then u^a = Re F^-1 uhat^a.

Readings of points the paper leaves open:
  * F is the unitary DFT (oracle.dft).
  * Conjugation in eq. (cov-multi-spectral): the dense derivation
    diag(F C_N^(jo) F*) = 1/(N-1) sum_k ahat_k^(j) conj(ahat_k^(o)) puts the
    conjugate on the observed block o; the printed formula has it on block j,
    which is the spectrum of C^(oj) instead.  ``printed_form=True`` selects the
    printed placement so that the brute-force pins can tell the two apart.
  * Several observed blocks: their mutual cross-covariances are neglected, as
    Sec. 2.2 does for the components of the morphed state, so every observed
    block o contributes its own gain chat^(jo)/(chat^(oo)+rhat_o); an observed
    block is updated only by its own innovation, an unobserved block j by the
    sum over o in O.
  * Where chat^(oo) + rhat_o == 0 the gain is 0 (no information: keep forecast).
  * The innovation uses the forecast member itself (u_k and u_k^f in eq. enkf
    denote the same member).
  * Tables given on the half spectrum [ny][nx/2+1] are extended to the full grid
    by the symmetry of a real field: even for variances, Hermitian for cross
    spectra.  The analysis is the real part of F^-1 of the spectral update.
"""

from __future__ import annotations

from typing import Dict, Optional, Sequence, Tuple

import numpy as np

from . import dft


# --------------------------------------------------------------------------
# half <-> full spectrum tables
# --------------------------------------------------------------------------
def half_to_full(h: np.ndarray, nx: int, hermitian: bool) -> np.ndarray:
    """Full-grid table from a half-spectrum one [..., ny, nx/2+1] (real-field symmetry)."""
    h = np.asarray(h)
    ny = h.shape[-2]
    L = nx // 2
    full = np.empty(h.shape[:-1] + (nx,), dtype=np.complex128 if hermitian else h.dtype)
    full[..., : L + 1] = h
    ky_neg = (-np.arange(ny)) % ny
    for kx in range(L + 1, nx):
        col = h[..., ky_neg, nx - kx]
        full[..., :, kx] = np.conj(col) if hermitian else col
    return full


def full_to_half(f: np.ndarray) -> np.ndarray:
    nx = f.shape[-1]
    return np.array(f[..., : nx // 2 + 1])


# --------------------------------------------------------------------------
# steps 1-2: spectra of anomalies, eq. (dii) and eq. (cov-multi-spectral)
# --------------------------------------------------------------------------
def ensemble_mean(ens: np.ndarray) -> np.ndarray:
    """Member mean of every block, [M][N][ny][nx] -> [M][ny][nx] (eq. dii, mean term)."""
    return np.asarray(ens, dtype=np.float64).mean(axis=1)


def anomaly_spectra(ens: np.ndarray) -> np.ndarray:
    """ahat_k^(j) = F(u_k^(j) - mean_k u_k^(j)), full complex spectra [M][N][ny][nx]."""
    e = np.asarray(ens, dtype=np.float64)
    return dft.fft2(e - e.mean(axis=1, keepdims=True))


def spectral_variance(ahat_o: np.ndarray) -> np.ndarray:
    """eq. (dii): chat = 1/(N-1) sum_k |ahat_k|^2 for one block's anomaly spectra [N][ny][nx]."""
    N = ahat_o.shape[0]
    return np.sum(np.abs(ahat_o) ** 2, axis=0) / (N - 1)


def spectral_cross(ahat_j: np.ndarray, ahat_o: np.ndarray, printed_form: bool = False) -> np.ndarray:
    """eq. (cov-multi-spectral): 1/(N-1) sum_k ahat_k^(j) conj(ahat_k^(o)).

    ``printed_form`` conjugates block j instead (the formula as printed)."""
    N = ahat_j.shape[0]
    if printed_form:
        return np.sum(np.conj(ahat_j) * ahat_o, axis=0) / (N - 1)
    return np.sum(ahat_j * np.conj(ahat_o), axis=0) / (N - 1)


class Spectrum:
    """Spectral covariance of a block state on the full grid.

    auto[o]       real chat^(oo) for observed o
    cross[(j,o)]  complex chat^(jo) for unobserved j, observed o
    """

    def __init__(self, auto: Dict[int, np.ndarray], cross: Dict[Tuple[int, int], np.ndarray]):
        self.auto = auto
        self.cross = cross


def estimate_spectrum(ens: np.ndarray, observed: Sequence[int], printed_form: bool = False) -> Spectrum:
    """Steps 1-2 for the tables the analysis needs (observed autos, unobserved x observed crosses)."""
    observed = np.asarray(observed).astype(bool)
    M = observed.shape[0]
    ahat = anomaly_spectra(ens)
    auto = {}
    cross = {}
    for o in range(M):
        if not observed[o]:
            continue
        auto[o] = spectral_variance(ahat[o])
        for j in range(M):
            if not observed[j]:
                cross[(j, o)] = spectral_cross(ahat[j], ahat[o], printed_form)
    return Spectrum(auto, cross)


def table_order(observed: Sequence[int]):
    """Order of the spectrum tables at the library boundary.

    First the auto table of every observed block (ascending), then for every
    observed o (ascending) the cross table of every unobserved j (ascending)."""
    observed = np.asarray(observed).astype(bool)
    obs = [int(i) for i in np.flatnonzero(observed)]
    un = [int(i) for i in np.flatnonzero(~observed)]
    return obs, [(j, o) for o in obs for j in un]


def spectrum_to_tables(spec: Spectrum, observed: Sequence[int]) -> np.ndarray:
    """Pack a Spectrum into the boundary's flat float64 layout (half spectrum).

    autos: [ny][nx/2+1] real each; crosses: [ny][nx/2+1][2] (re, im) each."""
    obs, pairs = table_order(observed)
    parts = [full_to_half(spec.auto[o]).astype(np.float64).ravel() for o in obs]
    for p in pairs:
        h = full_to_half(spec.cross[p])
        parts.append(np.stack([h.real, h.imag], axis=-1).ravel())
    return np.concatenate(parts) if parts else np.zeros(0)


def tables_to_spectrum(tables: np.ndarray, observed: Sequence[int], ny: int, nx: int) -> Spectrum:
    """Inverse of :func:`spectrum_to_tables`, extended to the full grid."""
    obs, pairs = table_order(observed)
    K = ny * (nx // 2 + 1)
    t = np.asarray(tables, dtype=np.float64).ravel()
    pos = 0
    auto = {}
    cross = {}
    for o in obs:
        auto[o] = half_to_full(t[pos: pos + K].reshape(ny, nx // 2 + 1), nx, hermitian=False)
        pos += K
    for p in pairs:
        h = t[pos: pos + 2 * K].reshape(ny, nx // 2 + 1, 2)
        auto_c = h[..., 0] + 1j * h[..., 1]
        cross[p] = half_to_full(auto_c, nx, hermitian=True)
        pos += 2 * K
    return Spectrum(auto, cross)


# --------------------------------------------------------------------------
# step 3: eq. (spectral-enkf) / eq. (spectral-multi-enkf)
# --------------------------------------------------------------------------
def _safe_ratio(num: np.ndarray, den: np.ndarray) -> np.ndarray:
    out = np.zeros(np.broadcast(num, den).shape, dtype=np.result_type(num, den))
    nz = den != 0
    np.divide(num, den, out=out, where=nz)
    return out


def gains(spec: Spectrum, rhat_full: Dict[int, np.ndarray], observed: Sequence[int]):
    """Per-wavenumber gains: chat^(oo)/(chat^(oo)+rhat_o) and chat^(jo)/(chat^(oo)+rhat_o)."""
    g = {}
    for o, c in spec.auto.items():
        den = c + rhat_full[o]
        g[(o, o)] = _safe_ratio(c, den)
        for (j, oo), cj in spec.cross.items():
            if oo == o:
                g[(j, o)] = _safe_ratio(cj, den)
    return g


def analyze(
    ens: np.ndarray,
    data: np.ndarray,
    pert: np.ndarray,
    rhat_half: np.ndarray,
    observed: Sequence[int],
    spectrum: Optional[np.ndarray] = None,
    printed_form: bool = False,
    return_parts: bool = False,
):
    """Analysis ensemble u^a [M][N][ny][nx] (float64).

    ens [M][N][ny][nx]; data [n_obs][ny][nx]; pert [N][n_obs][ny][nx];
    rhat_half [n_obs][ny][nx/2+1]; spectrum: None (estimated from ens, steps
    1-2) or boundary-layout tables (:func:`spectrum_to_tables`).
    """
    ens = np.asarray(ens, dtype=np.float64)
    M, N, ny, nx = ens.shape
    observed = np.asarray(observed).astype(bool)
    obs = [int(i) for i in np.flatnonzero(observed)]
    if spectrum is None:
        spec = estimate_spectrum(ens, observed, printed_form)
    else:
        spec = tables_to_spectrum(spectrum, observed, ny, nx)
    rhat_half = np.asarray(rhat_half, dtype=np.float64).reshape(len(obs), ny, nx // 2 + 1)
    r_full = {o: half_to_full(rhat_half[i], nx, hermitian=False) for i, o in enumerate(obs)}
    g = gains(spec, r_full, observed)
    data = np.asarray(data, dtype=np.float64)
    pert = np.asarray(pert, dtype=np.float64)
    ua = ens.copy()
    max_imag = 0.0
    for k in range(N):
        # innovation spectra for every observed block: F(d_o + e_{k,o} - u_k^(o))
        w = {o: dft.fft2(data[i] + pert[k, i] - ens[o, k]) for i, o in enumerate(obs)}
        for j in range(M):
            if observed[j]:
                S = g[(j, j)] * w[j]
            else:
                S = np.zeros((ny, nx), dtype=np.complex128)
                for o in obs:
                    S = S + g[(j, o)] * w[o]
            inc = dft.ifft2(S)
            max_imag = max(max_imag, float(np.max(np.abs(inc.imag))) if inc.size else 0.0)
            ua[j, k] = ens[j, k] + inc.real
    if return_parts:
        return ua, {"spectrum": spec, "gains": g, "max_imag": max_imag}
    return ua
