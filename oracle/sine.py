"""FFT EnKF with the real sine transform (Sec. 4: the experiments replace the periodic DFT by
the real sine FFT, which leaves the boundary unchanged), in FP64 (oracle; test infrastructure).

Grid ny x nx of nodes whose first and last rows and columns are the boundary; the
my x mx = (ny-2) x (nx-2) interior nodes are transformed with the orthonormal type-I discrete
sine transform in each direction,

    S_m[k, j] = sqrt(2/(m+1)) sin(pi (k+1)(j+1)/(m+1)),   k, j = 0..m-1,

which is symmetric and its own inverse.  Every basis function vanishes on the boundary nodes, so
any increment built from them is zero there.  The steps are those of Sec. 2.1 with F replaced by
the 2-D sine transform Sv = S_my v S_mx:

  1. ahat_k^(j) = S(u_k^(j) - ubar^(j)) on the interior, member mean removed in physical space.
  2. chat^(oo) = 1/(N-1) sum_k (ahat_k^(o))^2 and chat^(jo) = 1/(N-1) sum_k ahat_k^(j) ahat_k^(o)
     (eq. dii, eq. cov-multi-spectral; all coefficients are real, so the cross spectrum has no
     conjugation question).
  3. u_k^(j),a = u_k^(j) + S^-1[chat^(jo) / (chat^(oo) + rhat_o) . S(d_o + e_{k,o} - u_k^(o))]
     (eq. spectral-enkf, eq. spectral-multi-enkf) on the interior; boundary nodes keep u_k^(j).

Readings, as for the periodic oracle (oracle.enkf): several observed blocks neglect their mutual
cross-covariances (Sec. 2.2); the gain is 0 where chat^(oo) + rhat_o == 0; rhat_o is the variance
of the data error in the sine basis, so R = r I on the interior gives rhat_o = r.
"""

from __future__ import annotations

from typing import Dict, Sequence, Tuple

import numpy as np


def dst1_matrix(m: int) -> np.ndarray:
    """Orthonormal DST-I matrix S_m (m x m), the definition written out."""
    k = np.arange(1, m + 1)
    return np.sqrt(2.0 / (m + 1)) * np.sin(np.pi * np.outer(k, k) / (m + 1))


def sine2(v: np.ndarray) -> np.ndarray:
    """2-D orthonormal sine transform of the last two axes (interior-sized arrays)."""
    my, mx = v.shape[-2:]
    return dst1_matrix(my) @ v @ dst1_matrix(mx)


def isine2(vhat: np.ndarray) -> np.ndarray:
    """Inverse of sine2; S_m is symmetric and orthogonal, so it is its own inverse."""
    return sine2(vhat)


def interior(u: np.ndarray) -> np.ndarray:
    return np.asarray(u)[..., 1:-1, 1:-1]


def estimate(ens: np.ndarray, observed: Sequence[int]) -> Tuple[Dict[int, np.ndarray], Dict[Tuple[int, int], np.ndarray]]:
    """Steps 1-2: auto spectra chat^(oo) for observed o and cross spectra chat^(jo) for unobserved
    j, on the interior sine wavenumbers [my][mx]."""
    ens = np.asarray(ens, dtype=np.float64)
    M, N = ens.shape[:2]
    a = interior(ens) - interior(ens).mean(axis=1, keepdims=True)
    ahat = sine2(a)
    obs = [j for j in range(M) if observed[j]]
    auto = {o: np.sum(ahat[o] ** 2, axis=0) / (N - 1) for o in obs}
    cross = {(j, o): np.sum(ahat[j] * ahat[o], axis=0) / (N - 1)
             for o in obs for j in range(M) if not observed[j]}
    return auto, cross


def spectrum_tables(ens: np.ndarray, observed: Sequence[int]) -> np.ndarray:
    """The tables in library order: chat^(oo) for observed o ascending, then for observed o
    ascending chat^(jo) for unobserved j ascending, each [my][mx] real."""
    auto, cross = estimate(ens, observed)
    M = len(observed)
    obs = [j for j in range(M) if observed[j]]
    un = [j for j in range(M) if not observed[j]]
    parts = [auto[o] for o in obs] + [cross[(j, o)] for o in obs for j in un]
    return np.stack(parts) if parts else np.zeros((0,) + np.asarray(ens).shape[-2:])


def _ratio(num: np.ndarray, den: np.ndarray) -> np.ndarray:
    out = np.zeros_like(num, dtype=np.float64)
    np.divide(num, den, out=out, where=den != 0)
    return out


def gains(auto, cross, rhat: Dict[int, np.ndarray]):
    g = {}
    for o, c in auto.items():
        den = c + rhat[o]
        g[(o, o)] = _ratio(c, den)
        for (j, oo), cj in cross.items():
            if oo == o:
                g[(j, o)] = _ratio(cj, den)
    return g


def analyze(ens, data, pert, rhat, observed, return_parts: bool = False):
    """Analysis ensemble [M][N][ny][nx] (float64).

    ens [M][N][ny][nx]; data [n_obs][ny][nx]; pert [N][n_obs][ny][nx] (only the interior of data
    and pert enters); rhat [n_obs][ny-2][nx-2] data-error variance per sine wavenumber.
    """
    ens = np.asarray(ens, dtype=np.float64)
    M, N, ny, nx = ens.shape
    obs = [j for j in range(M) if observed[j]]
    auto, cross = estimate(ens, observed)
    rhat = np.asarray(rhat, dtype=np.float64).reshape(len(obs), ny - 2, nx - 2)
    g = gains(auto, cross, {o: rhat[i] for i, o in enumerate(obs)})
    data = interior(np.asarray(data, dtype=np.float64))
    pert = interior(np.asarray(pert, dtype=np.float64))
    ua = ens.copy()
    for k in range(N):
        w = {o: sine2(data[i] + pert[k, i] - interior(ens[o, k])) for i, o in enumerate(obs)}
        for j in range(M):
            if observed[j]:
                S = g[(j, j)] * w[j]
            else:
                S = np.zeros((ny - 2, nx - 2))
                for o in obs:
                    S = S + g[(j, o)] * w[o]
            ua[j, k, 1:-1, 1:-1] = ens[j, k, 1:-1, 1:-1] + isine2(S)
    if return_parts:
        return ua, {"auto": auto, "cross": cross, "gains": g}
    return ua
