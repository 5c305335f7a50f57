"""Dense brute-force forms for tiny grids (oracle; test infrastructure).

These follow the paper's linear-algebra statements directly, with no frequency
domain shortcut, and are used to pin the spectral oracle:
  * C_N = 1/(N-1) A A^T, the sample covariance of the ensemble (Sec. 2, "In the
    standard EnKF C_N is the sample covariance"), and its frequency-domain
    diagonal diag(F C_N F*) (Sec. 2.1, step 2: the diagonal of the sample
    covariance of the transformed ensemble);
  * the EnKF update of eq. (enkf) / eq. (multi-enkf),
      u_k^a = u_k + C H^T (H C H^T + R)^-1 (d + e_k - H u_k),
    solved with a dense LU, where the block covariance C^(ab) = F* diag(c^(ab)) F
    is the circulant (stationary) covariance whose frequency diagonal is c^(ab),
    R = blockdiag(F* diag(rhat_o) F), H selects the observed blocks and, as in
    Sec. 2.2, C^(o'o) = 0 for distinct observed blocks (or the full covariance,
    for the coupled variant).
"""

from __future__ import annotations

from typing import Dict, Sequence

import numpy as np

from . import dft


def anomaly_matrix(block: np.ndarray) -> np.ndarray:
    """A = [u_1 - ubar, ..., u_N - ubar] as a G x N matrix for one block [N][ny][nx]."""
    b = np.asarray(block, dtype=np.float64)
    N = b.shape[0]
    return (b - b.mean(axis=0, keepdims=True)).reshape(N, -1).T


def sample_covariance(block_j: np.ndarray, block_o: np.ndarray) -> np.ndarray:
    """C_N^(jo) = 1/(N-1) A_j A_o^T (G x G)."""
    Aj = anomaly_matrix(block_j)
    Ao = anomaly_matrix(block_o)
    return Aj @ Ao.T / (Aj.shape[1] - 1)


def freq_diagonal(C: np.ndarray, ny: int, nx: int) -> np.ndarray:
    """diag(F C F*) on the full grid [ny][nx] with F the unitary 2-D DFT matrix."""
    F = dft.dft2_matrix(ny, nx)
    return np.diag(F @ C @ F.conj().T).reshape(ny, nx)


def circulant(c_full: np.ndarray) -> np.ndarray:
    """F* diag(c) F as a dense G x G matrix (real when c is Hermitian-symmetric)."""
    ny, nx = c_full.shape
    F = dft.dft2_matrix(ny, nx)
    return F.conj().T @ np.diag(np.asarray(c_full, dtype=np.complex128).ravel()) @ F


def dense_analyze(
    ens: np.ndarray,
    data: np.ndarray,
    pert: np.ndarray,
    auto: Dict[int, np.ndarray],
    cross: Dict[tuple, np.ndarray],
    rhat_full: Dict[int, np.ndarray],
    observed: Sequence[int],
    neglect_observed_cross: bool = True,
) -> np.ndarray:
    """eq. (enkf) with the stationary block covariance built from full-grid tables.

    auto[o], cross[(j,o)], rhat_full[o] are full-grid frequency diagonals.  With
    ``neglect_observed_cross`` (Sec. 2.2) C^(o'o) = 0 for distinct observed blocks;
    without it cross[(o', o)] must be given for them and the full covariance is used."""
    ens = np.asarray(ens, dtype=np.float64)
    M, N, ny, nx = ens.shape
    G = ny * nx
    observed = np.asarray(observed).astype(bool)
    obs = [int(i) for i in np.flatnonzero(observed)]
    nO = len(obs)
    # columns of C belonging to the observed blocks: C[:, o] (M*G x nO*G)
    CHt = np.zeros((M * G, nO * G), dtype=np.complex128)
    for i, o in enumerate(obs):
        for a in range(M):
            if a == o:
                blk = circulant(auto[o])
            elif observed[a] and neglect_observed_cross:
                continue                      # neglected mutual cross-covariance
            else:
                blk = circulant(cross[(a, o)])
            CHt[a * G:(a + 1) * G, i * G:(i + 1) * G] = blk
    HCHt = np.zeros((nO * G, nO * G), dtype=np.complex128)
    for i, o in enumerate(obs):
        HCHt[i * G:(i + 1) * G, i * G:(i + 1) * G] = circulant(auto[o]) + circulant(rhat_full[o])
        if not neglect_observed_cross:
            for i2, o2 in enumerate(obs):
                if o2 != o:
                    HCHt[i2 * G:(i2 + 1) * G, i * G:(i + 1) * G] = circulant(cross[(o2, o)])
    if max(np.abs(CHt.imag).max(initial=0), np.abs(HCHt.imag).max(initial=0)) > 1e-9 * (
        np.abs(CHt).max(initial=1) + np.abs(HCHt).max(initial=1)
    ):
        raise ValueError("covariance tables are not Hermitian-symmetric")
    CHt = CHt.real
    HCHt = HCHt.real
    data = np.asarray(data, dtype=np.float64)
    pert = np.asarray(pert, dtype=np.float64)
    ua = ens.copy()
    for k in range(N):
        innov = np.concatenate([(data[i] + pert[k, i] - ens[o, k]).ravel() for i, o in enumerate(obs)])
        inc = CHt @ np.linalg.solve(HCHt, innov)
        ua[:, k] = ens[:, k] + inc.reshape(M, ny, nx)
    return ua
