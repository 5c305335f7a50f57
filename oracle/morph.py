"""Morphing transform and its inverse around the FFT EnKF (Sec. 2.2), in FP64 (oracle; test
infrastructure, imported only by the tests and the bench's CPU baseline).

The registration itself (finding T_k) is not part of this: the mappings are inputs.

Grid: periodic ny x nx nodes with unit spacing, node p = (y, x).  A mapping T : Omega -> Omega is a
displacement field stored as two components [2][ny][nx], T[0] along x (the fastest axis) and T[1]
along y, in grid units.  Fields are [ny][nx].

Readings (the paper fixes none of them):
  * Composition f o (I + T) at node p is f(p + T(p)), with f evaluated between nodes by bilinear
    interpolation on the periodic grid.
  * (I + T)^-1(p) is the point q with q + T(q) = p, found by the fixed-point iteration
    q_0 = p, q_{i+1} = p - T(q_i) (T interpolated bilinearly at q_i), at most n_iter steps, a point
    stopping after the first step that moves it by at most tol in each component.  It converges
    when T is a contraction, which the registration's conditions T ~ 0, grad T ~ 0 ask for.
  * The extended state of member k keeps the analysis layout: blocks (T_x, T_y, r^(1), ..., r^(M)),
    and the extended data is (T_0x, T_0y, r_0^(1)).

Steps (Sec. 2.2, eq. morphing-transform and eq. inverse-morphing):
  forward:   r_k^(j) = u_k^(j) o (I + T_k)^-1 - u_{N+1}^(j)
  reference: utilde_{N+1}^a = (1/N) sum_k utilde_k^a   (mean of T^a and of r^a over the members)
  inverse:   u_k^(j),a = (u_{N+1}^(j) + r_k^(j),a) o (I + T_k^a)

Parity is pinned in tests/test_oracle_morph.py: integer shifts against np.roll, the bilinear
interpolation against SciPy's map_coordinates (order 1, grid-wrap), the fixed-point inverse by its
defining equation, and the inverse's special cases (T = 0, identical members).
"""

from __future__ import annotations

import numpy as np


def interp_periodic(f: np.ndarray, qy: np.ndarray, qx: np.ndarray) -> np.ndarray:
    """Bilinear interpolation of the periodic field f [ny][nx] at the points (qy, qx)."""
    ny, nx = f.shape
    fy = np.floor(qy)
    fx = np.floor(qx)
    wy = qy - fy
    wx = qx - fx
    y0 = fy.astype(np.int64) % ny
    x0 = fx.astype(np.int64) % nx
    y1 = (y0 + 1) % ny
    x1 = (x0 + 1) % nx
    return ((1 - wy) * ((1 - wx) * f[y0, x0] + wx * f[y0, x1])
            + wy * ((1 - wx) * f[y1, x0] + wx * f[y1, x1]))


def node_coords(ny: int, nx: int):
    py, px = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    return py, px


def compose(f: np.ndarray, T: np.ndarray) -> np.ndarray:
    """f o (I + T) on the nodes: f(p + T(p)), T [2][ny][nx] = (T_x, T_y)."""
    py, px = node_coords(*f.shape)
    return interp_periodic(f, py + T[1], px + T[0])


def inverse_points(T: np.ndarray, n_iter: int, tol: float = 0.0):
    """(I + T)^-1 at every node p: q_0 = p, q_{i+1} = p - T(q_i); returns (qy, qx)."""
    T = np.asarray(T, dtype=np.float64)
    py, px = node_coords(T.shape[1], T.shape[2])
    return inverse_points_at(T, py, px, n_iter, tol)


def inverse_points_at(T: np.ndarray, py: np.ndarray, px: np.ndarray, n_iter: int, tol: float = 0.0):
    """(I + T)^-1 at the given nodes (py, px) only, by the same iteration.  A point stops after the
    first step that moves it by at most tol in each component (tol = 0: only when the iterate
    repeats, which changes nothing), else after n_iter steps."""
    T = np.asarray(T, dtype=np.float64)
    py = np.asarray(py, dtype=np.float64)
    px = np.asarray(px, dtype=np.float64)
    qy, qx = py.copy(), px.copy()
    active = np.ones(qy.shape, dtype=bool)
    for _ in range(n_iter):
        if not active.any():
            break
        tx = interp_periodic(T[0], qy, qx)
        ty = interp_periodic(T[1], qy, qx)
        ny_, nx_ = py - ty, px - tx
        done = (np.abs(ny_ - qy) <= tol) & (np.abs(nx_ - qx) <= tol)
        qy = np.where(active, ny_, qy)
        qx = np.where(active, nx_, qx)
        active &= ~done
    return qy, qx


def morph_forward(u: np.ndarray, u_ref: np.ndarray, T: np.ndarray, n_iter: int, tol: float = 0.0) -> np.ndarray:
    """Residuals r [M][K][ny][nx] of the members u [M][K][ny][nx] against u_ref [M][ny][nx] under
    the mappings T [2][K][ny][nx] (eq. morphing-transform)."""
    u = np.asarray(u, dtype=np.float64)
    u_ref = np.asarray(u_ref, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    M, K = u.shape[0], u.shape[1]
    r = np.empty_like(u)
    for k in range(K):
        qy, qx = inverse_points(T[:, k], n_iter, tol)
        for j in range(M):
            r[j, k] = interp_periodic(u[j, k], qy, qx) - u_ref[j]
    return r


def morph_reference(ext: np.ndarray) -> np.ndarray:
    """Transformed reference member: the member mean of the extended ensemble ext [C][K][ny][nx]
    (Sec. 2.2), returned as [C][1][ny][nx]."""
    ext = np.asarray(ext, dtype=np.float64)
    return ext.mean(axis=1, keepdims=True)


def morph_inverse(ext: np.ndarray, u_ref: np.ndarray) -> np.ndarray:
    """Physical members u [M][K][ny][nx] from the extended ensemble ext [M+2][K][ny][nx] =
    (T_x, T_y, r^(1..M)) and the reference u_ref [M][ny][nx] (eq. inverse-morphing)."""
    ext = np.asarray(ext, dtype=np.float64)
    u_ref = np.asarray(u_ref, dtype=np.float64)
    M, K = ext.shape[0] - 2, ext.shape[1]
    out = np.empty((M, K) + ext.shape[2:], dtype=np.float64)
    for k in range(K):
        T = np.stack([ext[0, k], ext[1, k]])
        for j in range(M):
            out[j, k] = compose(u_ref[j] + ext[2 + j, k], T)
    return out
