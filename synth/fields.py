"""Stationary Gaussian random fields and complete analysis problems (NumPy).

Every field is drawn on a doubly periodic ny x nx grid (x fastest) as
u = F^-1( sqrt(S) . F z ), with z white N(0,1), F the unitary 2-D DFT and S a
spectral density normalised so that its mean over the grid equals the point
variance.  Random streams come from ``numpy.random.SeedSequence(seed).spawn(5)``
in the order: truth, members, data noise, perturbations, latent fields.

Conventions shared with the library boundary:
  ensemble       [M][N][ny][nx]   values exactly representable in the storage dtype
  data           [n_obs][ny][nx]  float32
  perturbations  [N][n_obs][ny][nx]  storage dtype
  rhat           [n_obs][ny][nx/2+1] float64, spectral data-error variance in
                 unitary-DFT units (white noise of variance r has rhat == r)
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

STREAMS = ("truth", "members", "data_noise", "perturbations", "latent")


# --------------------------------------------------------------------------
# storage rounding (float32 <-> bfloat16 bit patterns, round to nearest even)
# --------------------------------------------------------------------------
def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even); return uint16 bits."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16).astype(np.uint16)
    nan = np.isnan(x)
    if nan.any():
        r = r.copy()
        r[nan] = 0x7FC0
    return r


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.ascontiguousarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def round_to_storage(x: np.ndarray, storage: str) -> np.ndarray:
    """Values of ``x`` rounded to the storage dtype, returned as float32."""
    x32 = np.asarray(x, dtype=np.float32)
    if storage == "f32":
        return x32.copy()
    if storage == "bf16":
        return bf16_bits_to_f32(f32_to_bf16_bits(x32))
    raise ValueError(storage)


# --------------------------------------------------------------------------
# spectra on the full grid
# --------------------------------------------------------------------------
def folded_wavenumbers(ny: int, nx: int):
    """Integer wavenumbers (cycles per domain) folded to [-n/2, n/2), full grid."""
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.fftfreq(nx) * nx
    return ky[:, None], kx[None, :]


def _xi2(ny: int, nx: int) -> np.ndarray:
    ky, kx = folded_wavenumbers(ny, nx)
    return (ky / ny) ** 2 + (kx / nx) ** 2


def _normalise(S: np.ndarray, var: float) -> np.ndarray:
    return S * (var / S.mean())


def se_spectrum(ny: int, nx: int, ell: float, var: float = 1.0) -> np.ndarray:
    """Squared-exponential covariance exp(-|h|^2/(2 ell^2)) (ell in cells)."""
    return _normalise(np.exp(-2.0 * np.pi ** 2 * ell ** 2 * _xi2(ny, nx)), var)


def matern32_spectrum(ny: int, nx: int, ell: float, var: float = 1.0) -> np.ndarray:
    """Matern nu=3/2 covariance in two dimensions: S ~ (3/ell^2 + 4 pi^2 |xi|^2)^(-5/2)."""
    return _normalise((3.0 / ell ** 2 + 4.0 * np.pi ** 2 * _xi2(ny, nx)) ** -2.5, var)


def powerlaw_spectrum(ny: int, nx: int, ell: float, beta: float, var: float = 1.0) -> np.ndarray:
    """S ~ (1 + (2 pi ell |xi|)^2)^(beta/2), beta < 0."""
    return _normalise((1.0 + 4.0 * np.pi ** 2 * ell ** 2 * _xi2(ny, nx)) ** (beta / 2.0), var)


def radial_wavenumber_half(ny: int, nx: int) -> np.ndarray:
    """|k| in integer units on the half spectrum [ny][nx/2+1]."""
    ky = np.fft.fftfreq(ny) * ny
    kx = np.arange(nx // 2 + 1, dtype=np.float64)
    return np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)


def half_to_full_even(h: np.ndarray, nx: int) -> np.ndarray:
    """Extend an even (real) half-spectrum table [.., ny, nx/2+1] to the full grid."""
    ny = h.shape[-2]
    full = np.empty(h.shape[:-1] + (nx,), dtype=h.dtype)
    full[..., : nx // 2 + 1] = h
    ky_neg = (-np.arange(ny)) % ny
    for kx in range(nx // 2 + 1, nx):
        full[..., :, kx] = h[..., ky_neg, nx - kx]
    return full


# --------------------------------------------------------------------------
# field synthesis
# --------------------------------------------------------------------------
def gaussian_field(S: np.ndarray, z: np.ndarray) -> np.ndarray:
    """u = F^-1(sqrt(S) . F z) with the unitary DFT; S even, z real white noise."""
    Z = np.fft.fft2(z, norm="ortho")
    return np.fft.ifft2(np.sqrt(S) * Z, norm="ortho").real


@dataclass
class Problem:
    """One analysis problem, every array in the layout the library expects."""

    ny: int
    nx: int
    M: int
    N: int
    observed: np.ndarray                # uint8 [M]
    storage: str                        # "f32" or "bf16"
    ensemble: np.ndarray                # float32 [M][N][ny][nx], storage-exact
    data: np.ndarray                    # float32 [n_obs][ny][nx]
    perturbations: np.ndarray           # float32 [N][n_obs][ny][nx], storage-exact
    rhat: np.ndarray                    # float64 [n_obs][ny][nx/2+1]
    truth: np.ndarray                   # float64 [M][ny][nx]
    spectra: List[np.ndarray] = field(default_factory=list)   # generating S per block (full grid)
    meta: dict = field(default_factory=dict)

    @property
    def n_obs(self) -> int:
        return int(np.count_nonzero(self.observed))

    @property
    def obs_index(self) -> List[int]:
        return [int(i) for i in np.flatnonzero(self.observed)]

    def ensemble_storage(self) -> np.ndarray:
        """Ensemble in its storage encoding (float32, or uint16 bfloat16 bits)."""
        return self.ensemble if self.storage == "f32" else f32_to_bf16_bits(self.ensemble)

    def perturbations_storage(self) -> np.ndarray:
        return self.perturbations if self.storage == "f32" else f32_to_bf16_bits(self.perturbations)


def _streams(seed: int):
    return [np.random.Generator(np.random.PCG64(s)) for s in np.random.SeedSequence(seed).spawn(len(STREAMS))]


def make_problem(
    ny: int,
    nx: int,
    N: int,
    spectra: Sequence[np.ndarray],
    observed: Sequence[int],
    rhat_half: np.ndarray,
    seed: int,
    storage: str = "f32",
    sigma2: Optional[Sequence[float]] = None,
    rho: float = 0.0,
    mean: Optional[Sequence[float]] = None,
) -> Problem:
    """Draw truth, N members, data and perturbations for an M-block state.

    Block b of a draw is sigma_b * F^-1(sqrt(S_b) . F(rho z0 + sqrt(1-rho^2) z_b)):
    ``spectra`` are normalised to mean 1 internally and scaled by sigma2[b]; a
    shared latent white field z0 per draw correlates the blocks (rho = 0: none).
    Data on observed block o is truth^(o) plus noise with spectral variance
    rhat_o; perturbation e_{k,o} is an independent draw of the same noise.
    """
    M = len(spectra)
    observed = np.asarray(observed, dtype=np.uint8)
    assert observed.shape == (M,)
    obs = [int(i) for i in np.flatnonzero(observed)]
    n_obs = len(obs)
    if sigma2 is None:
        sigma2 = [float(S.mean()) for S in spectra]
    shape_S = [S / S.mean() for S in spectra]
    mean = [0.0] * M if mean is None else list(mean)
    rhat_half = np.asarray(rhat_half, dtype=np.float64).reshape(n_obs, ny, nx // 2 + 1)
    g_truth, g_members, g_noise, g_pert, g_latent = _streams(seed)
    c = np.sqrt(max(0.0, 1.0 - rho * rho))

    def draw(gen_blocks, z0):
        out = np.empty((M, ny, nx))
        for b in range(M):
            zb = gen_blocks.standard_normal((ny, nx))
            z = rho * z0 + c * zb if rho != 0.0 else zb
            out[b] = mean[b] + np.sqrt(sigma2[b]) * gaussian_field(shape_S[b], z)
        return out

    truth = draw(g_truth, g_latent.standard_normal((ny, nx)))
    ens = np.empty((M, N, ny, nx))
    for k in range(N):
        z0 = g_latent.standard_normal((ny, nx))
        ens[:, k] = draw(g_members, z0)
    r_full = [half_to_full_even(rhat_half[i], nx) for i in range(n_obs)]
    data = np.empty((n_obs, ny, nx))
    for i, o in enumerate(obs):
        data[i] = truth[o] + gaussian_field(r_full[i], g_noise.standard_normal((ny, nx)))
    pert = np.empty((N, n_obs, ny, nx))
    for k in range(N):
        for i in range(n_obs):
            pert[k, i] = gaussian_field(r_full[i], g_pert.standard_normal((ny, nx)))
    return Problem(
        ny=ny, nx=nx, M=M, N=N, observed=observed, storage=storage,
        ensemble=round_to_storage(ens, storage),
        data=data.astype(np.float32),
        perturbations=round_to_storage(pert, storage),
        rhat=rhat_half.copy(),
        truth=truth,
        spectra=[np.asarray(s, dtype=np.float64) * 1.0 for s in spectra],
        meta={"seed": seed, "rho": rho, "sigma2": list(sigma2)},
    )


# --------------------------------------------------------------------------
# the five workloads (config index i uses seed 20260000 + i)
# --------------------------------------------------------------------------
def make_config1(seed: int = 20260001, ny: int = 64, nx: int = 64, N: int = 5) -> Problem:
    """1 block, SE spectrum ell=8 var 1, H=I, rhat=0.1 flat, FP32 storage."""
    S = se_spectrum(ny, nx, 8.0, 1.0)
    rh = np.full((1, ny, nx // 2 + 1), 0.1)
    p = make_problem(ny, nx, N, [S], [1], rh, seed, "f32")
    p.meta["config"] = "plain 1 block %dx%d N=%d" % (ny, nx, N)
    return p


def make_config2(seed: int = 20260002, ny: int = 512, nx: int = 512, N: int = 5) -> Problem:
    """3 blocks (SE ell 4/16/32, var 1/0.5/2, latent rho 0.6), block 0 observed, rhat 0.05."""
    spectra = [se_spectrum(ny, nx, l, v) for l, v in ((4.0, 1.0), (16.0, 0.5), (32.0, 2.0))]
    rh = np.full((1, ny, nx // 2 + 1), 0.05)
    p = make_problem(ny, nx, N, spectra, [1, 0, 0], rh, seed, "f32", sigma2=[1.0, 0.5, 2.0], rho=0.6)
    p.meta["config"] = "plain 3 blocks %dx%d N=%d" % (ny, nx, N)
    return p


CONFIG3_ELLS = (8.0, 8.0 * 16.0 ** (1 / 3), 8.0 * 16.0 ** (2 / 3), 128.0)


def config3_rhat(ny: int, nx: int, n_obs: int = 2) -> np.ndarray:
    """rhat(k) = 0.1 / max(|k|, 1) on the half spectrum, |k| in integer units."""
    r = 0.1 / np.maximum(radial_wavenumber_half(ny, nx), 1.0)
    return np.repeat(r[None], n_obs, axis=0)


def make_config3(seed: int = 20260003, ny: int = 4096, nx: int = 4096, N: int = 20,
                 storage: str = "bf16") -> Problem:
    """4 blocks, Matern-3/2 ell 8..128 (geometric), rho 0.6, blocks 0,1 observed,
    rhat ~ 0.1/|k|, BF16 storage.  NumPy version: use for reduced sizes only."""
    spectra = [matern32_spectrum(ny, nx, l, 1.0) for l in CONFIG3_ELLS]
    p = make_problem(ny, nx, N, spectra, [1, 1, 0, 0], config3_rhat(ny, nx), seed, storage,
                     sigma2=[1.0] * 4, rho=0.6)
    p.meta["config"] = "large 4 blocks %dx%d N=%d %s" % (ny, nx, N, storage)
    return p


BATCH_SIDES = (64, 96, 128, 192, 256, 384, 512, 768, 1024)


def batched_item_params(count: int = 256, seed: int = 20260004, sides: Sequence[int] = BATCH_SIDES,
                        n_range=(5, 25)):
    """Shapes and parameters of the batched workload (no fields drawn)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    items = []
    for i in range(count):
        s = int(rng.choice(np.asarray(sides)))
        square = bool(rng.random() < 0.5)
        ny, nx = (s, s) if square else (s // 2, s)
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        ell = float(np.exp(rng.uniform(np.log(2.0), np.log(64.0))))
        r = float(np.exp(rng.uniform(np.log(0.01), np.log(1.0))))
        items.append(dict(ny=ny, nx=nx, N=N, ell=ell, r=r, seed=int(rng.integers(1 << 31))))
    return items


def make_batched_items(count: int = 256, seed: int = 20260004, sides: Sequence[int] = BATCH_SIDES,
                       n_range=(5, 25)) -> List[Problem]:
    """Independent single-block analyses of uneven sizes (SE spectra, flat rhat)."""
    out = []
    for it in batched_item_params(count, seed, sides, n_range):
        ny, nx = it["ny"], it["nx"]
        S = se_spectrum(ny, nx, it["ell"], 1.0)
        rh = np.full((1, ny, nx // 2 + 1), it["r"])
        p = make_problem(ny, nx, it["N"], [S], [1], rh, it["seed"], "f32")
        p.meta.update(it)
        out.append(p)
    return out


def smooth_mappings(seed: int, K: int, ny: int, nx: int, amp: float, ell: float) -> np.ndarray:
    """K random smooth displacement fields T_k = (T_x, T_y), float32 [2][K][ny][nx], in grid units
    (Sec. 2.2: random smooth mappings from Fourier series whose coefficients decay quickly; here a
    squared-exponential spectrum of length ell cells), each component scaled to max |T| = amp."""
    rng = np.random.Generator(np.random.PCG64(seed))
    S = se_spectrum(ny, nx, ell)
    T = np.empty((2, K, ny, nx), dtype=np.float32)
    for c in range(2):
        for k in range(K):
            g = gaussian_field(S, rng.standard_normal((ny, nx)))
            T[c, k] = (amp * g / max(np.abs(g).max(), 1e-30)).astype(np.float32)
    return T


def smooth_members(seed: int, M: int, K: int, ny: int, nx: int, ell: float) -> np.ndarray:
    """M x K unit-variance squared-exponential fields, float32 [M][K][ny][nx]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    S = se_spectrum(ny, nx, ell)
    u = np.empty((M, K, ny, nx), dtype=np.float32)
    for j in range(M):
        for k in range(K):
            u[j, k] = gaussian_field(S, rng.standard_normal((ny, nx))).astype(np.float32)
    return u
