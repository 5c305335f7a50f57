"""Device-side (torch) drawing of large analysis problems, same recipe as synth.fields.

Used where NumPy synthesis of the fields would take minutes (the 4096^2,
4-block, 20-member workload).  Fields are u = F^-1(sqrt(S) . F z) with z white
N(0,1) drawn by a seeded torch generator on the device; spectra are the same
functions of the folded wavenumber as in synth.fields.
"""

from __future__ import annotations

import math
from typing import Sequence

import torch

from .fields import CONFIG3_ELLS


def _xi2_half(ny: int, nx: int, device) -> torch.Tensor:
    ky = torch.fft.fftfreq(ny, device=device, dtype=torch.float64)[:, None]
    kx = torch.fft.rfftfreq(nx, device=device, dtype=torch.float64)[None, :]
    return ky ** 2 + kx ** 2


def _normalise_half(S: torch.Tensor, nx: int, var: float) -> torch.Tensor:
    # mean over the full grid from the half spectrum (columns 1..nx/2-1 appear twice)
    w = torch.full((S.shape[-1],), 2.0, dtype=S.dtype, device=S.device)
    w[0] = 1.0
    w[-1] = 1.0
    mean = (S * w).sum() / (S.shape[0] * nx)
    return S * (var / mean)


def matern32_half(ny: int, nx: int, ell: float, device) -> torch.Tensor:
    S = (3.0 / ell ** 2 + 4.0 * math.pi ** 2 * _xi2_half(ny, nx, device)) ** -2.5
    return _normalise_half(S, nx, 1.0)


def radial_half(ny: int, nx: int, device) -> torch.Tensor:
    ky = torch.fft.fftfreq(ny, device=device, dtype=torch.float64)[:, None] * ny
    kx = torch.arange(nx // 2 + 1, device=device, dtype=torch.float64)[None, :]
    return torch.sqrt(ky ** 2 + kx ** 2)


def _field(sqrtS: torch.Tensor, z: torch.Tensor, ny: int, nx: int) -> torch.Tensor:
    Z = torch.fft.rfft2(z, norm="ortho")
    return torch.fft.irfft2(Z * sqrtS, s=(ny, nx), norm="ortho")


class DeviceProblem:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def make_config3_torch(device="cuda", seed: int = 20260003, ny: int = 4096, nx: int = 4096, N: int = 20,
                       storage=torch.bfloat16, ells: Sequence[float] = CONFIG3_ELLS, rho: float = 0.6,
                       observed=(1, 1, 0, 0)) -> DeviceProblem:
    """4 Matern-3/2 blocks, latent correlation rho, rhat = 0.1/max(|k|,1), drawn on the device."""
    M = len(ells)
    obs = [i for i in range(M) if observed[i]]
    n_obs = len(obs)
    gens = [torch.Generator(device=device) for _ in range(5)]
    for i, g in enumerate(gens):
        g.manual_seed(seed * 16 + i)
    g_truth, g_members, g_noise, g_pert, g_latent = gens
    sq = [matern32_half(ny, nx, l, device).sqrt().to(torch.float32) for l in ells]
    c = math.sqrt(1.0 - rho * rho)

    def draw(gen, z0, out=None):
        res = out if out is not None else torch.empty(M, ny, nx, device=device)
        for b in range(M):
            z = rho * z0 + c * torch.randn(ny, nx, device=device, generator=gen)
            res[b] = _field(sq[b], z, ny, nx)
        return res

    truth = draw(g_truth, torch.randn(ny, nx, device=device, generator=g_latent))
    ens = torch.empty(M, N, ny, nx, device=device, dtype=storage)
    tmp = torch.empty(M, ny, nx, device=device)
    for k in range(N):
        draw(g_members, torch.randn(ny, nx, device=device, generator=g_latent), tmp)
        ens[:, k] = tmp.to(storage)
    rhat1 = 0.1 / torch.clamp(radial_half(ny, nx, device), min=1.0)
    rhat = rhat1[None].repeat(n_obs, 1, 1).contiguous()
    sr = rhat1.sqrt().to(torch.float32)
    data = torch.empty(n_obs, ny, nx, device=device)
    for i, o in enumerate(obs):
        data[i] = truth[o] + _field(sr, torch.randn(ny, nx, device=device, generator=g_noise), ny, nx)
    pert = torch.empty(N, n_obs, ny, nx, device=device, dtype=storage)
    for k in range(N):
        for i in range(n_obs):
            pert[k, i] = _field(sr, torch.randn(ny, nx, device=device, generator=g_pert), ny, nx).to(storage)
    return DeviceProblem(ny=ny, nx=nx, M=M, N=N, observed=list(observed), obs=obs, n_obs=n_obs,
                         ensemble=ens, data=data, perturbations=pert, rhat=rhat, truth=truth,
                         storage=storage, seed=seed)


def se_half(ny: int, nx: int, ell: float, device) -> torch.Tensor:
    S = torch.exp(-2.0 * math.pi ** 2 * ell ** 2 * _xi2_half(ny, nx, device))
    return _normalise_half(S, nx, 1.0)


def make_batched_torch(device="cuda", count: int = 256, seed: int = 20260004, storage=torch.float32,
                       sides=None, n_range=(5, 25)):
    """The batched workload (independent single-block analyses of uneven sizes) drawn on the
    device: shapes and parameters from synth.fields.batched_item_params, SE fields, flat rhat."""
    from .fields import BATCH_SIDES, batched_item_params
    items = []
    for it in batched_item_params(count, seed, sides or BATCH_SIDES, n_range):
        ny, nx, N = it["ny"], it["nx"], it["N"]
        g = torch.Generator(device=device)
        g.manual_seed(it["seed"])
        sq = se_half(ny, nx, it["ell"], device).sqrt().to(torch.float32)
        truth = _field(sq, torch.randn(ny, nx, device=device, generator=g), ny, nx)
        ens = torch.empty(N, ny, nx, device=device, dtype=storage)
        for k in range(N):
            ens[k] = _field(sq, torch.randn(ny, nx, device=device, generator=g), ny, nx).to(storage)
        r = it["r"]
        data = (truth + math.sqrt(r) * torch.randn(ny, nx, device=device, generator=g)).contiguous()
        pert = (math.sqrt(r) * torch.randn(N, ny, nx, device=device, generator=g)).to(storage).contiguous()
        rhat = torch.full((ny, nx // 2 + 1), r, device=device, dtype=torch.float64)
        items.append(DeviceProblem(ny=ny, nx=nx, N=N, ensemble=ens, data=data, perturbations=pert, rhat=rhat,
                                   truth=truth, ell=it["ell"], r=r))
    return items
