"""Thin wrapper over the C ABI for torch CUDA tensors: checks shapes/dtypes and passes pointers.

PyTorch supplies device memory and the current stream only; every step of the
analysis runs in the library's kernels.
"""

from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import abi

_STORAGE = {torch.float32: abi.FFTENKF_F32, torch.bfloat16: abi.FFTENKF_BF16}


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Plan:
    """One (grid, blocks, members, storage, observed mask) configuration."""

    def __init__(self, ny: int, nx: int, n_blocks: int, n_members: int, storage: torch.dtype,
                 observed: Sequence[int], coupled: bool = False):
        if storage not in _STORAGE:
            raise TypeError("storage must be torch.float32 or torch.bfloat16")
        self.ny, self.nx, self.M, self.N = ny, nx, n_blocks, n_members
        self.dtype = storage
        self.observed = [int(bool(o)) for o in observed]
        self.n_obs = sum(self.observed)
        self.handle = abi.fftenkf_plan_create(ny, nx, n_blocks, n_members, _STORAGE[storage], self.observed)
        if coupled:
            try:
                abi.fftenkf_set_coupled(self.handle, True)
            except Exception:
                self.close()
                raise
        self.coupled = bool(coupled)
        self.workspace_bytes = abi.fftenkf_workspace_size(self.handle)
        self.spectrum_doubles = abi.fftenkf_spectrum_size(self.handle)
        self._ws = None

    def close(self):
        if self.handle:
            abi.fftenkf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace(self, device="cuda") -> torch.Tensor:
        if self._ws is None:
            self._ws = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=device)
        return self._ws

    def _check(self, t: torch.Tensor, shape, dtype, name):
        if not t.is_cuda or tuple(t.shape) != tuple(shape) or t.dtype != dtype or not t.is_contiguous():
            raise ValueError("%s: expected contiguous CUDA %s %s, got %s %s %s" % (
                name, dtype, tuple(shape), t.device, t.dtype, tuple(t.shape)))

    def estimate_spectrum(self, ensemble: torch.Tensor, out: Optional[torch.Tensor] = None,
                          stream=None) -> torch.Tensor:
        self._check(ensemble, (self.M, self.N, self.ny, self.nx), self.dtype, "ensemble")
        if out is None:
            out = torch.empty(self.spectrum_doubles, dtype=torch.float64, device=ensemble.device)
        abi.fftenkf_estimate_spectrum(self.handle, ensemble, out, self.workspace(ensemble.device),
                                      _stream_handle(stream))
        return out

    def analyze(self, ensemble: torch.Tensor, data: torch.Tensor, perturbations: torch.Tensor,
                rhat: torch.Tensor, spectrum: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """In-place analysis of ``ensemble``; returns it."""
        self._check(ensemble, (self.M, self.N, self.ny, self.nx), self.dtype, "ensemble")
        self._check(data, (self.n_obs, self.ny, self.nx), torch.float32, "data")
        self._check(perturbations, (self.N, self.n_obs, self.ny, self.nx), self.dtype, "perturbations")
        self._check(rhat, (self.n_obs, self.ny, self.nx // 2 + 1), torch.float64, "rhat")
        if spectrum is not None:
            self._check(spectrum, (self.spectrum_doubles,), torch.float64, "spectrum")
        abi.fftenkf_analyze(self.handle, ensemble, data, perturbations, rhat, spectrum,
                            self.workspace(ensemble.device), _stream_handle(stream))
        return ensemble

    def analyze_seeded(self, ensemble: torch.Tensor, data: torch.Tensor, rhat: torch.Tensor, seed: int,
                       spectrum: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """In-place analysis with the perturbations drawn by the library from ``seed``; returns ``ensemble``."""
        self._check(ensemble, (self.M, self.N, self.ny, self.nx), self.dtype, "ensemble")
        self._check(data, (self.n_obs, self.ny, self.nx), torch.float32, "data")
        self._check(rhat, (self.n_obs, self.ny, self.nx // 2 + 1), torch.float64, "rhat")
        if spectrum is not None:
            self._check(spectrum, (self.spectrum_doubles,), torch.float64, "spectrum")
        abi.fftenkf_analyze_seeded(self.handle, ensemble, data, rhat, seed, spectrum,
                                   self.workspace(ensemble.device), _stream_handle(stream))
        return ensemble

    def device_status(self, stream=None) -> int:
        return abi.fftenkf_last_device_status(self.handle, _stream_handle(stream))


class SinePlan:
    """The real sine transform variant (Sec. 4): grid ny x nx including its boundary nodes, which
    the analysis leaves unchanged; the interior is analysed in the orthonormal DST-I basis."""

    def __init__(self, ny: int, nx: int, n_blocks: int, n_members: int, storage: torch.dtype,
                 observed: Sequence[int]):
        if storage not in _STORAGE:
            raise TypeError("storage must be torch.float32 or torch.bfloat16")
        self.ny, self.nx, self.M, self.N = ny, nx, n_blocks, n_members
        self.dtype = storage
        self.observed = [int(bool(o)) for o in observed]
        self.n_obs = sum(self.observed)
        self.handle = abi.fftenkf_sine_plan_create(ny, nx, n_blocks, n_members, _STORAGE[storage], self.observed)
        self.spectrum_doubles = abi.fftenkf_sine_spectrum_size(self.handle)

    def close(self):
        if self.handle:
            abi.fftenkf_sine_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    _check = Plan._check

    def estimate_spectrum(self, ensemble: torch.Tensor, out: Optional[torch.Tensor] = None,
                          stream=None) -> torch.Tensor:
        self._check(ensemble, (self.M, self.N, self.ny, self.nx), self.dtype, "ensemble")
        if out is None:
            out = torch.empty(self.spectrum_doubles, dtype=torch.float64, device=ensemble.device)
        abi.fftenkf_sine_estimate_spectrum(self.handle, ensemble, out, _stream_handle(stream))
        return out

    def analyze(self, ensemble: torch.Tensor, data: torch.Tensor, perturbations: torch.Tensor,
                rhat: torch.Tensor, stream=None) -> torch.Tensor:
        """In-place analysis of ``ensemble``; rhat [n_obs][ny-2][nx-2] per sine wavenumber."""
        self._check(ensemble, (self.M, self.N, self.ny, self.nx), self.dtype, "ensemble")
        self._check(data, (self.n_obs, self.ny, self.nx), torch.float32, "data")
        self._check(perturbations, (self.N, self.n_obs, self.ny, self.nx), self.dtype, "perturbations")
        self._check(rhat, (self.n_obs, self.ny - 2, self.nx - 2), torch.float64, "rhat")
        abi.fftenkf_sine_analyze(self.handle, ensemble, data, perturbations, rhat, _stream_handle(stream))
        return ensemble

    def device_status(self, stream=None) -> int:
        return abi.fftenkf_sine_last_device_status(self.handle, _stream_handle(stream))
