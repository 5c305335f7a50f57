"""Helpers shared by the GPU parity tests: upload problems, call the library, compare with the oracle."""

from __future__ import annotations

import numpy as np
import torch

from paper_1001_1588_gb300 import torch_api
from synth import fields


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm((got - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-300))


def to_device(p: fields.Problem, dev="cuda"):
    """Device tensors of a problem in the storage dtype the library expects."""
    dt = torch.float32 if p.storage == "f32" else torch.bfloat16
    ens = torch.from_numpy(np.ascontiguousarray(p.ensemble)).to(dev).to(dt).contiguous()
    pert = torch.from_numpy(np.ascontiguousarray(p.perturbations)).to(dev).to(dt).contiguous()
    data = torch.from_numpy(np.ascontiguousarray(p.data, dtype=np.float32)).to(dev)
    rhat = torch.from_numpy(np.ascontiguousarray(p.rhat, dtype=np.float64)).to(dev)
    return ens, data, pert, rhat


def plan_for(p: fields.Problem) -> torch_api.Plan:
    dt = torch.float32 if p.storage == "f32" else torch.bfloat16
    return torch_api.Plan(p.ny, p.nx, p.M, p.N, dt, p.observed)


def gpu_analyze(p: fields.Problem, spectrum=None):
    plan = plan_for(p)
    ens, data, pert, rhat = to_device(p)
    spec = None if spectrum is None else torch.from_numpy(np.ascontiguousarray(spectrum, dtype=np.float64)).cuda()
    plan.analyze(ens, data, pert, rhat, spec)
    st = plan.device_status()
    out = ens.float().cpu().numpy().astype(np.float64)
    plan.close()
    return out, st


def gpu_spectrum(p: fields.Problem):
    plan = plan_for(p)
    ens, _, _, _ = to_device(p)
    out = plan.estimate_spectrum(ens)
    st = plan.device_status()
    res = out.cpu().numpy()
    plan.close()
    return res, st
