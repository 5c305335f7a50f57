"""GPU parity of the real sine transform variant (fftenkf_sine_*, Sec. 4) against the FP64 oracle
in oracle/sine.py: analyses, spectrum tables, the untouched boundary, and the unsupported sizes.
Tolerances as in test_gpu_parity: FP32 storage 1e-5, BF16 5e-3."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sine  # noqa: E402
from synth import fields  # noqa: E402

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 5e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_1588_gb300 import abi
    abi.lib()


def _gu():
    from tests import gpu_util
    return gpu_util


def _problem(ny, nx, M, N, observed, storage, seed, ells=(4.0, 9.0, 16.0, 6.0)):
    S = [fields.se_spectrum(ny, nx, l, 1.0) for l in ells[:M]]
    n_obs = int(np.sum(observed))
    return fields.make_problem(ny, nx, N, S, observed, np.full((n_obs, ny, nx // 2 + 1), 0.1), seed=seed,
                               storage=storage, rho=0.6)


def _sine_rhat(n_obs, ny, nx, kind):
    if kind == "flat":
        return np.full((n_obs, ny - 2, nx - 2), 0.1)
    ky = np.arange(1, ny - 1)[:, None]
    kx = np.arange(1, nx - 1)[None, :]
    return np.repeat((0.1 / np.sqrt(ky ** 2 + kx ** 2))[None], n_obs, axis=0)


def _run(p, rhat):
    from paper_1001_1588_gb300 import torch_api
    dt = torch.float32 if p.storage == "f32" else torch.bfloat16
    plan = torch_api.SinePlan(p.ny, p.nx, p.M, p.N, dt, p.observed)
    ens, data, pert, _ = _gu().to_device(p)
    r = torch.from_numpy(np.ascontiguousarray(rhat)).cuda()
    plan.analyze(ens, data, pert, r)
    st = plan.device_status()
    out = ens.float().cpu().numpy().astype(np.float64)
    plan.close()
    return out, st


@pytest.mark.parametrize("ny,nx,M,N,observed,storage,kind", [
    (33, 33, 1, 5, [1], "f32", "flat"),
    (49, 65, 3, 5, [1, 0, 0], "f32", "flat"),
    (65, 97, 4, 6, [1, 1, 0, 0], "bf16", "inverse"),
    (257, 129, 2, 8, [1, 0], "bf16", "flat"),
    (97, 193, 3, 4, [0, 1, 1], "f32", "inverse"),
])
def test_sine_analysis_matches_oracle(ny, nx, M, N, observed, storage, kind):
    p = _problem(ny, nx, M, N, observed, storage, seed=ny + nx)
    rhat = _sine_rhat(int(np.sum(observed)), ny, nx, kind)
    ua, st = _run(p, rhat)
    assert st == 0
    ref = sine.analyze(p.ensemble, p.data, p.perturbations, rhat, p.observed)
    tol = TOL32 if storage == "f32" else TOL16
    assert _gu().rel_l2(ua, ref) <= tol
    # the boundary nodes are returned exactly as given
    for sl in (np.s_[..., 0, :], np.s_[..., -1, :], np.s_[..., :, 0], np.s_[..., :, -1]):
        np.testing.assert_array_equal(ua[sl], p.ensemble[sl])
    # the increment itself, not only the state, is within tolerance
    assert _gu().rel_l2(ua - p.ensemble, ref - p.ensemble) <= (1e-4 if storage == "f32" else 2e-2)


def test_sine_analysis_several_tiles_bf16():
    """A grid whose extension spans several row and column tiles (1024 x 1024 periodic)."""
    p = _problem(513, 513, 2, 8, [1, 0], "bf16", seed=7)
    rhat = _sine_rhat(1, 513, 513, "inverse")
    ua, st = _run(p, rhat)
    assert st == 0
    ref = sine.analyze(p.ensemble, p.data, p.perturbations, rhat, p.observed)
    assert _gu().rel_l2(ua, ref) <= TOL16


def test_sine_spectrum_tables():
    from paper_1001_1588_gb300 import torch_api
    p = _problem(49, 33, 3, 6, [1, 0, 1], "f32", seed=3)
    plan = torch_api.SinePlan(p.ny, p.nx, p.M, p.N, torch.float32, p.observed)
    ens, _, _, _ = _gu().to_device(p)
    got = plan.estimate_spectrum(ens).cpu().numpy()
    assert plan.device_status() == 0
    plan.close()
    ref = sine.spectrum_tables(p.ensemble, p.observed)
    assert got.size == ref.size
    for t in range(ref.shape[0]):
        assert _gu().rel_l2(got.reshape(ref.shape)[t], ref[t]) <= TOL32, t


def test_sine_unobserved_plan_keeps_forecast():
    from paper_1001_1588_gb300 import torch_api
    plan = torch_api.SinePlan(33, 33, 2, 3, torch.float32, [0, 0])
    ens = torch.randn(2, 3, 33, 33, device="cuda")
    before = ens.clone()
    plan.analyze(ens, torch.zeros(0, 33, 33, device="cuda"), torch.zeros(3, 0, 33, 33, device="cuda"),
                 torch.zeros(0, 31, 31, dtype=torch.float64, device="cuda"))
    assert torch.equal(ens, before)
    plan.close()


def test_sine_unsupported_sizes():
    from paper_1001_1588_gb300 import abi, torch_api
    for ny, nx in ((420, 420), (33, 2), (4098, 33), (8, 33)):
        with pytest.raises(abi.FftEnkfError) as ei:
            torch_api.SinePlan(ny, nx, 1, 4, torch.float32, [1])
        assert ei.value.status in (abi.FFTENKF_EUNSUPPORTED, abi.FFTENKF_EINVAL)


def test_sine_full_size_properties():
    """The size the benchmark times (2049 x 2049 nodes, 4 blocks, 20 members, BF16; periodic
    extension 4096 x 4096): status 0, finite output, the boundary returned exactly, and a
    sampled observed member moved by the analysis."""
    from paper_1001_1588_gb300 import torch_api
    g = torch.Generator(device="cuda").manual_seed(20260003)
    ny = nx = 2049
    ens = (torch.randn(4, 20, ny, nx, device="cuda", generator=g)).to(torch.bfloat16)
    data = torch.randn(2, ny, nx, device="cuda", generator=g)
    pert = (0.3 * torch.randn(20, 2, ny, nx, device="cuda", generator=g)).to(torch.bfloat16)
    rhat = torch.full((2, ny - 2, nx - 2), 0.1, dtype=torch.float64, device="cuda")
    before = ens.clone()
    plan = torch_api.SinePlan(ny, nx, 4, 20, torch.bfloat16, [1, 1, 0, 0])
    plan.analyze(ens, data, pert, rhat)
    assert plan.device_status() == 0
    plan.close()
    assert torch.isfinite(ens.float()).all()
    for sl in (np.s_[..., 0, :], np.s_[..., -1, :], np.s_[..., :, 0], np.s_[..., :, -1]):
        assert torch.equal(ens[sl], before[sl])
    inc = (ens.float() - before.float())[0, 3].double().cpu().numpy()
    assert np.max(np.abs(inc[1:-1, 1:-1])) > 0.1                   # the analysis did move the state
