"""GPU parity of the coupled observed-block analysis (fftenkf_set_coupled) against the FP64
oracle in oracle/coupled.py: analyses, spectrum tables, the singular bracket rules and the
unsupported cases.  Tolerances as in test_gpu_parity: FP32 storage 1e-5, BF16 5e-3."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import coupled, enkf  # noqa: E402
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


def _plan(p):
    from paper_1001_1588_gb300 import torch_api
    dt = torch.float32 if p.storage == "f32" else torch.bfloat16
    return torch_api.Plan(p.ny, p.nx, p.M, p.N, dt, p.observed, coupled=True)


def _analyze(p):
    plan = _plan(p)
    ens, data, pert, rhat = _gu().to_device(p)
    plan.analyze(ens, data, pert, rhat)
    st = plan.device_status()
    out = ens.float().cpu().numpy().astype(np.float64)
    plan.close()
    return out, st


def _two_observed(ny, nx, N, M, storage="f32", seed=3, rho=0.7):
    S = [fields.se_spectrum(ny, nx, l, 1.0) for l in (3.0, 6.0, 10.0, 4.0)[:M]]
    observed = [1, 1] + [0] * (M - 2)
    rh = np.full((2, ny, nx // 2 + 1), 0.1)
    return fields.make_problem(ny, nx, N, S, observed, rh, seed=seed, storage=storage, rho=rho)


@pytest.mark.parametrize("ny,nx,N,M,storage", [(64, 96, 6, 4, "f32"), (128, 128, 5, 2, "f32"),
                                               (96, 64, 8, 3, "bf16"), (256, 512, 20, 4, "bf16")])
def test_coupled_analysis_matches_oracle(ny, nx, N, M, storage):
    p = _two_observed(ny, nx, N, M, storage)
    ua, st = _analyze(p)
    assert st == 0
    ref = coupled.analyze(p.ensemble, p.data, p.perturbations, p.rhat, p.observed)
    tol = TOL32 if storage == "f32" else TOL16
    assert _gu().rel_l2(ua, ref) <= tol
    # the coupled update differs from the neglect rule on correlated observed blocks
    plain = enkf.analyze(p.ensemble, p.data, p.perturbations, p.rhat, p.observed)
    assert _gu().rel_l2(ua - p.ensemble, plain - p.ensemble) > 10 * tol


def test_coupled_single_observed_equals_plain_rule():
    p = fields.make_config2(ny=64, nx=64)
    ua, st = _analyze(p)
    assert st == 0
    ref = coupled.analyze(p.ensemble, p.data, p.perturbations, p.rhat, p.observed)
    assert _gu().rel_l2(ua, ref) <= TOL32
    ua_plain, _ = _gu().gpu_analyze(p)
    assert _gu().rel_l2(ua, ua_plain) <= TOL32


def test_coupled_spectrum_tables():
    p = _two_observed(48, 64, 5, 4)
    plan = _plan(p)
    ens, _, _, _ = _gu().to_device(p)
    spec = plan.estimate_spectrum(ens).cpu().numpy()
    assert plan.device_status() == 0
    plan.close()
    auto, cross = coupled.estimate(p.ensemble, p.observed)
    obs = [0, 1]
    K = p.ny * (p.nx // 2 + 1)
    pos = 0
    for o in obs:
        ref = enkf.full_to_half(auto[o])
        assert _gu().rel_l2(spec[pos:pos + K].reshape(ref.shape), ref) <= TOL32
        pos += K
    for o in obs:
        for j in range(p.M):
            if j == o:
                continue
            ref = enkf.full_to_half(cross[(j, o)])
            got = spec[pos:pos + 2 * K].reshape(ref.shape + (2,))
            assert _gu().rel_l2(got, np.stack([ref.real, ref.imag], axis=-1)) <= TOL32, (j, o)
            pos += 2 * K
    assert pos == spec.size


def test_coupled_rank_one_bracket_with_zero_rhat():
    """N = 2 and rhat = 0: the bracket is rank 1 at every wavenumber (pseudo-inverse rule).
    White fields keep every wavenumber's variance far above FP32 resolution, so that the
    FP32 tables resolve the rank deficiency (det / (a11 a22) ~ 1e-7 < 1e-6), as the FP64
    oracle does; with variances near the FP32 underflow the decision is not resolved."""
    ny = nx = 32
    S = [np.ones((ny, nx))] * 3
    p = fields.make_problem(ny, nx, 2, S, [1, 1, 0], np.zeros((2, ny, nx // 2 + 1)), seed=17, rho=0.7)
    ua, st = _analyze(p)
    assert st == 0 and np.all(np.isfinite(ua))
    ref = coupled.analyze(p.ensemble, p.data, p.perturbations, p.rhat, p.observed)
    assert _gu().rel_l2(ua, ref) <= 1e-4


def test_coupled_zero_bracket_keeps_forecast():
    p = _two_observed(32, 64, 4, 3)
    p.ensemble[0, :] = p.ensemble[0, 0]
    p.ensemble[1, :] = p.ensemble[1, 0]
    p.rhat[:] = 0.0
    ua, st = _analyze(p)
    assert st == 0
    np.testing.assert_array_equal(ua, p.ensemble.astype(np.float64))


def test_coupled_unsupported_cases():
    from paper_1001_1588_gb300 import abi, torch_api
    with pytest.raises(abi.FftEnkfError) as ei:
        torch_api.Plan(32, 32, 4, 3, torch.float32, [1, 1, 1, 0], coupled=True)
    assert ei.value.status == abi.FFTENKF_EUNSUPPORTED
    with pytest.raises(abi.FftEnkfError) as ei:
        torch_api.Plan(4096, 4096, 4, 20, torch.bfloat16, [1, 1, 0, 0], coupled=True)
    assert ei.value.status == abi.FFTENKF_EUNSUPPORTED
    p = _two_observed(32, 32, 3, 3)
    plan = _plan(p)
    ens, data, pert, rhat = _gu().to_device(p)
    spec = torch.zeros(plan.spectrum_doubles, dtype=torch.float64, device="cuda")
    with pytest.raises(abi.FftEnkfError) as ei:
        plan.analyze(ens, data, pert, rhat, spec)
    assert ei.value.status == abi.FFTENKF_EUNSUPPORTED
    plan.close()
