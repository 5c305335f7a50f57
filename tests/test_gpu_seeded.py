"""GPU parity of fftenkf_analyze_seeded (perturbations drawn by the library in frequency space)
against the FP64 oracle: the oracle draws the same perturbations (oracle/perturb.py, its own
implementation of the generator's definition) and runs the plain analysis with them.
Tolerances as in test_gpu_parity: FP32 storage 1e-5, BF16 5e-3."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import coupled, enkf, perturb  # noqa: E402
from synth import fields  # noqa: E402

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 5e-3
SEED = 0x1234_5678_9ABC


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_1588_gb300 import abi
    abi.lib()


def _gu():
    from tests import gpu_util
    return gpu_util


def _seeded(p, seed, spectrum=None, coupled_mode=False):
    from paper_1001_1588_gb300 import torch_api
    dt = torch.float32 if p.storage == "f32" else torch.bfloat16
    plan = torch_api.Plan(p.ny, p.nx, p.M, p.N, dt, p.observed, coupled=coupled_mode)
    ens, data, _, rhat = _gu().to_device(p)
    spec = None if spectrum is None else torch.from_numpy(np.ascontiguousarray(spectrum)).cuda()
    plan.analyze_seeded(ens, data, rhat, seed, spec)
    st = plan.device_status()
    out = ens.float().cpu().numpy().astype(np.float64)
    plan.close()
    return out, st


def _oracle_pert(p, seed):
    return perturb.perturbations(p.ny, p.nx, p.rhat, seed, p.N)


@pytest.mark.parametrize("which", ["config1", "config2", "config3_bf16", "config3_f32",
                                   "config3_fused_bf16", "config3_fused_f32", "config2_fused"])
def test_seeded_analysis_matches_oracle(which):
    # the *_fused shapes (columns of 512 or more points, 1-2 observed blocks) draw the
    # perturbations inside the fused column pass, the others inside the separate column update
    if which == "config1":
        p, tol = fields.make_config1(ny=64, nx=64), TOL32
    elif which == "config2":
        p, tol = fields.make_config2(ny=128, nx=256), TOL32
    elif which == "config3_bf16":
        p, tol = fields.make_config3(ny=64, nx=96, N=6, storage="bf16"), TOL16
    elif which == "config3_f32":
        p, tol = fields.make_config3(ny=96, nx=64, N=5, storage="f32"), TOL32
    elif which == "config3_fused_bf16":
        p, tol = fields.make_config3(ny=1024, nx=64, N=6, storage="bf16"), TOL16
    elif which == "config3_fused_f32":
        p, tol = fields.make_config3(ny=4096, nx=32, N=4, storage="f32"), TOL32
    else:
        p, tol = fields.make_config2(ny=512, nx=128), TOL32
    ua, st = _seeded(p, SEED)
    assert st == 0
    e = _oracle_pert(p, SEED)
    ref = enkf.analyze(p.ensemble, p.data, e, p.rhat, p.observed)
    err = _gu().rel_l2(ua, ref)
    assert err <= tol
    # the drawn perturbations are applied: the analysis without them is at least 4x farther away
    no_e = enkf.analyze(p.ensemble, p.data, np.zeros_like(e), p.rhat, p.observed)
    assert _gu().rel_l2(ua, no_e) > 4 * err


def test_seeded_is_deterministic_per_seed():
    p = fields.make_config3(ny=64, nx=64, N=4, storage="bf16")
    a, _ = _seeded(p, 7)
    b, _ = _seeded(p, 7)
    c, _ = _seeded(p, 8)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_seeded_with_supplied_spectrum():
    p = fields.make_config1(seed=5, ny=64, nx=96)
    tables = enkf.spectrum_to_tables(enkf.Spectrum({0: p.spectra[0]}, {}), [1])
    ua, st = _seeded(p, SEED, spectrum=tables)
    assert st == 0
    e = _oracle_pert(p, SEED)
    ref = enkf.analyze(p.ensemble, p.data, e, p.rhat, p.observed, spectrum=tables)
    assert _gu().rel_l2(ua, ref) <= TOL32


def test_seeded_with_coupled_observed_blocks():
    S = [fields.se_spectrum(64, 64, l, 1.0) for l in (3.0, 6.0, 10.0)]
    p = fields.make_problem(64, 64, 5, S, [1, 1, 0], np.full((2, 64, 33), 0.1), seed=21, rho=0.7)
    ua, st = _seeded(p, SEED, coupled_mode=True)
    assert st == 0
    ref = coupled.analyze(p.ensemble, p.data, _oracle_pert(p, SEED), p.rhat, p.observed)
    assert _gu().rel_l2(ua, ref) <= TOL32
