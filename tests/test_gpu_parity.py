"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Tolerances (relative L2 over the whole output array): 1e-5 for FP32 storage,
5e-3 for BF16 storage (inputs, output and perturbations stored as bfloat16;
the comparison is with the oracle's unrounded FP64 result on the same rounded
inputs).  Spectra are compared table by table, whole-array relative L2.
"""

import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import enkf  # noqa: E402
from synth import fields  # noqa: E402

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 5e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_1588_gb300 import abi
    abi.lib()   # raises if the library has not been built


def _gu():
    from tests import gpu_util
    return gpu_util


def _oracle(p, spectrum=None):
    return enkf.analyze(p.ensemble, p.data, p.perturbations, p.rhat, p.observed, spectrum=spectrum)


def _tables(p):
    return enkf.spectrum_to_tables(enkf.estimate_spectrum(p.ensemble, p.observed), p.observed)


def _check_problem(p, tol):
    gu = _gu()
    ua, st = gu.gpu_analyze(p)
    assert st == 0
    ref = _oracle(p)
    e = gu.rel_l2(ua, ref)
    inc = gu.rel_l2(ua - p.ensemble, ref - p.ensemble)
    assert e <= tol, "analysis rel-L2 %.3e (increment %.3e)" % (e, inc)
    # the increment u^a - u on its own, at 10x the storage tolerance: the forecast dominates u^a,
    # so an error of the update could hide inside the analysis's relative error
    assert inc <= 10 * tol, "increment rel-L2 %.3e" % inc
    spec, st = gu.gpu_spectrum(p)
    assert st == 0
    es = gu.rel_l2(spec, _tables(p))
    assert es <= tol, "spectrum rel-L2 %.3e" % es
    return e, es


def test_config1_plain_64():
    _check_problem(fields.make_config1(), TOL32)


def test_config2_three_blocks_512():
    _check_problem(fields.make_config2(), TOL32)


@pytest.mark.parametrize("n", [128, 256])
def test_config3_shape_bf16(n):
    """4 Matern blocks, 2 observed, rhat ~ 1/|k|, rho 0.6, N=20, BF16 storage (reduced grid)."""
    _check_problem(fields.make_config3(ny=n, nx=n, N=20, storage="bf16"), TOL16)


def test_config3_shape_f32():
    _check_problem(fields.make_config3(ny=128, nx=128, N=20, storage="f32"), TOL32)


@pytest.mark.parametrize(
    "ny,nx,N",
    [(16, 16, 3), (32, 64, 5), (48, 96, 7), (96, 96, 5), (64, 192, 4), (192, 128, 6), (24, 48, 2),
     (384, 384, 3), (768, 256, 3), (32, 4096, 3), (4096, 32, 3), (1024, 1024, 3), (3072, 48, 2), (16, 6144, 2),
     (16, 8192, 2)],
)
def test_sizes_single_block(ny, nx, N):
    S = fields.se_spectrum(ny, nx, 3.0, 1.0)
    rh = np.full((1, ny, nx // 2 + 1), 0.1)
    p = fields.make_problem(ny, nx, N, [S], [1], rh, seed=1000 + ny + nx, storage="f32")
    _check_problem(p, TOL32)


@pytest.mark.parametrize(
    "observed",
    [[1, 1, 1], [0, 1, 1], [1, 0, 0, 0, 0, 0], [1, 1, 1, 0], [1, 1, 1, 1, 0, 0]],
)
def test_block_masks(observed):
    M = len(observed)
    ny, nx = 32, 48
    spectra = [fields.matern32_spectrum(ny, nx, 2.0 + 3 * b, 1.0) for b in range(M)]
    n_obs = int(np.sum(observed))
    kk = fields.radial_wavenumber_half(ny, nx)
    rh = np.stack([(0.05 + 0.05 * i) / np.maximum(kk, 1.0) for i in range(n_obs)])
    p = fields.make_problem(ny, nx, 6, spectra, observed, rh, seed=77 + M, storage="f32", rho=0.5)
    _check_problem(p, TOL32)


def test_supplied_spectrum():
    p = fields.make_config1(seed=5, ny=64, nx=96)
    S = p.spectra[0]
    tables = enkf.spectrum_to_tables(enkf.Spectrum({0: S}, {}), [1])
    ua, st = _gu().gpu_analyze(p, spectrum=tables)
    assert st == 0
    assert _gu().rel_l2(ua, _oracle(p, spectrum=tables)) <= TOL32


def test_rhat_limits_gpu():
    gu = _gu()
    p = fields.make_config2(ny=64, nx=64)
    p.rhat[:] = 1e30
    ua, _ = gu.gpu_analyze(p)
    assert np.max(np.abs(ua - p.ensemble)) <= 1e-6 * np.max(np.abs(p.ensemble))
    p = fields.make_config1(ny=64, nx=64)
    p.rhat[:] = 0.0
    p.perturbations[:] = 0.0
    ua, _ = gu.gpu_analyze(p)
    for k in range(p.N):
        assert gu.rel_l2(ua[0, k], p.data[0]) <= TOL32


def test_vanishing_denominator_keeps_forecast():
    """rhat = 0 and an observed block whose members are all equal: chat^(oo) = 0 and
    chat^(jo) = 0 at every wavenumber, so every denominator chat^(oo) + rhat is 0 and
    the gain is 0 (no information): the forecast is returned unchanged, as the oracle
    does.  Exercises the zero-denominator branch of the gain."""
    p = fields.make_config2(ny=64, nx=64)
    o = int(np.flatnonzero(p.observed)[0])
    p.ensemble[o, :] = p.ensemble[o, 0]
    p.rhat[:] = 0.0
    ua, st = _gu().gpu_analyze(p)
    assert st == 0
    ref = _oracle(p)
    np.testing.assert_array_equal(ref, p.ensemble.astype(np.float64))
    np.testing.assert_array_equal(ua, p.ensemble.astype(np.float64))


def test_golden_shift_closed_form_16():
    """The two-block worked example of tests/golden/two_block_shift.json on a 16 x 16 grid.

    Same construction: block 1 anomalies +-d_00, block 2 anomalies +-2 d_01,
    rhat = chat11 = 2/G so that gain11 = 1/2 and gain21 is a shift by +1 in x."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "two_block_shift.json")))
    ny = nx = 16
    G = ny * nx
    ens = np.zeros((2, 2, ny, nx))
    ens[0] = 1.0
    ens[0, 0, 0, 0] += 1
    ens[0, 1, 0, 0] -= 1
    ens[1, 0, 0, 1] = 2
    ens[1, 1, 0, 1] = -2
    d = np.full((1, ny, nx), 3.0)
    e = np.zeros((2, 1, ny, nx))
    e[0, 0, 1, 2] = 0.5
    p = fields.Problem(ny=ny, nx=nx, M=2, N=2, observed=np.array(g["observed"], np.uint8), storage="f32",
                       ensemble=ens.astype(np.float32), data=d.astype(np.float32),
                       perturbations=e.astype(np.float32), rhat=np.full((1, ny, nx // 2 + 1), 2.0 / G),
                       truth=np.zeros((2, ny, nx)))
    ua, _ = _gu().gpu_analyze(p)
    ref = np.empty_like(ens)
    for k in range(2):
        w = d[0] + e[k, 0] - ens[0, k]
        ref[0, k] = ens[0, k] + 0.5 * w
        ref[1, k] = ens[1, k] + np.roll(w, 1, axis=1)
    np.testing.assert_allclose(ua, ref, atol=1e-5)


def test_nonfinite_reported():
    from paper_1001_1588_gb300 import abi
    p = fields.make_config1(ny=32, nx=32)
    p.ensemble[0, 2, 5, 7] = np.nan
    _, st = _gu().gpu_analyze(p)
    assert st == abi.FFTENKF_ENONFINITE


def test_deterministic_bitwise():
    p = fields.make_config3(ny=64, nx=64, N=8, storage="bf16")
    a, _ = _gu().gpu_analyze(p)
    b, _ = _gu().gpu_analyze(p)
    assert np.array_equal(a, b)


def test_argument_errors():
    from paper_1001_1588_gb300 import abi, torch_api
    with pytest.raises(abi.FftEnkfError) as ei:
        torch_api.Plan(64, 64, 1, 1, torch.float32, [1])
    assert ei.value.status == abi.FFTENKF_EUNSUPPORTED
    plan = torch_api.Plan(64, 64, 1, 3, torch.float32, [1])
    ens = torch.zeros(1, 3, 64, 64, device="cuda")
    d = torch.zeros(1, 64, 64, device="cuda")
    r = torch.zeros(1, 64, 33, device="cuda", dtype=torch.float64)
    with pytest.raises(abi.FftEnkfError) as ei:
        abi.fftenkf_analyze(plan.handle, ens, d, None, r, None, plan.workspace(), 0)
    assert ei.value.status == abi.FFTENKF_EINVAL
    with pytest.raises(abi.FftEnkfError) as ei:
        abi.fftenkf_analyze(plan.handle, ens.data_ptr() + 4, d, ens, r, None, plan.workspace(), 0)
    assert ei.value.status == abi.FFTENKF_EINVAL
    with pytest.raises(abi.FftEnkfError) as ei:
        abi.fftenkf_analyze(plan.handle, ens, d, ens, r, None, plan.workspace().data_ptr() + 16, 0)
    assert ei.value.status == abi.FFTENKF_EINVAL
    plan.close()


@pytest.mark.parametrize("ny,nx", [(64, 64), (96, 192), (512, 256), (48, 4096), (4096, 64)])
def test_narrow_schedule(ny, nx):
    """The alternative (radix-8) line-FFT schedule computes the same analysis."""
    from paper_1001_1588_gb300 import abi
    gu = _gu()
    spectra = [fields.matern32_spectrum(ny, nx, 3.0 + 5 * b, 1.0) for b in range(3)]
    rh = np.full((2, ny, nx // 2 + 1), 0.1)
    p = fields.make_problem(ny, nx, 4, spectra, [1, 0, 1], rh, seed=9 + ny, storage="f32", rho=0.5)
    plan = gu.plan_for(p)
    abi.fftenkf_set_schedule(plan.handle, [1] * abi.fftenkf_pass_count())
    assert abi.fftenkf_get_schedule(plan.handle)[2] == 1
    ens, data, pert, rhat = gu.to_device(p)
    spec = plan.estimate_spectrum(ens).cpu().numpy()
    plan.analyze(ens, data, pert, rhat)
    assert plan.device_status() == 0
    ua = ens.cpu().numpy().astype(np.float64)
    plan.close()
    assert gu.rel_l2(ua, _oracle(p)) <= TOL32
    assert gu.rel_l2(spec, _tables(p)) <= TOL32
