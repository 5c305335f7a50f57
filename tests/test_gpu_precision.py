"""GPU parity where the precision rules of the analysis matter, and the bounded-wait error path.

* A large common mean (300 with unit anomalies), FP32 and BF16 storage: the ensemble mean of
  eq. (dii) would be subtracted from values 300 times the anomalies; the library never forms it,
  but transforms the differences from the first member (exact for close values) and subtracts
  the products of their transformed sum, and forms the innovation d + e - u as (d - u) + e
  (d - u exact for close values).  Gates: the analysis and the spectrum tables at the
  storage tolerance (1e-5 FP32, 5e-3 BF16, relative L2 over the whole array); for FP32 the
  increment u^a - u at 1e-4 (the forecast, 300 times larger, would hide an increment error in the
  analysis).  With BF16 storage the output itself is rounded at 300 (spacing 2), so only the
  analysis and the tables are gated there.
* The bounded waits: with the test setting that makes every CTA's first bulk-copy wait of the
  forward row pass give up at once, a call reports FFTENKF_ETIMEOUT; with it off again, the next
  call is OK and matches the oracle.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import enkf  # noqa: E402
from synth import fields  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_1588_gb300 import abi
    abi.lib()


def _large_mean_problem(ny, nx, N, storage, seed):
    M = 4
    spectra = [fields.matern32_spectrum(ny, nx, 3.0 + 5.0 * b, 1.0) for b in range(M)]
    kk = fields.radial_wavenumber_half(ny, nx)
    rh = np.stack([0.1 / np.maximum(kk, 1.0), 0.05 / np.maximum(kk, 1.0)])
    return fields.make_problem(ny, nx, N, spectra, [1, 1, 0, 0], rh, seed=seed, storage=storage, rho=0.6,
                               mean=[300.0, -250.0, 280.0, 310.0])


@pytest.mark.parametrize("storage,ny,nx", [("f32", 256, 256), ("bf16", 256, 256), ("f32", 1024, 64)])
def test_large_common_mean(storage, ny, nx):
    from tests import gpu_util as gu
    p = _large_mean_problem(ny, nx, 8, storage, seed=300 + ny)
    tol = 1e-5 if storage == "f32" else 5e-3
    spec, st = gu.gpu_spectrum(p)
    assert st == 0
    tab = enkf.spectrum_to_tables(enkf.estimate_spectrum(p.ensemble, p.observed), p.observed)
    assert gu.rel_l2(spec, tab) <= tol
    ua, st = gu.gpu_analyze(p)
    assert st == 0
    ref = enkf.analyze(p.ensemble, p.data, p.perturbations, p.rhat, p.observed)
    assert gu.rel_l2(ua, ref) <= tol
    if storage == "f32":
        assert gu.rel_l2(ua - p.ensemble, ref - p.ensemble) <= 1e-4


def test_bounded_wait_expiry_then_recovery():
    from paper_1001_1588_gb300 import abi
    from tests import gpu_util as gu
    p = fields.make_config3(ny=256, nx=256, N=6, storage="f32")
    plan = gu.plan_for(p)
    ens, data, pert, rhat = gu.to_device(p)
    abi.fftenkf_set_expire_first_wait(plan.handle, 1)
    plan.analyze(ens, data, pert, rhat)
    assert plan.device_status() == abi.FFTENKF_ETIMEOUT
    plan.estimate_spectrum(ens)
    assert plan.device_status() == abi.FFTENKF_ETIMEOUT
    abi.fftenkf_set_expire_first_wait(plan.handle, 0)
    ens, data, pert, rhat = gu.to_device(p)
    plan.analyze(ens, data, pert, rhat)
    assert plan.device_status() == abi.FFTENKF_OK
    ua = ens.float().cpu().numpy().astype(np.float64)
    plan.close()
    ref = enkf.analyze(p.ensemble, p.data, p.perturbations, p.rhat, p.observed)
    assert gu.rel_l2(ua, ref) <= 1e-5


@pytest.mark.parametrize("ny,nx", [(64, 64), (512, 64)])      # column-statistics epilogue; fused column pass
@pytest.mark.parametrize("ratio", [1e-6, 1e-9])
def test_gain_band_small_chat_over_rhat(ny, nx, ratio):
    """The gain quotient where chat/rhat is tiny, isolated: white members of standard deviation
    `ratio` (chat about ratio^2), rhat = 1e30 below |k| = ny/4 (no update there) and `ratio` above
    (chat/rhat about `ratio`), white data, no perturbations.  The whole increment then lies in the
    high-k band and is about `ratio` times the innovation (as large as the members, so the FP32
    output keeps its digits), and FFT round-off of other bands cannot hide an error of the FP32
    quotient there; the increment must match the FP64 oracle to 1e-5 (relative L2), and its low
    band must stay 0."""
    from tests import gpu_util as gu
    rng = np.random.default_rng(4242 + ny)
    N = 5
    ens = (ratio * rng.standard_normal((1, N, ny, nx))).astype(np.float32).astype(np.float64)
    data = rng.standard_normal((1, ny, nx)).astype(np.float32).astype(np.float64)
    pert = np.zeros((N, 1, ny, nx))
    kk = fields.radial_wavenumber_half(ny, nx)
    rhat = np.where(kk < ny / 4, 1e30, ratio)[None]
    p = fields.Problem(ny=ny, nx=nx, M=1, N=N, observed=np.array([1], np.uint8), storage="f32",
                       ensemble=ens.astype(np.float32), data=data.astype(np.float32),
                       perturbations=pert.astype(np.float32), rhat=rhat, truth=np.zeros((1, ny, nx)))
    ua, st = gu.gpu_analyze(p)
    assert st == 0
    ref = enkf.analyze(p.ensemble, p.data, p.perturbations, p.rhat, p.observed)
    inc, inc_ref = ua - ens, ref - ens
    assert np.abs(inc_ref).max() > 0.1 * ratio   # the band update is there and of the expected size
    assert gu.rel_l2(inc, inc_ref) <= 1e-5
    low = kk < ny / 4
    got_hat = np.fft.rfft2(inc[0, 0], norm="ortho")
    assert np.abs(got_hat[low]).max() <= 1e-6 * np.abs(got_hat).max()
