"""GPU parity of the fused column pass (statistics, gains and update per column, tables in tensor
memory) against the FP64 oracle, for both of its line-FFT schedules.

The fused pass runs for one or two observed blocks on columns of 512 to 4096 points.  Shapes
cover an even and an odd number of blocks (a block pair padded with an empty line), one and two
observed blocks, several column counts (ragged against the CTAs' column groups), FP32 and BF16
storage, and the spectrum estimate (tables written instead of gains).  Tolerances as in
test_gpu_parity: 1e-5 (FP32) / 5e-3 (BF16) relative L2 of the analysis and of every table;
the increment u^a - u is gated too, at 10x the tolerance, since the forecast dominates u^a.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import enkf  # noqa: E402
from synth import fields  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "bf16": 5e-3}
FUSED = 9   # pass index of col_fused in the schedule vector


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_1588_gb300 import abi
    abi.lib()


def _problem(ny, nx, N, observed, storage, seed):
    M = len(observed)
    spectra = [fields.matern32_spectrum(ny, nx, 3.0 + 4.0 * b, 1.0) for b in range(M)]
    n_obs = int(np.sum(observed))
    kk = fields.radial_wavenumber_half(ny, nx)
    rh = np.stack([(0.05 + 0.05 * i) / np.maximum(kk, 1.0) for i in range(n_obs)])
    return fields.make_problem(ny, nx, N, spectra, observed, rh, seed=seed, storage=storage, rho=0.6)


def _run(p, sel):
    from paper_1001_1588_gb300 import abi
    from tests import gpu_util as gu
    plan = gu.plan_for(p)
    sched = abi.fftenkf_get_schedule(plan.handle)
    sched[FUSED] = sel
    abi.fftenkf_set_schedule(plan.handle, sched)
    ens, data, pert, rhat = gu.to_device(p)
    spec = plan.estimate_spectrum(ens).cpu().numpy()
    st1 = plan.device_status()
    plan.analyze(ens, data, pert, rhat)
    st2 = plan.device_status()
    ua = ens.float().cpu().numpy().astype(np.float64)
    plan.close()
    return ua, spec, st1, st2


@pytest.mark.parametrize("sel", [0, 1])
@pytest.mark.parametrize(
    "ny,nx,N,observed,storage",
    [
        (512, 64, 6, [1, 1, 0, 0], "f32"),
        (512, 96, 5, [0, 1, 0], "f32"),          # odd block count, observed block not first
        (1024, 48, 4, [1, 0, 1, 0, 0], "f32"),   # odd block count, two observed
        (2048, 32, 3, [1, 0], "f32"),            # one observed block, one unobserved
        (4096, 32, 4, [1, 1, 0, 0], "f32"),
        (4096, 64, 5, [1, 1, 0, 0], "bf16"),
        (1024, 1024, 3, [1], "f32"),             # single block
        (256, 4096, 3, [1, 1, 0, 0], "bf16"),    # 4096-wide rows: anomaly + innovation rows in one pass
        (512, 1024, 4, [1, 0, 1, 0], "f32"),     # the same pass with FP32 members
    ],
)
def test_fused_parity(ny, nx, N, observed, storage, sel):
    from tests import gpu_util as gu
    p = _problem(ny, nx, N, observed, storage, seed=4000 + ny + nx + N)
    ua, spec, st1, st2 = _run(p, sel)
    assert st1 == 0 and st2 == 0
    ref = enkf.analyze(p.ensemble, p.data, p.perturbations, p.rhat, p.observed)
    tol = TOL[storage]
    assert gu.rel_l2(ua, ref) <= tol
    assert gu.rel_l2(ua - p.ensemble, ref - p.ensemble) <= 10 * tol
    tab = enkf.spectrum_to_tables(enkf.estimate_spectrum(p.ensemble, p.observed), p.observed)
    assert gu.rel_l2(spec, tab) <= tol


def test_fused_matches_separate_passes():
    """The fused pass and the separate statistics / update passes (selected by the narrow
    statistics schedule) compute the same analysis to FP32 rounding."""
    from paper_1001_1588_gb300 import abi
    from tests import gpu_util as gu
    p = _problem(1024, 128, 6, [1, 1, 0, 0], "f32", seed=77)
    ua_fused, _, _, _ = _run(p, 0)
    plan = gu.plan_for(p)
    sched = abi.fftenkf_get_schedule(plan.handle)
    sched[2] = 1   # col_stats narrow: the separate passes
    abi.fftenkf_set_schedule(plan.handle, sched)
    ens, data, pert, rhat = gu.to_device(p)
    plan.analyze(ens, data, pert, rhat)
    assert plan.device_status() == 0
    ua_sep = ens.float().cpu().numpy().astype(np.float64)
    plan.close()
    assert gu.rel_l2(ua_fused - p.ensemble, ua_sep - p.ensemble) <= 1e-5
