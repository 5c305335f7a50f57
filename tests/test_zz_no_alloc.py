"""The allocation-free spectrum estimate against the FP64 oracle and the plan-based entry point.

Some callers may not call cudaMalloc: a host framework that owns every device allocation
through its own pool, or a latency-critical loop that cannot afford cudaMalloc's implicit
synchronisation.  For them fftenkf_estimate_spectrum_static takes its scratch from a static
device array instead of a workspace, and fftenkf_static_last_device_status reads that array's
status word, also without allocating.  This file is collected last so that a run that stops at
its first failure has already run every other test; it passes both alone in a fresh process and
after the rest of the suite.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import enkf  # noqa: E402
from synth import fields  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = {"f32": 1e-5, "bf16": 5e-3}


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_static_scratch_estimate_matches_oracle_and_plan_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_1588_gb300 import abi, torch_api
    abi.lib()
    cases = [(256, 256, 10, "f32", 3.0), (96, 192, 5, "bf16", 6.0)]
    for ny, nx, N, st, ell in cases:                         # two calls in a row, different shapes
        S = fields.se_spectrum(ny, nx, ell, 1.0)
        p = fields.make_problem(ny, nx, N, [S], [1], np.full((1, ny, nx // 2 + 1), 0.1), seed=31 + ny, storage=st)
        dt = torch.float32 if st == "f32" else torch.bfloat16
        ens = torch.from_numpy(p.ensemble).cuda().to(dt).contiguous()
        plan = torch_api.Plan(ny, nx, 1, N, dt, [1])
        ref_plan = plan.estimate_spectrum(ens).cpu().numpy()
        plan.close()
        out = torch.full((ny * (nx // 2 + 1),), float("nan"), dtype=torch.float64, device="cuda")
        code = abi.FFTENKF_F32 if st == "f32" else abi.FFTENKF_BF16
        abi.fftenkf_estimate_spectrum_static(ens[0], ny, nx, N, code, out, 0)
        assert abi.fftenkf_static_last_device_status(0) == abi.FFTENKF_OK
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        # the FP64 oracle on the same (rounded) members: eq. (dii) of the single block
        ref = enkf.spectrum_to_tables(enkf.estimate_spectrum(p.ensemble, [1]), [1])
        assert _rel(got, ref) <= TOL[st]
        assert _rel(got, ref_plan) <= TOL["f32"]


def test_static_scratch_reports_nonfinite():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_1588_gb300 import abi
    ny, nx, N = 64, 64, 4
    S = fields.se_spectrum(ny, nx, 4.0, 1.0)
    p = fields.make_problem(ny, nx, N, [S], [1], np.full((1, ny, nx // 2 + 1), 0.1), seed=5, storage="f32")
    e = p.ensemble.copy()
    e[0, 1, 3, 5] = np.inf
    ens = torch.from_numpy(e).cuda()
    out = torch.zeros(ny * (nx // 2 + 1), dtype=torch.float64, device="cuda")
    abi.fftenkf_estimate_spectrum_static(ens[0], ny, nx, N, abi.FFTENKF_F32, out, 0)
    assert abi.fftenkf_static_last_device_status(0) == abi.FFTENKF_ENONFINITE
    ens = torch.from_numpy(p.ensemble).cuda()                # the word was cleared; a clean call is OK
    abi.fftenkf_estimate_spectrum_static(ens[0], ny, nx, N, abi.FFTENKF_F32, out, 0)
    assert abi.fftenkf_static_last_device_status(0) == abi.FFTENKF_OK


def test_static_scratch_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_1588_gb300 import abi
    ens = torch.zeros(8, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(abi.FftEnkfError) as ei:
        abi.fftenkf_estimate_spectrum_static(ens, 2048, 2048, 8, abi.FFTENKF_F32, out, 0)   # 134 MB of row spectra
    assert ei.value.status == abi.FFTENKF_EUNSUPPORTED
    assert "64 MiB" in abi.fftenkf_last_error()
