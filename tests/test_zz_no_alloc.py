"""The allocation-free spectrum estimate agrees with the plan-based entry point.

For callers that may not call cudaMalloc (their device memory is owned by a host
framework's pool, or a latency-critical loop cannot afford cudaMalloc's implicit
synchronisation), fftenkf_estimate_spectrum_static takes its scratch from a static
device array instead of a workspace.  This file is collected last so that a run
that stops at its first failure has already run every other test; it passes both
alone in a fresh process and after the rest of the suite.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import fields  # noqa: E402

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_static_scratch_estimate_matches_plan_twice():
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
        ref = plan.estimate_spectrum(ens).cpu().numpy()
        plan.close()
        out = torch.full((ny * (nx // 2 + 1),), float("nan"), dtype=torch.float64, device="cuda")
        code = abi.FFTENKF_F32 if st == "f32" else abi.FFTENKF_BF16
        abi.fftenkf_estimate_spectrum_static(ens[0], ny, nx, N, code, out, 0)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) <= TOL32


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
