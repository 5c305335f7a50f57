"""GPU parity of the batched analyses on the benchmark's own draw: the 256 single-block analyses of
uneven sizes (sides 64..1024, square and 2:1, N 5..25) that bench.py --workload batched times,
drawn on the device by the same generator, in FP32 and in BF16 storage.

Every item is checked for finite output and a non-zero increment; a deterministic sample of items
(the cheapest of every side length, and the cheapest item of the largest side) is checked
element by element against the FP64 oracle on the same (rounded) inputs: 1e-5 relative L2 (FP32),
5e-3 (BF16; the output is rounded to BF16).  The increment u^a - u is gated at 10x those.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import enkf  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_1588_gb300 import abi as a
    a.lib()
    return a


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _sample(items):
    """The cheapest item (ny nx N) of every side length max(ny, nx)."""
    best = {}
    for i, it in enumerate(items):
        side = max(it.ny, it.nx)
        cost = it.ny * it.nx * it.N
        if side not in best or cost < best[side][0]:
            best[side] = (cost, i)
    return sorted(i for _, i in best.values())


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_batched_benchmark_draw(abi, storage):
    from synth.fields_torch import make_batched_torch
    dt = torch.float32 if storage == "f32" else torch.bfloat16
    code = abi.FFTENKF_F32 if storage == "f32" else abi.FFTENKF_BF16
    tol = 1e-5 if storage == "f32" else 5e-3
    items = make_batched_torch(device="cuda", count=256, storage=dt)
    sample = _sample(items)
    assert len(sample) >= 8
    host = {i: (items[i].ensemble.double().cpu().numpy()[None], items[i].data.double().cpu().numpy()[None],
                items[i].perturbations.double().cpu().numpy()[:, None], items[i].rhat.cpu().numpy()[None])
            for i in sample}
    before = [it.ensemble.clone() for it in items]
    b = abi.fftenkf_plan_batched([(it.ny, it.nx, it.N) for it in items], code)
    ws = torch.empty(abi.fftenkf_batch_workspace_size(b), dtype=torch.uint8, device="cuda")
    abi.fftenkf_analyze_batched(b, [it.ensemble for it in items], [it.data for it in items],
                                [it.perturbations for it in items], [it.rhat for it in items], ws, 0)
    assert abi.fftenkf_batch_last_device_status(b, 0) == 0
    abi.fftenkf_batch_destroy(b)
    for it, u0 in zip(items, before):
        assert bool(torch.isfinite(it.ensemble.float()).all())
        assert float((it.ensemble.float() - u0.float()).abs().max()) > 0.0
    for i in sample:
        ens, data, pert, rhat = host[i]
        ref = enkf.analyze(ens, data, pert, rhat, np.array([1], np.uint8))[0]
        got = items[i].ensemble.double().cpu().numpy()
        assert _rel(got, ref) <= tol, (i, items[i].ny, items[i].nx, items[i].N)
        assert _rel(got - ens[0], ref - ens[0]) <= 10 * tol, (i, items[i].ny, items[i].nx, items[i].N)
