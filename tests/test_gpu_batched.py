"""GPU parity of the batched analyses (uneven sizes in one persistent launch per pass,
replayed as a CUDA graph) against the FP64 oracle, item by item (FP32 storage, 1e-5)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import enkf  # noqa: E402
from synth import fields  # noqa: E402

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def abi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_1588_gb300 import abi as a
    a.lib()
    return a


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _upload(items):
    dev = []
    for p in items:
        dev.append(dict(ens=torch.from_numpy(p.ensemble[0]).cuda().contiguous(),
                        data=torch.from_numpy(p.data[0]).cuda().contiguous(),
                        pert=torch.from_numpy(p.perturbations[:, 0]).cuda().contiguous(),
                        rhat=torch.from_numpy(p.rhat[0]).cuda().contiguous()))
    return dev


def _run(abi, b, dev, ws):
    abi.fftenkf_analyze_batched(b, [d["ens"] for d in dev], [d["data"] for d in dev], [d["pert"] for d in dev],
                                [d["rhat"] for d in dev], ws, 0)
    assert abi.fftenkf_batch_last_device_status(b, 0) == 0


def _check(items, dev):
    worst = 0.0
    for p, d in zip(items, dev):
        ref = enkf.analyze(p.ensemble, p.data, p.perturbations, p.rhat, p.observed)[0]
        worst = max(worst, _rel(d["ens"].cpu().numpy().astype(np.float64), ref))
    return worst


def test_batched_mixed_sizes(abi):
    items = fields.make_batched_items(count=14, seed=123, sides=(64, 96, 128, 192, 256, 384), n_range=(5, 12))
    shapes = {(p.ny, p.nx) for p in items}
    assert len(shapes) >= 5
    b = abi.fftenkf_plan_batched([(p.ny, p.nx, p.N) for p in items], abi.FFTENKF_F32)
    ws = torch.empty(abi.fftenkf_batch_workspace_size(b), dtype=torch.uint8, device="cuda")
    dev = _upload(items)
    _run(abi, b, dev, ws)                      # captures the graph
    assert _check(items, dev) <= TOL32
    dev = _upload(items)
    _run(abi, b, dev, ws)                      # replays it with new pointers
    assert _check(items, dev) <= TOL32
    abi.fftenkf_batch_destroy(b)


def test_batched_autotune_and_edge_sizes(abi):
    specs = [(16, 32, 2), (24, 48, 3), (1024, 1024, 3), (512, 2048, 2), (48, 32, 25), (768, 768, 4)]
    items = []
    for i, (ny, nx, N) in enumerate(specs):
        S = fields.se_spectrum(ny, nx, 2.0 + i, 1.0)
        rh = np.full((1, ny, nx // 2 + 1), 0.02 + 0.1 * i)
        items.append(fields.make_problem(ny, nx, N, [S], [1], rh, seed=500 + i, storage="f32"))
    b = abi.fftenkf_plan_batched([(p.ny, p.nx, p.N) for p in items], abi.FFTENKF_F32)
    ws = torch.empty(abi.fftenkf_batch_workspace_size(b), dtype=torch.uint8, device="cuda")
    ms = abi.fftenkf_batch_autotune(b, ws, 0)
    assert ms > 0
    bt, sc = abi.fftenkf_batch_schedule(b)
    assert all(t in (128, 256) for t in bt) and all(s in (0, 1) for s in sc)
    dev = _upload(items)
    _run(abi, b, dev, ws)
    assert _check(items, dev) <= TOL32
    abi.fftenkf_batch_destroy(b)


def test_batched_rejects_bad_items(abi):
    with pytest.raises(abi.FftEnkfError):
        abi.fftenkf_plan_batched([(64, 64, 5), (2048, 64, 5)], abi.FFTENKF_F32)
    with pytest.raises(abi.FftEnkfError):
        abi.fftenkf_plan_batched([(64, 64, 1)], abi.FFTENKF_F32)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_batched_planned_and_persistent_items_together(abi, storage):
    """Analyses of at least 512 x 256 points run on their own plans on graph branches, the
    others in the persistent passes: a mix of both (fused and separate column passes among
    the planned ones), replayed with new pointers (a new capture), every item against the
    oracle on the same rounded inputs."""
    specs = [(512, 512, 5), (64, 64, 5), (512, 1024, 3), (384, 768, 4), (96, 192, 6), (256, 256, 2)]
    items = []
    for i, (ny, nx, N) in enumerate(specs):
        S = fields.se_spectrum(ny, nx, 3.0 + 2 * i, 1.0)
        rh = np.full((1, ny, nx // 2 + 1), 0.05 + 0.05 * i)
        items.append(fields.make_problem(ny, nx, N, [S], [1], rh, seed=700 + i, storage=storage))
    dt = torch.float32 if storage == "f32" else torch.bfloat16
    code = abi.FFTENKF_F32 if storage == "f32" else abi.FFTENKF_BF16
    tol = TOL32 if storage == "f32" else 5e-3
    b = abi.fftenkf_plan_batched([(p.ny, p.nx, p.N) for p in items], code)
    ws = torch.empty(abi.fftenkf_batch_workspace_size(b), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        dev = []
        for p in items:
            dev.append(dict(ens=torch.from_numpy(p.ensemble[0]).cuda().to(dt).contiguous(),
                            data=torch.from_numpy(p.data[0].astype(np.float32)).cuda().contiguous(),
                            pert=torch.from_numpy(p.perturbations[:, 0]).cuda().to(dt).contiguous(),
                            rhat=torch.from_numpy(p.rhat[0]).cuda().contiguous()))
        _run(abi, b, dev, ws)
        for p, d in zip(items, dev):
            ref = enkf.analyze(p.ensemble, p.data, p.perturbations, p.rhat, p.observed)[0]
            got = d["ens"].float().cpu().numpy().astype(np.float64)
            assert _rel(got, ref) <= tol, (p.ny, p.nx, p.N)
            assert _rel(got - p.ensemble[0], ref - p.ensemble[0]) <= 10 * tol, (p.ny, p.nx, p.N)
    abi.fftenkf_batch_destroy(b)


def test_batched_status_reports_a_planned_item(abi):
    """A non-finite member in an analysis that runs on its own plan is reported by the batch's
    status read-out (ENONFINITE), as one in the persistent passes is."""
    specs = [(512, 512, 4), (64, 64, 4)]
    items = []
    for i, (ny, nx, N) in enumerate(specs):
        S = fields.se_spectrum(ny, nx, 4.0, 1.0)
        items.append(fields.make_problem(ny, nx, N, [S], [1], np.full((1, ny, nx // 2 + 1), 0.1), seed=900 + i,
                                         storage="f32"))
    b = abi.fftenkf_plan_batched([(p.ny, p.nx, p.N) for p in items], abi.FFTENKF_F32)
    ws = torch.empty(abi.fftenkf_batch_workspace_size(b), dtype=torch.uint8, device="cuda")
    dev = _upload(items)
    dev[0]["ens"][1, 7, 9] = float("inf")
    abi.fftenkf_analyze_batched(b, [d["ens"] for d in dev], [d["data"] for d in dev], [d["pert"] for d in dev],
                                [d["rhat"] for d in dev], ws, 0)
    assert abi.fftenkf_batch_last_device_status(b, 0) == abi.FFTENKF_ENONFINITE
    dev = _upload(items)   # finite again: OK and correct
    _run(abi, b, dev, ws)
    assert _check(items, dev) <= TOL32
    abi.fftenkf_batch_destroy(b)
