"""Parity at the benchmark's full size and launch configuration: 4 blocks 4096 x 4096, N=20,
BF16 storage, 2 observed (the workload bench.py times, drawn by the same device generator).

The oracle cannot transform 200 full-size fields in a test, so it computes sampled
outputs one by one: unitary DFT coefficients at chosen wavenumbers, each an O(G)
contraction per field (oracle.dft.coefficients).
  * chat^(oo)(k), chat^(jo)(k) at the sampled k from the coefficients of the members
    (eq. dii, eq. cov-multi-spectral; the mean is removed from the coefficients, which is
    the same as removing it from the fields by linearity);
  * the analysis increment's coefficient F(u^a - u)^(j)_k(k) against
    sum_o G^(jo)(k) F(d_o + e_{k,o} - u_k^(o))(k) with the oracle's gains at k
    (eq. spectral-multi-enkf).
The inputs are the exact BF16 values the GPU used; the GPU result is rounded to BF16,
hence the BF16 tolerance on the increment.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dft  # noqa: E402

pytestmark = pytest.mark.gpu

KS = [(0, 0), (0, 1), (1, 0), (1, 1), (2, 3), (4095, 2), (7, 7), (5, 40), (4088, 17), (33, 64), (100, 5), (2048, 0),
      (0, 2048), (3, 2048), (1500, 1999)]


def _coef(t, ks):
    """Unitary DFT coefficients of a device field (any dtype) at ks, in FP64."""
    return dft.coefficients(t.float().cpu().numpy().astype(np.float64), ks)


def test_full_size_sampled_parity():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_1588_gb300 import torch_api
    from synth.fields_torch import make_config3_torch
    ny = nx = 4096
    N, M = 20, 4
    p = make_config3_torch(device="cuda", ny=ny, nx=nx, N=N)
    obs = p.obs
    un = [j for j in range(M) if j not in obs]
    plan = torch_api.Plan(ny, nx, M, N, torch.bfloat16, p.observed)
    spec = plan.estimate_spectrum(p.ensemble).cpu().numpy()
    u0 = p.ensemble.clone()
    plan.analyze(p.ensemble, p.data, p.perturbations, p.rhat)
    assert plan.device_status() == 0
    L1 = nx // 2 + 1
    K = ny * L1
    # oracle: sampled coefficients of every member of every block
    C = np.empty((M, N, len(KS)), dtype=np.complex128)
    for j in range(M):
        for k in range(N):
            C[j, k] = _coef(u0[j, k], KS)
    A = C - C.mean(axis=1, keepdims=True)
    auto = {o: np.sum(np.abs(A[o]) ** 2, axis=0) / (N - 1) for o in obs}
    cross = {(j, o): np.sum(A[j] * np.conj(A[o]), axis=0) / (N - 1) for o in obs for j in un}
    idx = [ky * L1 + kx for ky, kx in KS]
    got, ref = [], []
    for i, o in enumerate(obs):
        got.append(spec[i * K + np.array(idx)])
        ref.append(auto[o])
    for q, (j, o) in enumerate([(j, o) for o in obs for j in un]):
        base = len(obs) * K + q * 2 * K
        got.append(spec[base + 2 * np.array(idx)] + 1j * spec[base + 2 * np.array(idx) + 1])
        ref.append(cross[(j, o)])
    got, ref = np.concatenate(got), np.concatenate(ref)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4
    # oracle gains at the sampled k and the increment's coefficients
    rhat = p.rhat.cpu().numpy()
    r = {o: np.array([rhat[i, ky, kx] for ky, kx in KS]) for i, o in enumerate(obs)}
    D = {o: _coef(p.data[i], KS) for i, o in enumerate(obs)}
    inc_got, inc_ref = [], []
    for k in range(N):
        w = {o: D[o] + _coef(p.perturbations[k, i], KS) - C[o, k] for i, o in enumerate(obs)}
        for j in range(M):
            if j in obs:
                want = auto[j] / (auto[j] + r[j]) * w[j]
            else:
                want = sum(cross[(j, o)] / (auto[o] + r[o]) * w[o] for o in obs)
            inc_ref.append(want)
            inc_got.append(_coef(p.ensemble[j, k], KS) - C[j, k])
    inc_got, inc_ref = np.concatenate(inc_got), np.concatenate(inc_ref)
    assert np.linalg.norm(inc_got - inc_ref) / np.linalg.norm(inc_ref) <= 5e-3
    plan.close()
