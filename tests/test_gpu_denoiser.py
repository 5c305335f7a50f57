"""GPU parity of the learned-spectrum kernels against the FP64 oracle (oracle/mlp.py),
the estimator-distribution shortcut of the training targets, and the benefit of the
trained network on held-out analyses."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import enkf, mlp  # noqa: E402
from synth import fields  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_1588_gb300 import abi as a
    a.lib()
    return a


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _bf16(theta):
    """The network the kernels evaluate: weights rounded to BF16, biases kept in FP32."""
    t = np.asarray(theta, np.float32).astype(np.float64).copy()
    pos = 0
    for i, o in mlp.LAYERS:
        w = t[pos:pos + i * o]
        t[pos:pos + i * o] = torch.from_numpy(w.astype(np.float32)).to(torch.bfloat16).double().numpy()
        pos += i * o + o
    return t


def _theta(seed=1):
    rng = np.random.default_rng(seed)
    return (mlp.init_params(seed) + 0.05 * rng.standard_normal(mlp.param_count())).astype(np.float32)


def test_param_count(abi):
    assert abi.fftenkf_mlp_param_count() == mlp.param_count() == 33088


def test_features_match_oracle(abi):
    ny, nx = 96, 128
    d = abi.fftenkf_denoiser_create(ny, nx, 5)
    p = fields.make_config1(seed=3, ny=ny, nx=nx)
    tabs = [enkf.spectrum_to_tables(enkf.estimate_spectrum(p.ensemble, [1]), [1])]
    tabs.append(np.exp(np.random.default_rng(2).standard_normal(tabs[0].size)) * 1e-20)
    chat = torch.from_numpy(np.stack(tabs)).cuda()
    feat = torch.empty(2, 256, device="cuda")
    mean = torch.empty(2, device="cuda")
    abi.fftenkf_denoiser_features(d, chat, 2, feat, mean, 0)
    for i in range(2):
        ref, mu = mlp.features(mlp.bin_log(tabs[i], ny, nx), ny, nx)
        assert _rel(feat[i].cpu().numpy(), ref) <= 1e-5
        assert abs(float(mean[i]) - mu) <= 1e-5 * abs(mu) + 1e-6
    abi.fftenkf_denoiser_destroy(d)


def test_forward_and_gradient_match_oracle(abi):
    theta = _theta(4)
    rng = np.random.default_rng(5)
    B = 37                                            # spans several CTAs and a ragged last one
    X = rng.standard_normal((B, 256)).astype(np.float32)
    Y = rng.standard_normal((B, 128)).astype(np.float32)
    tb = _bf16(theta)
    ref_out, _ = mlp.forward(tb, X)
    ref_g = mlp.backward(tb, X.astype(np.float64), Y.astype(np.float64))
    P = mlp.param_count()
    pt = torch.from_numpy(theta).cuda()
    Xt, Yt = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    out = torch.empty(B, 128, device="cuda")
    abi.fftenkf_mlp_forward(pt, Xt, B, out, 0)
    assert _rel(out.cpu().numpy(), ref_out) <= 1e-4
    g = torch.empty(P, device="cuda")
    loss = torch.empty(1, device="cuda")
    abi.fftenkf_mlp_gradient(pt, Xt, Yt, B, g, loss, 0)
    assert _rel(g.cpu().numpy(), ref_g) <= 1e-3
    assert abs(float(loss) - mlp.loss(ref_out, Y)) <= 1e-4 * mlp.loss(ref_out, Y)


def test_adam_matches_oracle(abi):
    P = mlp.param_count()
    rng = np.random.default_rng(6)
    th, m, v, g = (rng.standard_normal(P).astype(np.float32) for _ in range(4))
    v = np.abs(v)
    ref = mlp.adam(th.astype(np.float64), m.astype(np.float64), v.astype(np.float64), g.astype(np.float64), 3, lr=2e-3)
    T = [torch.from_numpy(a.copy()).cuda() for a in (th, m, v, g)]
    abi.fftenkf_mlp_adam(T[0], T[1], T[2], T[3], 3, 2e-3, 0)
    for got, want in zip(T[:3], ref):
        assert _rel(got.cpu().numpy(), want) <= 1e-6


def test_denoise_spectrum_end_to_end_and_fallback(abi):
    ny = nx = 128
    theta = _theta(7)
    p = fields.make_config1(seed=8, ny=ny, nx=nx)
    tab = enkf.spectrum_to_tables(enkf.estimate_spectrum(p.ensemble, [1]), [1])
    feats, mu = mlp.features(mlp.bin_log(tab, ny, nx), ny, nx)
    out, _ = mlp.forward(_bf16(theta), feats[None])
    ref = mlp.unbin(out[0] + mu, ny, nx).ravel()
    d = abi.fftenkf_denoiser_create(ny, nx, 5)
    cin = torch.from_numpy(tab).cuda()
    cout = torch.empty_like(cin)
    pt = torch.from_numpy(theta).cuda()
    assert abi.fftenkf_denoise_spectrum(d, pt, cin, cout, 5, 0) == 0
    assert _rel(cout.cpu().numpy(), ref) <= 1e-4
    assert abi.fftenkf_denoise_spectrum(d, pt, cin, cout, 7, 0) == 1     # other ensemble size: plain estimate
    assert np.array_equal(cout.cpu().numpy(), tab)
    bad = torch.full_like(pt, float("nan"))
    assert abi.fftenkf_denoise_spectrum(d, bad, cin, cout, 5, 0) == 1    # non-finite network output
    assert np.array_equal(cout.cpu().numpy(), tab)
    abi.fftenkf_denoiser_destroy(d)


def test_sampled_target_matches_literal_large_ensemble(abi):
    """The chi-square draw of the 500-member estimate bins like literal 500-member ensembles."""
    from paper_1001_1588_gb300 import denoiser as dn
    ny = nx = 64
    pr = dn.Pairs(ny, nx, members=5)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    torch.manual_seed(11)
    from paper_1001_1588_gb300 import torch_api
    big = torch_api.Plan(ny, nx, 1, 500, torch.float32, [1])
    for ell, beta in ((4.0, -3.0), (20.0, -4.5)):
        S = dn.powerlaw_half(ny, nx, ell, beta, "cuda")
        ens = dn.draw_fields(S, 500, gen, ny, nx)[None].contiguous()
        lit = big.estimate_spectrum(ens)
        smp = dn.sampled_estimate(S, 500, gen, pr.selfc).reshape(-1).contiguous()
        f1, m1 = pr.features(lit[None].contiguous(), 1)
        f2, m2 = pr.features(smp[None].contiguous(), 1)
        b1 = (f1[0, :128] + m1[0]).cpu().numpy()
        b2 = (f2[0, :128] + m2[0]).cpu().numpy()
        assert np.max(np.abs(b1 - b2)) < 0.25
        assert abs(float(b1.mean() - b2.mean())) < 0.03
    big.close()
    pr.close()


def test_trained_network_improves_heldout_rmse(abi):
    from paper_1001_1588_gb300 import denoiser as dn
    ny = nx = 256
    pr = dn.Pairs(ny, nx, members=5)
    X, Y = pr.generate(2560, seed=1)
    pr.close()
    params, m, v, step, hist = dn.train(X, Y, epochs=12, batch=128, lr=2e-3, seed=0)
    assert hist[-1] < hist[0]
    ev, _ = dn.evaluate(params, ny, nx, n_draws=24, seed=99)
    assert ev["fallbacks"] == 0
    assert ev["true_spectrum"] <= ev["plain"]
    assert ev["learned"] < ev["plain"], ev
