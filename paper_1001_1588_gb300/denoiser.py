"""Training and evaluation of the learned spectral-variance denoiser (GPU, library kernels).

Training pairs.  For a random stationary field model (power-law spectrum
S ~ (1 + (2 pi l |xi|)^2)^(beta/2), l log-uniform in [2, 64] cells, beta uniform
in [-5, -2], unit variance) the input is the plain method's own estimate: N = 5
members drawn on the device, eq. (dii) through fftenkf_estimate_spectrum, binned
by the library's feature kernel.  The target is the binned log spectrum that the
same estimator returns for a 500-member ensemble.  Its per-wavenumber value is
drawn from that estimator's exact distribution for Gaussian fields (unitary DFT):
chat = S X/(N-1) with X ~ Gamma(N-1, 1) at complex modes and X ~ chi^2_{N-1} at
self-conjugate ones, instead of synthesising 500 fields per pair; a test checks
this against literal 500-member ensembles.

Training uses fftenkf_mlp_gradient and fftenkf_mlp_adam (mean squared error in
log space, Adam, FP32 master weights, BF16 forward copy).  Evaluation: held-out
analyses (one block, H = I, rhat = 0.1 flat, N = 5) scored by the RMSE of the
analysis-ensemble mean against the truth, for the plain estimate, the learned
spectrum and the true spectrum (the lower bound).

    python -m paper_1001_1588_gb300.denoiser --pairs 20000 --grid 1024 --epochs 20 --out weights.bin
"""

from __future__ import annotations

import argparse
import json
import math
import os
import struct
import sys
import time

import numpy as np
import torch

from . import abi, torch_api

MAGIC = b"FEKFMLP1"


# ---------------------------------------------------------------- checkpoint
def save(path, params, m=None, v=None, step=0, grid=(1024, 1024), members=5):
    """Flat binary: magic, header (param count, step, ny, nx, members, has_adam), params [, m, v] (float32)."""
    P = params.numel()
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<6q", P, step, grid[0], grid[1], members, int(m is not None)))
        f.write(params.detach().float().cpu().numpy().tobytes())
        if m is not None:
            f.write(m.detach().float().cpu().numpy().tobytes())
            f.write(v.detach().float().cpu().numpy().tobytes())


def load(path, device="cuda"):
    with open(path, "rb") as f:
        if f.read(8) != MAGIC:
            raise ValueError("not a denoiser checkpoint")
        P, step, ny, nx, members, has_adam = struct.unpack("<6q", f.read(48))
        arr = np.frombuffer(f.read(), dtype=np.float32)
    params = torch.from_numpy(arr[:P].copy()).to(device)
    m = v = None
    if has_adam:
        m = torch.from_numpy(arr[P:2 * P].copy()).to(device)
        v = torch.from_numpy(arr[2 * P:3 * P].copy()).to(device)
    return dict(params=params, m=m, v=v, step=step, grid=(ny, nx), members=members)


def init_params(seed=0, device="cuda"):
    """He-style uniform initialisation with zero biases (same rule as the oracle's)."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for i, o in ((256, 64), (64, 64), (64, 64), (64, 128)):
        lim = math.sqrt(6.0 / i)
        parts.append((torch.rand(o * i, generator=g, dtype=torch.float64) * 2 - 1) * lim)
        parts.append(torch.zeros(o, dtype=torch.float64))
    return torch.cat(parts).float().to(device)


# ---------------------------------------------------------------- field models
def _xi2_half(ny, nx, device):
    ky = torch.fft.fftfreq(ny, device=device, dtype=torch.float64)[:, None]
    kx = torch.fft.rfftfreq(nx, device=device, dtype=torch.float64)[None, :]
    return ky ** 2 + kx ** 2


def powerlaw_half(ny, nx, ell, beta, device):
    S = (1.0 + 4.0 * math.pi ** 2 * ell ** 2 * _xi2_half(ny, nx, device)) ** (beta / 2.0)
    w = torch.full((S.shape[1],), 2.0, dtype=S.dtype, device=device)
    w[0] = 1.0
    w[-1] = 1.0
    return S / ((S * w).sum() / (ny * nx))


def self_conjugate_mask(ny, nx, device):
    m = torch.zeros(ny, nx // 2 + 1, dtype=torch.bool, device=device)
    for ky in (0, ny // 2):
        for kx in (0, nx // 2):
            m[ky, kx] = True
    return m


def draw_fields(S, n, gen, ny, nx):
    sq = S.sqrt().float()
    out = torch.empty(n, ny, nx, device=S.device)
    for k in range(n):
        z = torch.randn(ny, nx, device=S.device, generator=gen)
        out[k] = torch.fft.irfft2(torch.fft.rfft2(z, norm="ortho") * sq, s=(ny, nx), norm="ortho")
    return out


def sampled_estimate(S, n_members, gen, selfc):
    """A draw of eq. (dii)'s output for an n_members ensemble of fields with spectrum S."""
    nu = n_members - 1
    a = torch.full_like(S, float(nu))
    a = torch.where(selfc, torch.full_like(S, nu / 2.0), a)
    X = torch._standard_gamma(a)          # seeded through torch.manual_seed by the caller
    X = torch.where(selfc, 2.0 * X, X)
    return S * X / nu


# ---------------------------------------------------------------- pairs
class Pairs:
    def __init__(self, ny, nx, members=5, target_members=500, device="cuda"):
        self.ny, self.nx, self.N, self.Nt = ny, nx, members, target_members
        self.device = device
        self.plan = torch_api.Plan(ny, nx, 1, members, torch.float32, [1])
        self.den = abi.fftenkf_denoiser_create(ny, nx, members)
        self.selfc = self_conjugate_mask(ny, nx, device)

    def close(self):
        self.plan.close()
        abi.fftenkf_denoiser_destroy(self.den)

    def features(self, chat, batch):
        feat = torch.empty(batch, 256, device=self.device)
        mean = torch.empty(batch, device=self.device)
        abi.fftenkf_denoiser_features(self.den, chat, batch, feat, mean,
                                      int(torch.cuda.current_stream().cuda_stream))
        return feat, mean

    def generate(self, n, seed, chunk=64):
        rng = np.random.default_rng(seed)
        gen = torch.Generator(device=self.device)
        gen.manual_seed(seed)
        torch.manual_seed(seed)
        K1 = self.ny * (self.nx // 2 + 1)
        X = torch.empty(n, 256, device=self.device)
        Y = torch.empty(n, 128, device=self.device)
        for s0 in range(0, n, chunk):
            b = min(chunk, n - s0)
            chat_in = torch.empty(b, K1, dtype=torch.float64, device=self.device)
            chat_t = torch.empty(b, K1, dtype=torch.float64, device=self.device)
            for i in range(b):
                ell = float(np.exp(rng.uniform(np.log(2.0), np.log(64.0))))
                beta = float(rng.uniform(-5.0, -2.0))
                S = powerlaw_half(self.ny, self.nx, ell, beta, self.device)
                ens = draw_fields(S, self.N, gen, self.ny, self.nx)[None].contiguous()
                self.plan.estimate_spectrum(ens, chat_in[i])
                chat_t[i] = sampled_estimate(S, self.Nt, gen, self.selfc).reshape(-1)
            fi, mi = self.features(chat_in, b)
            ft, mt = self.features(chat_t, b)
            X[s0:s0 + b] = fi
            Y[s0:s0 + b] = ft[:, :128] + mt[:, None] - mi[:, None]
        return X, Y


# ---------------------------------------------------------------- training
def train(X, Y, epochs=20, batch=256, lr=1e-3, seed=0, params=None, m=None, v=None, step=0, log=None):
    dev = X.device
    P = abi.fftenkf_mlp_param_count()
    params = init_params(seed, dev) if params is None else params
    m = torch.zeros(P, device=dev) if m is None else m
    v = torch.zeros(P, device=dev) if v is None else v
    grads = torch.empty(P, device=dev)
    loss = torch.zeros(1, device=dev)
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    stream = int(torch.cuda.current_stream().cuda_stream)
    history = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(dev)
        tot = 0.0
        nb = 0
        for s0 in range(0, n - batch + 1, batch):
            idx = perm[s0:s0 + batch]
            xb = X[idx].contiguous()
            yb = Y[idx].contiguous()
            abi.fftenkf_mlp_gradient(params, xb, yb, batch, grads, loss, stream)
            step += 1
            abi.fftenkf_mlp_adam(params, m, v, grads, step, lr, stream)
            tot += float(loss.item()) if (s0 // batch) % 16 == 0 else 0.0
            nb += 1 if (s0 // batch) % 16 == 0 else 0
        history.append(tot / max(nb, 1))
        if log:
            log("epoch %d loss %.4f" % (ep, history[-1]))
    return params, m, v, step, history


def predict_loss(params, X, Y):
    out = torch.empty(X.shape[0], 128, device=X.device)
    abi.fftenkf_mlp_forward(params, X.contiguous(), X.shape[0], out, int(torch.cuda.current_stream().cuda_stream))
    return float(((out - Y) ** 2).mean().item())


# ---------------------------------------------------------------- evaluation
def evaluate(params, ny, nx, n_draws=64, members=5, r=0.1, seed=777, device="cuda"):
    """Held-out analysis RMSE of the ensemble mean for plain, learned and true spectra."""
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    plan = torch_api.Plan(ny, nx, 1, members, torch.float32, [1])
    den = abi.fftenkf_denoiser_create(ny, nx, members)
    stream = int(torch.cuda.current_stream().cuda_stream)
    K1 = ny * (nx // 2 + 1)
    rhat = torch.full((1, ny, nx // 2 + 1), r, dtype=torch.float64, device=device)
    res = {"plain": [], "learned": [], "true_spectrum": [], "fallbacks": 0}
    learned = torch.empty(K1, dtype=torch.float64, device=device)
    for _ in range(n_draws):
        ell = float(np.exp(rng.uniform(np.log(2.0), np.log(64.0))))
        beta = float(rng.uniform(-5.0, -2.0))
        S = powerlaw_half(ny, nx, ell, beta, device)
        truth = draw_fields(S, 1, gen, ny, nx)[0]
        ens0 = draw_fields(S, members, gen, ny, nx)[None].contiguous()
        data = (truth + math.sqrt(r) * torch.randn(ny, nx, device=device, generator=gen))[None].contiguous()
        pert = (math.sqrt(r) * torch.randn(members, 1, ny, nx, device=device, generator=gen)).contiguous()
        chat = plan.estimate_spectrum(ens0)
        res["fallbacks"] += abi.fftenkf_denoise_spectrum(den, params, chat, learned, members, stream)
        for key, spec in (("plain", None), ("learned", learned), ("true_spectrum", S.reshape(-1).contiguous())):
            ens = ens0.clone()
            plan.analyze(ens, data, pert, rhat, spec)
            mean = ens[0].mean(dim=0)
            res[key].append(float(torch.sqrt(((mean - truth) ** 2).mean()).item()))
    plan.close()
    abi.fftenkf_denoiser_destroy(den)
    out = {k: (float(np.mean(v)) if isinstance(v, list) else v) for k, v in res.items()}
    d = np.array(res["learned"]) - np.array(res["plain"])
    out["learned_minus_plain_mean"] = float(d.mean())
    out["learned_minus_plain_ci95"] = float(1.96 * d.std(ddof=1) / np.sqrt(len(d)))
    out["learned_better_fraction"] = float(np.mean(d < 0))
    out["draws"] = n_draws
    return out, res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--grid", type=int, default=1024)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval", type=int, default=64)
    ap.add_argument("--out", default="")
    ap.add_argument("--resume", default="")
    a = ap.parse_args(argv)
    torch.cuda.set_device(0)
    t0 = time.time()
    pairs = Pairs(a.grid, a.grid)
    X, Y = pairs.generate(a.pairs, seed=20260005)
    Xv, Yv = pairs.generate(max(256, a.pairs // 20), seed=20260105)
    pairs.close()
    t_gen = time.time() - t0
    ck = load(a.resume) if a.resume else {}
    t1 = time.time()
    params, m, v, step, hist = train(X, Y, a.epochs, a.batch, a.lr, params=ck.get("params"), m=ck.get("m"),
                                     v=ck.get("v"), step=ck.get("step", 0), log=lambda s: print(s, file=sys.stderr))
    torch.cuda.synchronize()
    t_train = time.time() - t1
    if a.out:
        save(a.out, params, m, v, step, (a.grid, a.grid), 5)
    ev, _ = evaluate(params, a.grid, a.grid, n_draws=a.eval)
    print(json.dumps({"pairs": a.pairs, "grid": a.grid, "epochs": a.epochs, "train_loss": hist[-1],
                      "val_loss": predict_loss(params, Xv, Yv),
                      "val_loss_plain_bins": float(((Xv[:, :128] - Yv) ** 2).mean().item()),
                      "seconds_pairs": t_gen, "seconds_train": t_train, "steps": step, "eval": ev}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
