#!/usr/bin/env python
"""FFT EnKF analysis benchmark: grid-pts x members per second at 4096^2, N=20.

Workload (one "step" = one complete analysis, Sec. 2.1 eq. spectral-multi-enkf):
4 blocks on a 4096 x 4096 periodic grid, 20 members, Matern-3/2 fields with
length scales 8..128 cells correlated 0.6 through a shared latent field, BF16
storage of members and perturbations, blocks 0 and 1 observed with
rhat = 0.1/max(|k|,1).  Inputs are drawn on the device once; every timed step
re-analyses the ensemble in place (2.7 GB of members, larger than L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (one full-size 4096^2 oracle DFT per step, scaled to the analysis's
200 transforms).  Under torchrun every rank analyses its own independent
problem (no collective on the data path, weak scaling).
"""

from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NY = NX = 4096
M, N, N_OBS = 4, 20, 2
OBSERVED = (1, 1, 0, 0)
METRIC = "FFT-EnKF analysis grid-pts×members/s at 4096², N=20; % of HBM roofline"
UNIT = "grid-pts*members/s"
WORKLOAD = "FFT EnKF analysis, 4 blocks 4096x4096, N=20, BF16 storage, 2 observed (Matern-3/2, rhat~1/|k|)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ny", type=int, default=NY)
    ap.add_argument("--nx", type=int, default=NX)
    ap.add_argument("--members", type=int, default=N)
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cufft", action="store_true", help="skip the torch.fft (cuFFT) reference timing")
    ap.add_argument("--no-seeded", action="store_true", help="skip the timing of the seeded (drawn-perturbation) analysis")
    ap.add_argument("--no-side", action="store_true",
                    help="sine workload: skip the side timing of the periodic extension-size analysis")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP32-storage run of the headline draw (the equal-RMSE precision comparison)")
    ap.add_argument("--workload", default="large", choices=["large", "batched", "coupled", "sine", "morph", "compare", "oracle"],
                    help="large: 4 blocks 4096^2 N=20 (default, the headline); batched: 256 mixed analyses; "
                         "coupled: 3 blocks 4096^2 N=20 with coupled observed blocks; "
                         "sine: real sine transform variant on 2049^2 nodes, 4 blocks, N=20; "
                         "compare: precision, learned-spectrum and batched forms at equal analysis RMSE; "
                         "morph: morphing FFT EnKF, 2 blocks 4096^2 N=20 FP32 (T_x, T_y, r^(1) observed); "
                         "oracle: the FP64 oracle's host times on configs 1, 2, the 1024^2 shape and a batched sample")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--fused-schedule", default="auto", choices=["auto", "0", "1"],
                    help="line-FFT schedule of the fused column pass (auto: the faster on the workload)")
    return ap.parse_args()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def hbm_peak():
    pk = peaks()
    if "hbm_gbs" in pk:
        return float(pk["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------ byte model
def pass_bytes(ny, nx, M, N, n_obs, s):
    """Algorithmic HBM bytes of one launch of every pass (what the pass must move)."""
    G = ny * nx
    L = nx // 2
    K1 = (L + 1) * ny
    line = L * ny * 8                 # one field's packed row spectra, complex float
    n_un = M - n_obs
    nf = n_obs + 2 * n_obs * n_un     # floats per wavenumber of the covariance / gain tables
    return {
        "row_fwd_anomaly": M * N * G * s + M * N * line,   # members in (pivot rows re-read through L2), rows out
        "rhat_transpose": 2 * n_obs * K1 * 8,
        "col_stats": M * N * line + n_obs * K1 * 8 + nf * K1 * 4,      # rows in, rhat in, gains out
        "gain": nf * K1 * 4 + n_obs * K1 * 8 + nf * K1 * 4,            # caller-spectrum analyses only
        "row_fwd_innovation": 2 * n_obs * N * G * s + n_obs * G * 4 + n_obs * N * line,
        "col_update": n_obs * N * line + nf * K1 * 4 + M * N * line,
        # fused column pass: anomaly rows in, innovation rows in, rhat in, increment rows out
        "col_fused": M * N * line + n_obs * N * line + n_obs * K1 * 8 + M * N * line,
        "row_inv": M * N * line + 2 * M * N * G * s,
    }


def analysis_bytes(ny, nx, M, N, n_obs, s):
    """The analysis's algorithmic bytes without the separate mean pass (ensemble read for
    chat and for the update, innovations, data, rhat, gains written+read, output,
    one write+read of every transform's intermediate)."""
    G = ny * nx
    K = ny * (nx // 2 + 1)
    n_un = M - n_obs
    return (2 * M * N * G * s + n_obs * N * G * s + n_obs * N * G * s + n_obs * G * 4 + n_obs * K * 8
            + 2 * (n_obs * K * 4 + n_un * n_obs * K * 8) + M * N * G * s + (2 * M * N + n_obs * N) * 2 * K * 8)


# ------------------------------------------------------------ cuFFT reference point
def cufft_reference(ny, nx, M_, N_, n_obs, dev, steps=3, chunk=20):
    """Time of the analysis's 2-D real transforms alone through torch.fft (cuFFT), FP32:
    (M + n_obs) N forward R2C and M N inverse C2R transforms of ny x nx, in batches of `chunk`
    fields, no other work.  A reference point, not this library's path."""
    import torch
    x = torch.randn(chunk, ny, nx, device=dev)
    X = torch.fft.rfft2(x)
    n_fwd, n_inv = (M_ + n_obs) * N_, M_ * N_

    def one():
        for _ in range(n_fwd // chunk):
            torch.fft.rfft2(x, out=X)
        for _ in range(n_inv // chunk):
            torch.fft.irfft2(X, s=(ny, nx), out=x)

    one()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        one()
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    del x, X
    return {"ms_per_step": ms, "transforms": n_fwd + n_inv, "dtype": "f32",
            "note": "torch.fft rfft2/irfft2 (cuFFT) of the analysis's %d forward and %d inverse transforms in "
                    "batches of %d fields; transforms only (no mean, statistics, gains, BF16 I/O)"
                    % (n_fwd, n_inv, chunk)}


# ------------------------------------------------------------ multi-rank reduction
def pick_fused_schedule(plan, step, stream, reps=2):
    """Autotune the fused column pass's line-FFT schedule (0: 16 values per thread, 1: 8 values,
    twice the threads) on the workload itself, before the warm-up: each candidate runs `reps`
    analyses after one untimed one; the faster is kept.  Returns the chosen schedule."""
    import torch
    from paper_1001_1588_gb300 import abi
    fused = abi.fftenkf_pass_count() - 1
    base = abi.fftenkf_get_schedule(plan.handle)
    best, best_ms = base[fused], None
    for sel in (0, 1):
        sched = list(base)
        sched[fused] = sel
        abi.fftenkf_set_schedule(plan.handle, sched)
        step()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            step()
        t1.record(stream)
        t1.synchronize()
        ms = t0.elapsed_time(t1)
        if best_ms is None or ms < best_ms:
            best, best_ms = sel, ms
    sched = list(base)
    sched[fused] = best
    abi.fftenkf_set_schedule(plan.handle, sched)
    return best


def max_over_ranks(value, dist_mod=None, device=None):
    """The largest of every rank's value: a job's time is its slowest rank's."""
    if dist_mod is None or not dist_mod.is_initialized() or dist_mod.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms):
    """Whole-job rate: every rank's units over the slowest rank's time (weak scaling)."""
    return float(units_per_rank) * world / (ms / 1e3)


# ------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "50"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def begin(self):
        """Wait (at most 3 s) until the sampler produces lines; only later samples are summarised."""
        t0 = time.time()
        while self.proc and not self.lines and time.time() - t0 < 3.0:
            time.sleep(0.02)
        self.first = len(self.lines)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[getattr(self, "first", 0):]:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_traffic(pass_name):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        t = json.load(open(path))
    except Exception:
        return None
    ent = t.get(pass_name)
    if not ent or ent.get("source_sha") != source_sha():
        return None
    return ent.get("dram_bytes_per_launch_full")


# sources outside the analysis path whose counters profiles/traffic.json holds: front ends that
# reach the periodic analysis only through its C ABI (sine, batched, allocation-free), and the
# kernels of other workloads (batched, learned spectrum, morphing).  The hash identifies the
# analysis path's kernels and everything they include.
OTHER_SOURCES = ("sine_api.cu", "batch_api.cu", "batch.cuh", "k_batch.cuh", "k_batch.cu", "k_mlp.cu", "mlp_api.cu",
                 "morph_api.cu", "static_api.cu")


def _code_only(text):
    """A source without its comments and blank space: a comment edit leaves the kernels unchanged."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_sha():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1001_1588_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")) and f not in OTHER_SOURCES and not f.startswith("k_batch_"):
            h.update(_code_only(open(os.path.join(csrc, f), encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


# ------------------------------------------------------------ oracle (CPU) baseline
def oracle_sample(ny, nx, n_transforms, seed=7):
    """Time n_transforms full-size oracle 2-D DFTs (dense DFT-matrix products in FP64),
    alternating forward and inverse."""
    import numpy as np
    from oracle import dft
    u = np.random.default_rng(seed).standard_normal((ny, nx))
    t0 = time.perf_counter()
    U = u
    for i in range(n_transforms):
        U = dft.fft2(U) if i % 2 == 0 else dft.ifft2(U)
    return time.perf_counter() - t0


def oracle_rate(ny, nx, M_, N_, n_obs, seconds_per_transform):
    """Metric of the oracle: one analysis costs (2 M N + n_obs N) full-size transforms."""
    transforms = 2 * M_ * N_ + n_obs * N_
    t = transforms * seconds_per_transform
    return ny * nx * N_ / t, transforms


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        return max(int(i.get("num_threads", 1)) for i in threadpool_info()) or os.cpu_count()
    except Exception:
        return os.cpu_count()


def run_oracle_configs(a):
    """Host timings of the FP64 oracle (oracle.enkf.analyze: estimate, gains and update with the
    explicit DFT) on the parity configurations: 1 and 2 in full, the learned-spectrum shape (1024^2,
    N=5, one block) in full, and a sample of the batched workload (the cheapest item of every side
    length).  A baseline only; one JSON line, no GPU."""
    import numpy as np
    from oracle import enkf
    from synth import fields
    threads = cpu_threads()

    def timed(p):
        t0 = time.perf_counter()
        enkf.analyze(p.ensemble, p.data, p.perturbations, p.rhat, p.observed)
        return time.perf_counter() - t0

    res = {}
    for name, p in (("1: 1 block 64^2, N=5", fields.make_config1()),
                    ("2: 3 blocks 512^2, N=5", fields.make_config2())):
        t = timed(p)
        res[name] = {"seconds": t, "value": p.ny * p.nx * p.N / t}
    S = fields.powerlaw_spectrum(1024, 1024, 8.0, -3.5)
    p5 = fields.make_problem(1024, 1024, 5, [S], [1], np.full((1, 1024, 513), 0.1), 20260005, "f32")
    t = timed(p5)
    res["5: 1 block 1024^2, N=5 (plain estimate)"] = {"seconds": t, "value": p5.ny * p5.nx * p5.N / t}
    best = {}
    for it in fields.batched_item_params():
        side = max(it["ny"], it["nx"])
        cost = it["ny"] * it["nx"] * it["N"]
        if side not in best or cost < best[side]["ny"] * best[side]["nx"] * best[side]["N"]:
            best[side] = it
    tot_t, tot_u = 0.0, 0.0
    for it in best.values():
        S = fields.se_spectrum(it["ny"], it["nx"], it["ell"], 1.0)
        p = fields.make_problem(it["ny"], it["nx"], it["N"], [S], [1],
                                np.full((1, it["ny"], it["nx"] // 2 + 1), it["r"]), it["seed"], "f32")
        tot_t += timed(p)
        tot_u += it["ny"] * it["nx"] * it["N"]
    res["4: sample of %d batched items (the cheapest of every side)" % len(best)] = {
        "seconds": tot_t, "value": tot_u / tot_t}
    print(json.dumps({"metric": "FP64 oracle analysis, grid-pts*members/s on the host cores", "unit": UNIT,
                      "workload": "oracle", "kind": "oracle", "cores": threads, "configs": res,
                      "note": "oracle.enkf.analyze (explicit unitary DFT by dense DFT-matrix products, FP64); "
                              "a baseline, not a target"}))
    return 0


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    for _ in range(a.warmup):
        oracle_sample(a.ny, a.nx, 1)
    total = 0.0
    for _ in range(a.steps):
        total += oracle_sample(a.ny, a.nx, 1)
    spt = total / a.steps
    rate, transforms = oracle_rate(a.ny, a.nx, M, a.members, N_OBS, spt)
    sample = ("one full-size %dx%d oracle DFT per step (dense DFT-matrix products, FP64); an analysis "
              "is %d such transforms, the per-wavenumber work is O(G) and not counted" % (a.ny, a.nx, transforms))
    out = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": a.gpus,
        # ms_per_step: the timed sample (one transform) per step, as run; the analysis it stands for
        # would take ms_per_analysis_extrapolated
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": spt * 1e3,
        "ms_per_analysis_extrapolated": spt * transforms * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "grid": [a.ny, a.nx], "members": a.members,
                                        "blocks": M, "observed": N_OBS},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


# ------------------------------------------------------------ our arm
def analysis_rmse(ens, truth):
    """RMSE of the ensemble mean against the truth, per block and over all blocks:
    sqrt(mean_x (mean_k u_k(x) - truth(x))^2) (the evaluation of the learned-spectrum config)."""
    mean = ens.float().mean(dim=1)
    err = (mean - truth.float()) ** 2
    return [float(x) for x in err.mean(dim=(1, 2)).sqrt()], float(err.mean().sqrt())


def compare_precision(dev, ny, nx, Nm, steps=5, warmup=3):
    """The headline draw analysed with FP32 and with BF16 member storage (the BF16 members are the
    FP32 ones rounded): ms per analysis and the analysis RMSE against the truth of each, on the same
    draw, so that throughput is compared at (near) equal RMSE."""
    import torch
    from paper_1001_1588_gb300 import torch_api
    from synth.fields_torch import make_config3_torch
    out = {}
    stream = torch.cuda.current_stream(dev)
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        prob = make_config3_torch(device=dev, ny=ny, nx=nx, N=Nm, storage=dt)
        plan = torch_api.Plan(ny, nx, M, Nm, dt, OBSERVED)
        plan.workspace(dev)
        f_blocks, f_total = analysis_rmse(prob.ensemble, prob.truth)
        ens = prob.ensemble.clone()
        plan.analyze(ens, prob.data, prob.perturbations, prob.rhat)    # the analysis of the draw itself
        a_blocks, a_total = analysis_rmse(ens, prob.truth)
        for _ in range(warmup):
            plan.analyze(ens, prob.data, prob.perturbations, prob.rhat)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            plan.analyze(ens, prob.data, prob.perturbations, prob.rhat)
        t1.record(stream)
        t1.synchronize()
        st = plan.device_status()
        plan.close()
        out[name] = {"ms_per_analysis": t0.elapsed_time(t1) / steps, "rmse_forecast": f_total,
                     "rmse_analysis": a_total, "rmse_analysis_blocks": a_blocks, "rmse_forecast_blocks": f_blocks,
                     "status": st}
        del prob, ens
        torch.cuda.empty_cache()
    out["speedup_bf16_over_f32"] = out["f32"]["ms_per_analysis"] / out["bf16"]["ms_per_analysis"]
    out["rmse_rel_diff_bf16_vs_f32"] = (out["bf16"]["rmse_analysis"] - out["f32"]["rmse_analysis"]) / out["f32"]["rmse_analysis"]
    return out


def compare_batched(dev, count=256, steps=5):
    """The batched draw in FP32 and in BF16 storage: ms per batch (autotuned, graph-replayed) and the
    mean over items of the analysis RMSE against each item's truth, on the same draw."""
    import numpy as np
    import torch
    from paper_1001_1588_gb300 import abi
    from synth.fields_torch import make_batched_torch
    out = {}
    stream = torch.cuda.current_stream(dev)
    for name, dt, code in (("f32", torch.float32, abi.FFTENKF_F32), ("bf16", torch.bfloat16, abi.FFTENKF_BF16)):
        items = make_batched_torch(device=dev, count=count, storage=dt)
        ens0 = [it.ensemble.clone() for it in items]
        b = abi.fftenkf_plan_batched([(it.ny, it.nx, it.N) for it in items], code)
        ws = torch.empty(abi.fftenkf_batch_workspace_size(b), dtype=torch.uint8, device=dev)
        abi.fftenkf_batch_autotune(b, ws, 0)
        for it, e0 in zip(items, ens0):
            it.ensemble.copy_(e0)

        def step():
            abi.fftenkf_analyze_batched(b, [it.ensemble for it in items], [it.data for it in items],
                                        [it.perturbations for it in items], [it.rhat for it in items], ws,
                                        int(stream.cuda_stream))

        step()
        rm_f = float(np.mean([analysis_rmse(e0[None], it.truth[None])[1] for it, e0 in zip(items, ens0)]))
        rm_a = float(np.mean([analysis_rmse(it.ensemble[None], it.truth[None])[1] for it in items]))
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            step()
        t1.record(stream)
        t1.synchronize()
        st = abi.fftenkf_batch_last_device_status(b, int(stream.cuda_stream))
        abi.fftenkf_batch_destroy(b)
        out[name] = {"ms_per_batch": t0.elapsed_time(t1) / steps, "rmse_forecast_mean": rm_f,
                     "rmse_analysis_mean": rm_a, "status": st}
    out["speedup_bf16_over_f32"] = out["f32"]["ms_per_batch"] / out["bf16"]["ms_per_batch"]
    out["rmse_rel_diff_bf16_vs_f32"] = (out["bf16"]["rmse_analysis_mean"] - out["f32"]["rmse_analysis_mean"]) / out["f32"]["rmse_analysis_mean"]
    return out


def compare_learned(dev, grid=1024, pairs=20000, epochs=12, n_draws=64, steps=5):
    """Learned against plain spectrum at grid^2, N = 5 (the learned-spectrum config): the MLP is
    trained on the GPU by the library's kernels on `pairs` (N = 5 estimate, N = 500 target) pairs,
    then analysis RMSE over held-out draws for the plain estimate, the learned spectrum and the true
    generating spectrum; ms per analysis of the plain path and of the learned path (estimate,
    denoise, analysis with the supplied spectrum)."""
    import math
    import torch
    from paper_1001_1588_gb300 import abi, denoiser, torch_api
    t0 = time.time()
    pr = denoiser.Pairs(grid, grid)
    X, Y = pr.generate(pairs, seed=20260005)
    pr.close()
    params, _, _, step_, hist = denoiser.train(X, Y, epochs, 256, 1e-3)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    ev, _ = denoiser.evaluate(params, grid, grid, n_draws=n_draws)
    # timing of one analysis each way on a draw of the same family
    stream = torch.cuda.current_stream(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(99)
    S = denoiser.powerlaw_half(grid, grid, 8.0, -3.5, dev)
    ens = denoiser.draw_fields(S, 5, gen, grid, grid)[None].contiguous()
    truth = denoiser.draw_fields(S, 1, gen, grid, grid)[0]
    data = (truth + math.sqrt(0.1) * torch.randn(grid, grid, device=dev, generator=gen))[None].contiguous()
    pert = (math.sqrt(0.1) * torch.randn(5, 1, grid, grid, device=dev, generator=gen)).contiguous()
    rhat = torch.full((1, grid, grid // 2 + 1), 0.1, dtype=torch.float64, device=dev)
    plan = torch_api.Plan(grid, grid, 1, 5, torch.float32, [1])
    den = abi.fftenkf_denoiser_create(grid, grid, 5)
    learned = torch.empty(grid * (grid // 2 + 1), dtype=torch.float64, device=dev)

    def plain():
        plan.analyze(ens, data, pert, rhat)

    def with_learned():
        chat = plan.estimate_spectrum(ens)
        abi.fftenkf_denoise_spectrum(den, params, chat, learned, 5, int(stream.cuda_stream), want_flag=False)
        plan.analyze(ens, data, pert, rhat, learned)

    times = {}
    for name, fn in (("plain", plain), ("learned", with_learned)):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        times[name] = e0.elapsed_time(e1) / steps
    plan.close()
    abi.fftenkf_denoiser_destroy(den)
    # the plain estimate with more members: the ensemble size at which it matches the learned
    # spectrum's RMSE at N = 5, and what that ensemble costs per analysis
    sweep = plain_members_sweep(dev, grid, (5, 10, 20, 40), n_draws=n_draws)
    match = next((n for n, v in sweep.items() if v["rmse"] <= ev["learned"]), None)
    return {"grid": grid, "members": 5, "pairs": pairs, "epochs": epochs, "train_steps": step_,
            "train_loss": hist[-1], "seconds_pairs_and_train": t_train, "eval": ev,
            "ms_per_analysis_plain": times["plain"], "ms_per_analysis_learned": times["learned"],
            "plain_by_members": sweep, "plain_members_matching_learned_rmse": match}


def plain_members_sweep(dev, grid, Ns, n_draws=32, r=0.1, seed=777, steps=5):
    """Analysis RMSE (mean over held-out draws of the learned-spectrum family: power-law spectra,
    ell log-uniform in [2, 64], slope uniform in [-5, -2], rhat = r) and ms per analysis of the plain
    FFT EnKF with N members, for each N in Ns."""
    import math
    import numpy as np
    import torch
    from paper_1001_1588_gb300 import denoiser, torch_api
    stream = torch.cuda.current_stream(dev)
    rhat = torch.full((1, grid, grid // 2 + 1), r, dtype=torch.float64, device=dev)
    out = {}
    for N in Ns:
        rng = np.random.default_rng(seed)
        gen = torch.Generator(device=dev)
        gen.manual_seed(seed + N)
        plan = torch_api.Plan(grid, grid, 1, N, torch.float32, [1])
        rm = []
        for _ in range(n_draws):
            ell = float(np.exp(rng.uniform(np.log(2.0), np.log(64.0))))
            beta = float(rng.uniform(-5.0, -2.0))
            S = denoiser.powerlaw_half(grid, grid, ell, beta, dev)
            truth = denoiser.draw_fields(S, 1, gen, grid, grid)[0]
            ens = denoiser.draw_fields(S, N, gen, grid, grid)[None].contiguous()
            data = (truth + math.sqrt(r) * torch.randn(grid, grid, device=dev, generator=gen))[None].contiguous()
            pert = (math.sqrt(r) * torch.randn(N, 1, grid, grid, device=dev, generator=gen)).contiguous()
            plan.analyze(ens, data, pert, rhat)
            rm.append(float(torch.sqrt(((ens[0].mean(dim=0) - truth) ** 2).mean()).item()))
        for _ in range(3):
            plan.analyze(ens, data, pert, rhat)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            plan.analyze(ens, data, pert, rhat)
        e1.record(stream)
        e1.synchronize()
        plan.close()
        out[N] = {"rmse": float(np.mean(rm)), "ms_per_analysis": e0.elapsed_time(e1) / steps}
    return out


def run_compare(a):
    """One JSON line with the comparisons of the precision, learned-spectrum and batched forms with
    the plain FP32 FFT EnKF at (near) equal analysis RMSE."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    res = {"metric": "equal-RMSE comparisons (analysis RMSE of the ensemble mean vs truth, ms per analysis)",
           "workload": "compare", "n_gpus": 1, "data": "synthetic"}
    res["precision_4x4096x4096_N20"] = compare_precision(dev, a.ny, a.nx, a.members)
    res["batched_256"] = compare_batched(dev, a.batch)
    res["learned_1024_N5"] = compare_learned(dev)
    print(json.dumps(res))
    return 0


def run_ours(a):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_1001_1588_gb300 import abi, torch_api
    from synth.fields_torch import make_config3_torch

    ny, nx, Nm = a.ny, a.nx, a.members
    prob = make_config3_torch(device=dev, seed=20260003 + 1000 * rank, ny=ny, nx=nx, N=Nm)
    plan = torch_api.Plan(ny, nx, M, Nm, torch.bfloat16, OBSERVED)
    plan.workspace(dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.analyze(prob.ensemble, prob.data, prob.perturbations, prob.rhat)

    if a.fused_schedule == "auto":
        fused_schedule = pick_fused_schedule(plan, step, stream)
    else:   # fixed, e.g. under a profiler, whose serialisation would bias the choice
        fused_schedule = int(a.fused_schedule)
        sched = abi.fftenkf_get_schedule(plan.handle)
        sched[abi.fftenkf_pass_count() - 1] = fused_schedule
        abi.fftenkf_set_schedule(plan.handle, sched)
    for _ in range(max(a.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    if plan.device_status() != 0:
        raise RuntimeError("device status after warm-up: %s" % abi.fftenkf_last_error())

    abi.fftenkf_set_profiling(plan.handle, True)
    abi.fftenkf_pass_times(plan.handle)         # reset
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        gpu_id = str(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(gpu_id) as clk:
        clk.begin()
        start.record(stream)
        for _ in range(a.steps):
            step()
        stop.record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ms = start.elapsed_time(stop)
    times = abi.fftenkf_pass_times(plan.handle)
    abi.fftenkf_set_profiling(plan.handle, False)
    ms = max_over_ranks(ms, dist if world > 1 else None, dev)
    value = job_throughput(float(ny) * nx * Nm * a.steps, world, ms)

    # roofline of the dominant pass
    s = 2
    pb = pass_bytes(ny, nx, M, Nm, N_OBS, s)
    per_pass = {}
    for name, (tot, cnt) in times.items():
        if cnt:
            per_pass[name] = {"ms_per_launch": tot / cnt, "launches": cnt, "share": None}
    # rhat_transpose runs on the plan's auxiliary stream, overlapping the anomaly rows: its event
    # time is wall time shared with them, so shares are taken over the caller-stream passes
    aux = {"rhat_transpose"}
    total_pass_ms = sum(v["ms_per_launch"] * v["launches"] for k, v in per_pass.items() if k not in aux)
    for k, v in per_pass.items():
        if k in aux:
            v["stream"] = "auxiliary (overlapped)"
        else:
            v["share"] = v["ms_per_launch"] * v["launches"] / total_pass_ms if total_pass_ms else None
    dom = max((k for k in per_pass if k in pb), key=lambda k: per_pass[k]["ms_per_launch"] * per_pass[k]["launches"])
    peak, peak_kind = hbm_peak()
    achieved = pb[dom] / (per_pass[dom]["ms_per_launch"] / 1e3) / 1e9
    for k, v in per_pass.items():
        if k in pb:
            v["alg_gbs"] = pb[k] / (v["ms_per_launch"] / 1e3) / 1e9
            v["frac_of_peak"] = v["alg_gbs"] / peak
    B_alg = analysis_bytes(ny, nx, M, Nm, N_OBS, s)
    step_ms = ms / a.steps

    # end to end through the public API with host buffers (pinned), copies inside the timed region:
    # every step copies its inputs host -> device, analyzes, and copies its result back.  Steps are
    # streamed as a user streaming analyses would: device inputs in NB buffers, host -> device
    # copies on one stream, the analysis on the compute stream, device -> host on a third, so
    # that step i+1's input copy overlaps step i's analysis and result copy and waits only for the
    # result copy of step i+1-NB.  The host link (about 211 GB/s in, 193 out, 340 both ways on
    # this machine, whatever the number of streams) bounds a step at (in + out bytes) / 340 GB/s.
    def e2e_run(host_src, analyze_fn, NB=2):
        """ms per step, bytes in and out per step of the streamed pipeline over host copies of
        host_src (the first is the ensemble, analysed in place and copied back)."""
        h_in = [t.cpu().pin_memory() for t in host_src]
        h_out = [torch.empty_like(h_in[0]).pin_memory() for _ in range(NB)]
        d_in = [[torch.empty_like(t) for t in host_src] for _ in range(NB)]
        bi = sum(t.numel() * t.element_size() for t in h_in)
        bo = h_out[0].numel() * h_out[0].element_size()
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(NB)]
        ev_done = [torch.cuda.Event() for _ in range(NB)]
        ev_out = [torch.cuda.Event() for _ in range(NB)]
        for e in ev_out:
            e.record(s_out)

        def e2e_step(i):
            b = i % NB
            s_in.wait_event(ev_out[b])                 # the buffer's previous result has left
            with torch.cuda.stream(s_in):
                for dt, ht in zip(d_in[b], h_in):
                    dt.copy_(ht, non_blocking=True)
                ev_in[b].record(s_in)
            stream.wait_event(ev_in[b])
            analyze_fn(d_in[b], i)
            ev_done[b].record(stream)
            s_out.wait_event(ev_done[b])
            with torch.cuda.stream(s_out):
                h_out[b].copy_(d_in[b][0], non_blocking=True)
                ev_out[b].record(s_out)

        for i in range(NB):
            e2e_step(i)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s_in)
        for i in range(a.e2e_steps):
            e2e_step(i)
        stream.wait_event(ev_out[(a.e2e_steps - 1) % NB])
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ems = max_over_ranks(e0.elapsed_time(e1), dist if world > 1 else None, dev)
        del d_in, h_in, h_out
        return ems, bi, bo

    e2e = None
    e2e_seeded = None
    if not a.no_e2e and a.e2e_steps > 0:
        NB = 2
        ems, bi, bo = e2e_run((prob.ensemble, prob.data, prob.perturbations, prob.rhat),
                              lambda d, i: plan.analyze(*d, stream=stream), NB)
        e2e = {"value": job_throughput(float(ny) * nx * Nm * a.e2e_steps, world, ems), "unit": UNIT,
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "steps": a.e2e_steps,
               "ms_per_step": ems / a.e2e_steps,
               "pipeline": "inputs in %d device buffers; host->device, analysis and device->host on three "
                           "streams, step i+1's input copy overlapping step i" % NB}
        if not a.no_seeded:
            # the same pipeline with the perturbations drawn by the library: no perturbation upload
            ems, bi, bo = e2e_run((prob.ensemble, prob.data, prob.rhat),
                                  lambda d, i: plan.analyze_seeded(d[0], d[1], d[2], 777 + i, stream=stream), NB)
            e2e_seeded = {"value": job_throughput(float(ny) * nx * Nm * a.e2e_steps, world, ems), "unit": UNIT,
                          "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "steps": a.e2e_steps,
                          "ms_per_step": ems / a.e2e_steps,
                          "note": "fftenkf_analyze_seeded: ensemble, data and rhat uploaded, perturbations drawn"}

    # the same analyses with the perturbations drawn by the library (fftenkf_analyze_seeded)
    equal_rmse = None
    if not a.no_compare and world == 1:
        try:
            equal_rmse = compare_precision(dev, ny, nx, Nm)
        except Exception as exc:   # reported, not fatal to the headline line
            equal_rmse = {"error": str(exc)[:200]}
    seeded = None
    if not a.no_seeded:
        for _ in range(max(a.warmup, 1)):
            plan.analyze_seeded(prob.ensemble, prob.data, prob.rhat, 12345)
        torch.cuda.synchronize(dev)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for i in range(a.steps):
            plan.analyze_seeded(prob.ensemble, prob.data, prob.rhat, 12345 + i)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        sms = max_over_ranks(s0.elapsed_time(s1), dist if world > 1 else None, dev) / a.steps
        seeded = {"ms_per_step": sms, "value": job_throughput(float(ny) * nx * Nm, world, sms), "unit": UNIT,
                  "note": "perturbations drawn in frequency space by the library; no perturbation field read"}

    cufft = None
    if rank == 0 and not a.no_cufft:
        cufft = cufft_reference(ny, nx, M, Nm, N_OBS, dev)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        n_tr = 2
        t = oracle_sample(ny, nx, n_tr)
        rate, transforms = oracle_rate(ny, nx, M, Nm, N_OBS, t / n_tr)
        cpu = {"value": rate, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
               "sample": "%d full-size %dx%d oracle DFTs (forward + inverse, dense DFT-matrix products in FP64) "
                         "timed in %.1f s and scaled to the %d transforms of one analysis" % (n_tr, ny, nx, t, transforms)}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (bf16 storage, f64 gain)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [ny, nx], "members": Nm, "blocks": M, "observed": N_OBS,
                       "l2": "inputs larger than L2 (2.7 GB ensemble re-read every step)",
                       "parallelism": "independent analysis per GPU" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": kernel_traffic(dom), "alg_bytes_per_launch": pb[dom]},
            "analysis_roofline": {"alg_bytes": B_alg, "achieved_gbs": B_alg / (step_ms / 1e3) / 1e9,
                                  "frac": B_alg / (step_ms / 1e3) / 1e9 / peak},
            "passes": per_pass,
            "fused_schedule": fused_schedule,
            "clocks": clk.summary(),
            "e2e": e2e,
            "e2e_seeded": e2e_seeded,
            "gpu_launches": sum(v["launches"] for v in per_pass.values()),
            "cpu_baseline": cpu,
            "cufft_reference": cufft,
            "seeded": seeded,
            "equal_rmse_precision": equal_rmse,
            "source_sha": source_sha(),
        }
        print(json.dumps(out))
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------ batched workload
def batched_bytes(items, s):
    """Algorithmic bytes of the batch: the analysis model per item with M = 1 block, observed."""
    return sum(analysis_bytes(it.ny, it.nx, 1, it.N, 1, s) for it in items)


def coupled_bytes(ny, nx, M_, N_, n_obs, s):
    """Byte model of the coupled analysis: the plain model with the gain tables of every block
    (M n_obs complex, written and read) instead of the neglect rule's, plus the covariance
    tables (observed autos, the observed pair, the unobserved crosses) written and read once."""
    K = ny * (nx // 2 + 1)
    n_un = M_ - n_obs
    plain_gains = 2 * (n_obs * K * 4 + n_un * n_obs * K * 8)
    coupled_gains = 2 * (M_ * n_obs * K * 8)
    tables = 2 * (n_obs * K * 4 + (n_obs * (n_obs - 1) // 2 + n_obs * n_un) * K * 8)
    return analysis_bytes(ny, nx, M_, N_, n_obs, s) - plain_gains + coupled_gains + tables


def run_coupled(a):
    """Coupled observed blocks on the largest 4096^2 state whose coupled column statistics fit
    in shared memory: 3 Matern-3/2 blocks (l = 8, 20.16, 50.8), blocks 0 and 1 observed, N=20,
    BF16; the neglect-rule analysis of the same inputs is timed beside it."""
    import torch
    from paper_1001_1588_gb300 import abi, torch_api
    from synth.fields_torch import CONFIG3_ELLS, make_config3_torch

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    ny, nx, Nm, M3 = a.ny, a.nx, a.members, 3
    prob = make_config3_torch(device=dev, ny=ny, nx=nx, N=Nm, ells=CONFIG3_ELLS[:M3], observed=(1, 1, 0))
    out = {}
    peak, peak_kind = hbm_peak()
    for name, coupled in (("coupled", True), ("neglect_rule", False)):
        plan = torch_api.Plan(ny, nx, M3, Nm, torch.bfloat16, (1, 1, 0), coupled=coupled)
        plan.workspace(dev)
        ens0 = prob.ensemble.clone()
        for _ in range(max(a.warmup, 1)):
            plan.analyze(prob.ensemble, prob.data, prob.perturbations, prob.rhat)
        torch.cuda.synchronize(dev)
        if plan.device_status() != 0:
            raise RuntimeError("device status: %s" % abi.fftenkf_last_error())
        abi.fftenkf_set_profiling(plan.handle, True)
        abi.fftenkf_pass_times(plan.handle)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(None) as clk:
            clk.begin()
            e0.record()
            for _ in range(a.steps):
                plan.analyze(prob.ensemble, prob.data, prob.perturbations, prob.rhat)
            e1.record()
            torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / a.steps
        times = abi.fftenkf_pass_times(plan.handle)
        B = coupled_bytes(ny, nx, M3, Nm, 2, 2) if coupled else analysis_bytes(ny, nx, M3, Nm, 2, 2)
        out[name] = {"ms_per_step": ms, "value": float(ny) * nx * Nm / (ms / 1e3),
                     "analysis_roofline": {"alg_bytes": B, "achieved_gbs": B / (ms / 1e3) / 1e9,
                                           "frac": B / (ms / 1e3) / 1e9 / peak, "peak": peak, "peak_kind": peak_kind},
                     "passes": {k: v[0] / v[1] for k, v in times.items() if v[1]}, "clocks": clk.summary()}
        prob.ensemble.copy_(ens0)
        plan.close()
    c = out["coupled"]
    print(json.dumps({
        "metric": "coupled-observed FFT-EnKF analysis grid-pts*members/s (3 blocks 4096^2, N=20, 2 observed)",
        "value": c["value"], "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": c["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (bf16 storage, f64 bracket inverse)", "data": "synthetic",
        "config": {"workload": "coupled observed blocks: 3 Matern-3/2 blocks 4096x4096, N=20, BF16, blocks 0, 1 "
                               "observed, observed cross-covariance kept"},
        "analysis_roofline": c["analysis_roofline"], "passes": c["passes"], "clocks": c["clocks"],
        "neglect_rule": out["neglect_rule"], "gpu_launches": 7 * a.steps,   # rhat_t, rows, stats, gain, rows, update, rows
    }))
    return 0


def sine_extension_bytes(ny, nx, M_, N_, n_obs, s):
    """Bytes the odd-extension form moves beyond the periodic analysis of the 2(ny-1) x 2(nx-1)
    extension: extension writes of ensemble, data and perturbations (reads of their interiors),
    the extended rhat, and the interior copy back."""
    Py, Px = 2 * (ny - 1), 2 * (nx - 1)
    G, Ge = ny * nx, Py * Px
    ext = (M_ * N_ * s + n_obs * 4 + N_ * n_obs * s) * (G + Ge)
    rh = n_obs * ((ny - 2) * (nx - 2) + Py * (Px // 2 + 1)) * 8
    back = 2 * M_ * N_ * (ny - 2) * (nx - 2) * s
    return ext + rh + back


def run_sine(a):
    """The real sine transform variant (Sec. 4) on 2049 x 2049 nodes (interior 2047^2, periodic
    extension 4096^2), 4 blocks, N=20, BF16, blocks 0 and 1 observed; inputs are the 2049^2
    window of the stationary 4096^2 Matern-3/2 fields; the periodic 4096^2 analysis the plan runs
    internally is timed beside it."""
    import torch
    from paper_1001_1588_gb300 import abi, torch_api
    from synth.fields_torch import make_config3_torch

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    n, Nm, M4 = 2049, a.members, 4
    prob = make_config3_torch(device=dev, ny=4096, nx=4096, N=Nm)
    ens = prob.ensemble[:, :, :n, :n].contiguous()
    data = prob.data[:, :n, :n].contiguous()
    pert = prob.perturbations[:, :, :n, :n].contiguous()
    k = torch.sqrt(torch.arange(1, n - 1, device=dev, dtype=torch.float64)[:, None] ** 2
                   + torch.arange(1, n - 1, device=dev, dtype=torch.float64)[None, :] ** 2)
    rhat = (0.1 / k)[None].repeat(2, 1, 1).contiguous()
    peak, peak_kind = hbm_peak()
    plan = torch_api.SinePlan(n, n, M4, Nm, torch.bfloat16, (1, 1, 0, 0))
    ens0 = ens.clone()
    for _ in range(max(a.warmup, 1)):
        plan.analyze(ens, data, pert, rhat)
    torch.cuda.synchronize(dev)
    if plan.device_status() != 0:
        raise RuntimeError("device status: %s" % abi.fftenkf_last_error())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(None) as clk:
        clk.begin()
        e0.record()
        for _ in range(a.steps):
            plan.analyze(ens, data, pert, rhat)
        e1.record()
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / a.steps
    plan.close()
    ens.copy_(ens0)
    del ens, ens0, data, pert
    ms_p = None
    if not a.no_side:
        # the periodic analysis of the extension's size, alone
        pp = torch_api.Plan(4096, 4096, M4, Nm, torch.bfloat16, (1, 1, 0, 0))
        pp.workspace(dev)
        for _ in range(max(a.warmup, 1)):
            pp.analyze(prob.ensemble, prob.data, prob.perturbations, prob.rhat)
        e0.record()
        for _ in range(a.steps):
            pp.analyze(prob.ensemble, prob.data, prob.perturbations, prob.rhat)
        e1.record()
        torch.cuda.synchronize(dev)
        ms_p = e0.elapsed_time(e1) / a.steps
        pp.close()
    B_native = analysis_bytes(n - 2, n - 2, M4, Nm, 2, 2)
    B_ext = analysis_bytes(4096, 4096, M4, Nm, 2, 2) + sine_extension_bytes(n, n, M4, Nm, 2, 2)
    print(json.dumps({
        "metric": "sine-transform FFT-EnKF analysis grid-pts*members/s (2049^2 nodes, 4 blocks, N=20)",
        "value": float(n) * n * Nm / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (bf16 storage, f64 mean and gains)", "data": "synthetic",
        "config": {"workload": "real sine transform (DST-I) variant: 4 Matern-3/2 blocks on 2049x2049 nodes "
                               "(boundary kept), N=20, BF16, blocks 0, 1 observed, odd extension to 4096x4096",
                   "l2": "inputs larger than L2"},
        "analysis_roofline": {"native_alg_bytes": B_native, "extension_alg_bytes": B_ext,
                              "achieved_gbs_extension": B_ext / (ms / 1e3) / 1e9,
                              "frac_extension": B_ext / (ms / 1e3) / 1e9 / peak,
                              "frac_native": B_native / (ms / 1e3) / 1e9 / peak, "peak": peak,
                              "peak_kind": peak_kind},
        "periodic_extension_ms": ms_p, "extension_overhead_ms": None if ms_p is None else ms - ms_p, "clocks": clk.summary(),
        "gpu_launches": 10 * a.steps,   # 3 extensions, rhat extension, 5 of the periodic analysis, interior copy
    }))
    return 0


def batched_launches(items):
    """Launches of one batched analysis: an analysis of at least 512 x 256 points runs on its own
    plan (rhat transposition, anomaly rows, innovation rows, inverse rows, and the fused column
    pass for 512-4096-point power-of-two columns, else the statistics and update passes); the
    others share the 7 persistent launches."""
    big = [it for it in items if it.ny * it.nx >= 512 * 256]
    n = sum(5 if (it.ny >= 512 and (it.ny & (it.ny - 1)) == 0) else 6 for it in big)
    return n + (7 if len(big) < len(items) else 0)


def run_batched(a):
    import torch
    from paper_1001_1588_gb300 import abi
    from synth.fields_torch import make_batched_torch

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    items = make_batched_torch(device=dev, count=a.batch)
    b = abi.fftenkf_plan_batched([(it.ny, it.nx, it.N) for it in items], abi.FFTENKF_F32)
    ws = torch.empty(abi.fftenkf_batch_workspace_size(b), dtype=torch.uint8, device=dev)
    tuned_ms = None if a.no_autotune else abi.fftenkf_batch_autotune(b, ws, 0)
    stream = torch.cuda.current_stream(dev)

    def step():
        abi.fftenkf_analyze_batched(b, [it.ensemble for it in items], [it.data for it in items],
                                    [it.perturbations for it in items], [it.rhat for it in items], ws,
                                    int(stream.cuda_stream))

    for _ in range(max(a.warmup, 1)):
        step()
    torch.cuda.synchronize(dev)
    if abi.fftenkf_batch_last_device_status(b, int(stream.cuda_stream)) != 0:
        raise RuntimeError("batched device status: %s" % abi.fftenkf_last_error())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(None) as clk:
        clk.begin()
        e0.record(stream)
        for _ in range(a.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / a.steps
    units = sum(it.ny * it.nx * it.N for it in items)
    B = batched_bytes(items, 4)
    peak, peak_kind = hbm_peak()
    bt, sc = abi.fftenkf_batch_schedule(b)
    out = {
        "metric": "batched FFT-EnKF analyses, grid-pts*members/s (%d mixed single-block analyses)" % len(items),
        "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "batched: %d single-block analyses, sides {64..1024} square and 2:1, N in 5..25, "
                               "SE spectra, flat rhat, FP32, one CUDA graph: analyses of >= 512x256 points on "
                               "their own plans on 8 branches, the others in 7 persistent launches" % len(items),
                   "grid_points_total": sum(it.ny * it.nx for it in items), "members_total": sum(it.N for it in items)},
        "analysis_roofline": {"alg_bytes": B, "achieved_gbs": B / (ms / 1e3) / 1e9,
                              "frac": B / (ms / 1e3) / 1e9 / peak, "peak": peak, "peak_kind": peak_kind},
        "schedule": {"cta_threads": bt, "line_fft": sc, "autotuned_sum_ms": tuned_ms},
        "clocks": clk.summary(), "gpu_launches": batched_launches(items) * a.steps,
    }
    print(json.dumps(out))
    abi.fftenkf_batch_destroy(b)
    return 0


def morph_bytes(ny, nx, M_, K):
    """Algorithmic bytes of the morphing kernels (FP32): forward reads T (8 B) and M members and
    writes M residuals per (member, node), plus the reference once; the inverse reads T and M
    residuals and writes M members per (member, node), plus the reference once; the reference mean
    reads C = M+2 channels of K members and writes C planes."""
    plane = ny * nx
    fwd = K * plane * (8 + 8 * M_) + 4 * M_ * plane
    inv = K * plane * (8 + 8 * M_) + 4 * M_ * plane
    ref = 4 * (M_ + 2) * plane * (K + 1)
    return fwd, ref, inv


def run_morph(a):
    """Morphing FFT EnKF (Sec. 2.2) at 4096^2, M = 2 physical blocks, N = 20, FP32: transform of the
    members and the data, FFT EnKF on the extended state (T_x, T_y, r^(1) observed, r^(2)
    unobserved), reference mean, inverse transform of the members and of the reference.  Inputs:
    smooth seeded fields (a 128^2 seeded grid upsampled on the device), displacements of up to 3
    cells, data perturbations of standard deviation 0.1, rhat = 0.01; the fixed-point inverse takes at
    most 20 steps and stops at a step of at most 1e-5 cells."""
    import torch
    from paper_1001_1588_gb300 import abi, torch_api
    from synth import fields

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    ny, nx, K, M_, n_iter, tol = a.ny, a.nx, a.members, 2, 20, 1e-5
    up = torch.nn.Upsample(size=(ny, nx), mode="bilinear", align_corners=False)

    def smooth(arr):
        return up(torch.from_numpy(arr).to(dev)).contiguous()

    u = smooth(fields.smooth_members(61, M_, K, 128, 128, ell=6.0))
    T = smooth(fields.smooth_mappings(62, K, 128, 128, amp=3.0, ell=6.0))
    u_ref = smooth(fields.smooth_members(63, M_, 1, 128, 128, ell=6.0))[:, 0].contiguous()
    d = smooth(fields.smooth_members(64, 1, 1, 128, 128, ell=6.0))
    T0 = smooth(fields.smooth_mappings(65, 1, 128, 128, amp=3.0, ell=6.0))
    g = torch.Generator(device=dev).manual_seed(66)
    pert = (0.1 * torch.randn((K, 3, ny, nx), generator=g, device=dev)).contiguous()
    rhat = torch.full((3, ny, nx // 2 + 1), 0.01, dtype=torch.float64, device=dev)
    ext = torch.empty((M_ + 2, K, ny, nx), dtype=torch.float32, device=dev)
    data = torch.empty((3, 1, ny, nx), dtype=torch.float32, device=dev)
    ext_ref = torch.empty((M_ + 2, ny, nx), dtype=torch.float32, device=dev)
    ua = torch.empty((M_, K, ny, nx), dtype=torch.float32, device=dev)
    ua_ref = torch.empty((M_, 1, ny, nx), dtype=torch.float32, device=dev)
    plan = torch_api.Plan(ny, nx, M_ + 2, K, torch.float32, (1, 1, 1, 0))
    s = torch.cuda.current_stream(dev).cuda_stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    acc = [0.0] * 5

    def step(timed):
        ext[:2].copy_(T)
        data[:2].copy_(T0)
        if timed:
            ev[0].record()
        abi.fftenkf_morph_forward(u, u_ref, ext, M_, K, ny, nx, n_iter, tol, s)
        abi.fftenkf_morph_forward(d, u_ref, data, 1, 1, ny, nx, n_iter, tol, s)
        if timed:
            ev[1].record()
        plan.analyze(ext, data.view(3, ny, nx), pert, rhat)
        if timed:
            ev[2].record()
        abi.fftenkf_morph_reference(ext, ext_ref, M_ + 2, K, ny, nx, s)
        if timed:
            ev[3].record()
        abi.fftenkf_morph_inverse(ext, u_ref, ua, M_, K, ny, nx, s)
        abi.fftenkf_morph_inverse(ext_ref, u_ref, ua_ref, M_, 1, ny, nx, s)
        if timed:
            ev[4].record()
            torch.cuda.synchronize(dev)
            for i in range(4):
                acc[i] += ev[i].elapsed_time(ev[i + 1])
            acc[4] += ev[0].elapsed_time(ev[4])

    for _ in range(max(a.warmup, 1)):
        step(False)
    torch.cuda.synchronize(dev)
    if plan.device_status() != 0:
        raise RuntimeError("device status: %s" % abi.fftenkf_last_error())
    with ClockSampler(None) as clk:
        clk.begin()
        for _ in range(a.steps):
            step(True)
    plan.close()
    f_ms, an_ms, r_ms, i_ms, ms = (x / a.steps for x in acc)
    fwd_b, ref_b, inv_b = morph_bytes(ny, nx, M_, K)
    fwd_b += morph_bytes(ny, nx, 1, 1)[0]
    inv_b += morph_bytes(ny, nx, M_, 1)[2]
    peak, peak_kind = hbm_peak()
    print(json.dumps({
        "metric": "morphing FFT-EnKF analysis grid-pts*members/s (4096^2, 2 blocks, N=20)",
        "value": float(ny) * nx * K / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (f64 mean and gains)", "data": "synthetic",
        "config": {"workload": "morphing FFT EnKF: 2 smooth blocks 4096x4096 and smooth mappings (|T| <= 3 cells), "
                               "N=20, FP32, extended state (T_x, T_y, r1, r2) with T_x, T_y, r1 observed, "
                               "fixed-point inverse: at most 20 steps, stop at a step of <= 1e-5 cells", "l2": "inputs larger than L2"},
        "parts_ms": {"forward": f_ms, "analysis": an_ms, "reference": r_ms, "inverse": i_ms},
        "roofline": {"bound": "hbm", "kernel": "morph_forward_kernel + morph_inverse_kernel",
                     "achieved": (fwd_b + inv_b) / ((f_ms + i_ms) / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": (fwd_b + inv_b) / ((f_ms + i_ms) / 1e3) / 1e9 / peak, "peak_kind": peak_kind,
                     "traffic": None},
        "reference_gbs": ref_b / (r_ms / 1e3) / 1e9,
        "clocks": clk.summary(),
        "gpu_launches": 11 * a.steps,   # 2 forward, 6 of the 4-block analysis, reference, 2 inverse
    }))
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "batched":
        return run_batched(a)
    if a.workload == "coupled":
        return run_coupled(a)
    if a.workload == "sine":
        return run_sine(a)
    if a.workload == "morph":
        return run_morph(a)
    if a.workload == "oracle":
        return run_oracle_configs(a)
    if a.workload == "compare":
        return run_compare(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
