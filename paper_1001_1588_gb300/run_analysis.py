"""Run the 4-block FFT EnKF analysis on synthetic fields and print per-pass device times.

    python -m paper_1001_1588_gb300.run_analysis [--ny 4096] [--members 20] [--steps 3] [--schedule 0,0,...]

Draws the Matern-3/2, 4-block, 2-observed BF16 workload on the device (synth.fields_torch),
runs two warm-up analyses and `--steps` timed ones with the library's per-pass CUDA-event
timing, and prints one JSON line {pass: ms per launch}.  Used to drive ncu captures.
"""

from __future__ import annotations

import argparse
import json
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--ny", type=int, default=4096)
    ap.add_argument("--members", type=int, default=20)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--schedule", default="")
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    from paper_1001_1588_gb300 import abi, torch_api
    from synth.fields_torch import make_config3_torch

    p = make_config3_torch(ny=a.ny, nx=a.ny, N=a.members)
    plan = torch_api.Plan(a.ny, a.ny, 4, a.members, torch.bfloat16, (1, 1, 0, 0))
    if a.schedule:
        abi.fftenkf_set_schedule(plan.handle, [int(x) for x in a.schedule.split(",")])
    plan.workspace()
    for _ in range(a.warmup):
        plan.analyze(p.ensemble, p.data, p.perturbations, p.rhat)
    torch.cuda.synchronize()
    abi.fftenkf_set_profiling(plan.handle, True)
    for _ in range(a.steps):
        plan.analyze(p.ensemble, p.data, p.perturbations, p.rhat)
    t = abi.fftenkf_pass_times(plan.handle)
    status = plan.device_status()
    out = {k: round(v[0] / v[1], 4) for k, v in t.items() if v[1]}
    out["sum_ms_per_step"] = round(sum(v[0] for v in t.values()) / max(a.steps, 1), 3)
    out["status"] = status
    print(json.dumps(out))
    plan.close()
    return 0 if status == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
