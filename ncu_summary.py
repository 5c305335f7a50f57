"""Summaries of ncu CSV logs of the analysis: launch lists, and DRAM traffic per pass.

    python ncu_summary.py launches LOG.csv
    python ncu_summary.py traffic LOG1.csv [LOG2.csv ...] --ny 4096 --small-members 4 \\
        --full-members 20 [--json profiles/traffic.json]

A LOG is `ncu --csv --log-file` output.  For `launches` it holds `--metrics gpu__time_duration.sum`
over any number of launches (per kernel: launches, total time, share).  For `traffic` every LOG
holds `--metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum` of one launch
of one kernel of the analysis (`-k <kernel> -c 1`), captured on a small case (small-members).  The
traffic of a full-size launch is the measured traffic / algorithmic ratio times the full-size
algorithmic bytes of bench.py's byte model (every pass's bytes grow in proportion to the members,
except rhat_transpose's, which do not depend on them).  Prints a markdown table; --json writes the
per-pass figures that bench.py reports as roofline.traffic, stamped with bench.py's source hash.
"""

from __future__ import annotations

import argparse
import csv
import importlib.util
import json
import os
import re
from collections import OrderedDict

ROOT = os.path.dirname(os.path.abspath(__file__))
# kernel name -> pass name of bench.py's byte model
PASSES = [
    (re.compile(r"rhat_transpose_kernel"), "rhat_transpose"),
    (re.compile(r"row_anom_kernel"), "row_fwd_anomaly"),
    (re.compile(r"row_fwd_kernel"), "row_fwd_innovation"),
    (re.compile(r"col_fused_kernel"), "col_fused"),
    (re.compile(r"col_stats_kernel"), "col_stats"),
    (re.compile(r"col_update_kernel"), "col_update"),
    (re.compile(r"row_inv_kernel"), "row_inv"),
]
OURS = re.compile(r"(rhat_transpose|row_anom|row_fwd|col_fused|col_stats|col_update|row_inv|gain_kernel|"
                  r"coupled_gain|chat_out|odd_extend|interior_copy|rhat_extend|sine_tables|mlp_|morph|batch|"
                  r"stage_twiddles|plain_twiddles)")


def read(path):
    """[(launch id, kernel, {metric: value})] in launch order, library kernels only."""
    rows = OrderedDict()
    with open(path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        name = r["Kernel Name"]
        if not OURS.search(name):
            continue
        ent = rows.setdefault(int(r["ID"]), (short(name), {}))
        ent[1][r["Metric Name"]] = float(r["Metric Value"].replace(",", ""))
    return [(k, n, m) for k, (n, m) in rows.items()]


def short(name):
    name = name.replace("void ", "").replace("fftenkf::", "")
    return re.sub(r"\(.*\)$", "", name)


def pass_of(kernel):
    for rx, p in PASSES:
        if rx.search(kernel):
            return p
    return None


def launches(path):
    agg = OrderedDict()
    for _, name, m in read(path):
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += m.get("gpu__time_duration.sum", 0.0) / 1e3
    tot = sum(v[1] for v in agg.values()) or 1.0
    out = ["| kernel | launches | total us | per launch us | share |", "|---|---|---|---|---|"]
    for name, (n, us) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        out.append("| `%s` | %d | %.0f | %.0f | %.1f%% |" % (name, n, us, us / n, 100.0 * us / tot))
    return "\n".join(out)


def bench_module():
    spec = importlib.util.spec_from_file_location("bench_model", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def traffic(paths, ny, nx, M, n_obs, s, n_small, n_full, sha):
    b = bench_module()
    small = b.pass_bytes(ny, nx, M, n_small, n_obs, s)
    full = b.pass_bytes(ny, nx, M, n_full, n_obs, s)
    table = ["| pass | kernel | time us (N=%d) | DRAM read GB | DRAM write GB | traffic GB | algorithmic GB | "
             "traffic/alg | traffic per full launch GB (N=%d) |" % (n_small, n_full), "|---|---|---|---|---|---|---|---|---|"]
    js = {}
    for path in paths:
        for _, kname, m in read(path):
            pname = pass_of(kname)
            if pname is None or pname in js:
                continue
            rd, wr = m.get("dram__bytes_read.sum", 0.0), m.get("dram__bytes_write.sum", 0.0)
            tr = rd + wr
            ratio = tr / small[pname]
            js[pname] = {"kernel": kname, "source_sha": sha, "small_case": "%dx%d M=%d N=%d" % (ny, nx, M, n_small),
                         "dram_bytes_per_launch_small": tr, "dram_bytes_per_launch_full": ratio * full[pname],
                         "scale": "traffic/algorithmic ratio at the small N times algorithmic bytes at the full N"}
            table.append("| %s | `%s` | %.0f | %.3f | %.3f | %.3f | %.3f | %.2f | %.2f |" % (
                pname, kname, m.get("gpu__time_duration.sum", 0.0) / 1e3, rd / 1e9, wr / 1e9, tr / 1e9,
                small[pname] / 1e9, ratio, ratio * full[pname] / 1e9))
    return "\n".join(table), js


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("mode", choices=["launches", "traffic"])
    ap.add_argument("csv", nargs="+")
    ap.add_argument("--ny", type=int, default=4096)
    ap.add_argument("--blocks", type=int, default=4)
    ap.add_argument("--observed", type=int, default=2)
    ap.add_argument("--storage-bytes", type=int, default=2)
    ap.add_argument("--small-members", type=int, default=4)
    ap.add_argument("--full-members", type=int, default=20)
    ap.add_argument("--json", default="")
    a = ap.parse_args(argv)
    if a.mode == "launches":
        for path in a.csv:
            print(launches(path))
        return 0
    sha = bench_module().source_sha()
    table, js = traffic(a.csv, a.ny, a.ny, a.blocks, a.observed, a.storage_bytes, a.small_members,
                        a.full_members, sha)
    print("Sources: `%s`\n" % sha)
    print(table)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(js, f, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
