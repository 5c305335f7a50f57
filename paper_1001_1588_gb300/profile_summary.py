"""Summaries of ncu CSV logs of the analysis (launch lists and DRAM traffic per pass).

    python -m paper_1001_1588_gb300.profile_summary launches LOG.csv
    python -m paper_1001_1588_gb300.profile_summary traffic LOG.csv --ny 4096 --small-members 4 \
        --full-members 20 [--json profiles/traffic.json]

LOG.csv is `ncu --csv --log-file` output of `--metrics gpu__time_duration.sum` (launches) or of
`--metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum` over one analysis
(traffic).  Launches of one analysis come in the order of PASS_ORDER; the traffic of a full-size
launch is the measured traffic/algorithmic ratio times the full-size algorithmic bytes of the
byte model in bench.py.  Prints a markdown table.
"""

from __future__ import annotations

import argparse
import csv
import importlib.util
import json
import os
import re
from collections import OrderedDict

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# kernels of one analysis with the library's estimated spectrum, in launch order
PASS_ORDER = ["rhat_transpose", "mean", "row_fwd_anomaly", "col_stats", "row_fwd_innovation", "col_update", "row_inv"]
OURS = re.compile(r"(rhat_transpose|mean_kernel|mean_staged_kernel|row_fwd_kernel|col_stats_kernel|gain_kernel|"
                  r"coupled_gain_kernel|col_update_kernel|row_inv_kernel|chat_out|odd_extend_kernel|interior_copy_kernel|"
                  r"rhat_extend_kernel|sine_tables_kernel)")


def read(path):
    """[(launch id, kernel, {metric: value})] in launch order, library kernels only."""
    rows = OrderedDict()
    with open(path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        name = r["Kernel Name"]
        if not OURS.search(name):
            continue
        key = int(r["ID"])
        ent = rows.setdefault(key, (short(name), {}))
        ent[1][r["Metric Name"]] = float(r["Metric Value"].replace(",", ""))
    return [(k, n, m) for k, (n, m) in rows.items()]


def short(name):
    name = name.replace("void ", "").replace("fftenkf::", "")
    return re.sub(r"\(.*\)$", "", name)


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


def byte_model():
    spec = importlib.util.spec_from_file_location("bench_model", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def traffic(path, ny, nx, M, n_obs, s, n_small, n_full, sha):
    b = byte_model()
    small = b.pass_bytes(ny, nx, M, n_small, n_obs, s)
    full = b.pass_bytes(ny, nx, M, n_full, n_obs, s)
    rows = read(path)
    if len(rows) < len(PASS_ORDER):
        raise SystemExit("expected %d launches of one analysis, found %d" % (len(PASS_ORDER), len(rows)))
    table = ["| pass | kernel | time us (N=%d) | DRAM read GB | DRAM write GB | traffic GB | algorithmic GB | "
             "traffic/alg | traffic per full launch GB (N=%d) |" % (n_small, n_full), "|---|---|---|---|---|---|---|---|---|"]
    js = {}
    for pname, (_, kname, m) in zip(PASS_ORDER, rows[:len(PASS_ORDER)]):
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
    ap.add_argument("csv")
    ap.add_argument("--ny", type=int, default=4096)
    ap.add_argument("--blocks", type=int, default=4)
    ap.add_argument("--observed", type=int, default=2)
    ap.add_argument("--storage-bytes", type=int, default=2)
    ap.add_argument("--small-members", type=int, default=4)
    ap.add_argument("--full-members", type=int, default=20)
    ap.add_argument("--json", default="")
    a = ap.parse_args(argv)
    if a.mode == "launches":
        print(launches(a.csv))
        return 0
    sha = byte_model().source_sha()
    table, js = traffic(a.csv, a.ny, a.ny, a.blocks, a.observed, a.storage_bytes, a.small_members, a.full_members, sha)
    print("Sources: `%s`\n" % sha)
    print(table)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(js, f, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
