"""Summaries of ncu launch lists for profiles/ (text in, markdown out).

Reads the CSV that ``ncu --csv --log-file X --metrics gpu__time_duration.sum[,dram__bytes_read.sum,
dram__bytes_write.sum]`` writes and prints a markdown table per kernel (launches, device time, share,
DRAM bytes when captured). With ``--traffic`` it adds the machine-readable lines bench.py reads:

    traffic_bytes_per_launch: <DRAM read + write bytes of the selected launches / units>
    sources: <files of the kernels measured, comma separated>
    source_sha: <hash of those files when the capture was summarised>

``--select REGEX`` restricts the traffic sum to kernels whose name matches; ``--units-regex REGEX``
divides it by the number of launches of the kernel that matches (one per unit, e.g. one per
multigrid cycle); without it the sum covers the whole capture (one unit).

    python -m paper_2011_13926_gb300.ncu_summary launches.csv [--traffic --sources a.cu,b.cu ...]
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import os
import re
from collections import OrderedDict

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCALE = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "tbyte": 1e12,
          "b": 1.0, "kb": 1e3, "mb": 1e6, "gb": 1e9, "tb": 1e12,
          "nsecond": 1e-9, "usecond": 1e-6, "msecond": 1e-3, "second": 1.0,
          "ns": 1e-9, "us": 1e-6, "ms": 1e-3, "s": 1.0}


def source_hash(files) -> str:
    """sha256 (16 hex digits) over the bytes of the files, paths relative to the repository root."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_launches(path):
    """[(id, kernel, {metric: value in bytes or seconds})] in launch order."""
    rows = OrderedDict()
    with open(path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]  # ncu prints its own log lines before the CSV
    for r in csv.DictReader(lines):
        key = r["ID"]
        ent = rows.setdefault(key, [r["Kernel Name"], {}])
        unit = r.get("Metric Unit", "").strip().lower()
        val = float(r["Metric Value"].replace(",", ""))
        ent[1][r["Metric Name"]] = val * _SCALE.get(unit, 1.0)
    return [(k, v[0], v[1]) for k, v in rows.items()]


def summarise(launches, select=None, units_regex=None):
    per = OrderedDict()
    total_t = 0.0
    for _, name, m in launches:
        t = m.get("gpu__time_duration.sum", 0.0)
        b = m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0)
        e = per.setdefault(name, [0, 0.0, 0.0])
        e[0] += 1
        e[1] += t
        e[2] += b
        total_t += t
    has_dram = any("dram__bytes_read.sum" in m for _, _, m in launches)
    out = ["| kernel | launches | total ms | share | avg us |" + (" DRAM MB |" if has_dram else ""),
           "|---|---|---|---|---|" + ("---|" if has_dram else "")]
    for name, (n, t, b) in sorted(per.items(), key=lambda kv: -kv[1][1]):
        row = f"| `{name}` | {n} | {t * 1e3:.2f} | {100 * t / total_t:.1f}% | {t / n * 1e6:.1f} |"
        if has_dram:
            row += f" {b / 1e6:.1f} |"
        out.append(row)
    out.append(f"| total | {len(launches)} | {total_t * 1e3:.2f} | 100% | |" + (
        f" {sum(v[2] for v in per.values()) / 1e6:.1f} |" if has_dram else ""))
    traffic, units = None, 1
    if has_dram:
        sel = re.compile(select) if select else None
        traffic = sum(v[2] for k, v in per.items() if sel is None or sel.search(k))
        if units_regex:
            ur = re.compile(units_regex)
            units = sum(v[0] for k, v in per.items() if ur.search(k))
            traffic = traffic / max(units, 1)
    return "\n".join(out), traffic, units


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("--traffic", action="store_true")
    ap.add_argument("--select", default=None)
    ap.add_argument("--units-regex", default=None)
    ap.add_argument("--sources", default="")
    a = ap.parse_args()
    table, traffic, units = summarise(read_launches(a.csv), a.select, a.units_regex)
    print(table)
    if a.traffic and traffic is not None:
        files = [f.strip() for f in a.sources.split(",") if f.strip()]
        print()
        print(f"- traffic_bytes_per_launch: {traffic:.6g}")
        print(f"- units: {units}")
        print(f"- sources: {', '.join(files)}")
        print(f"- source_sha: {source_hash(files)}")


if __name__ == "__main__":
    main()
