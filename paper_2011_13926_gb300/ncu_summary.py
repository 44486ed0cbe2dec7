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


def read_launches(path, by_grid=False):
    """[(id, kernel, {metric: value in bytes or seconds})] in launch order (by_grid: the
    kernel name carries its grid size, so that launches of one kernel on different
    grids, e.g. multigrid levels, stay apart)."""
    rows = OrderedDict()
    with open(path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]  # ncu prints its own log lines before the CSV
    for r in csv.DictReader(lines):
        key = r["ID"]
        label = r["Kernel Name"] + (f" grid {r['Grid Size']}" if by_grid else "")
        ent = rows.setdefault(key, [label, {}])
        unit = r.get("Metric Unit", "").strip().lower()
        val = float(r["Metric Value"].replace(",", ""))
        ent[1][r["Metric Name"]] = val * _SCALE.get(unit, 1.0)
    return [(k, v[0], v[1]) for k, v in rows.items()]


def short_name(name: str) -> str:
    """Kernel name without its parameter list and return type."""
    depth, cut = 0, len(name)
    for i, ch in enumerate(name):  # the first '(' outside template brackets opens the parameter list
        if ch == "<":
            depth += 1
        elif ch == ">":
            depth -= 1
        elif ch == "(" and depth == 0:
            cut = i
            break
    out = name[:cut]
    return out[5:] if out.startswith("void ") else out


def complete_units(launches, start_regex, end_regex):
    """The launches from the first one whose kernel matches start_regex through the last
    one matching end_regex: a capture cut off by its launch count (ncu -c) then holds
    whole units only (e.g. whole multigrid cycles, from the level-0 down pass to the
    level-0 up pass)."""
    st, en = re.compile(start_regex), re.compile(end_regex)
    first = next((i for i, (_, name, _) in enumerate(launches) if st.search(name)), None)
    last = next((i for i in range(len(launches) - 1, -1, -1) if en.search(launches[i][1])), None)
    if first is None or last is None or last < first:
        return []
    return launches[first:last + 1]


def summarise(launches, select=None, units_regex=None, short=False, only_selected=False):
    per = OrderedDict()
    total_t = 0.0
    for _, name, m in launches:
        if short:
            grid = name[name.rfind(" grid "):] if " grid " in name else ""
            name = short_name(name[:len(name) - len(grid)] if grid else name) + grid
        t = m.get("gpu__time_duration.sum", 0.0)
        b = m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0)
        e = per.setdefault(name, [0, 0.0, 0.0])
        e[0] += 1
        e[1] += t
        e[2] += b
        total_t += t
    has_dram = any("dram__bytes_read.sum" in m for _, _, m in launches)
    if only_selected and select:
        sel0 = re.compile(select)
        per = OrderedDict((k, v) for k, v in per.items() if sel0.search(k))
        total_t = sum(v[1] for v in per.values())
        launches = [x for x in launches if sel0.search(short_name(x[1]) if short else x[1])]
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
    ap.add_argument("--short-names", action="store_true", help="kernel names without parameter lists")
    ap.add_argument("--by-grid", action="store_true", help="one row per kernel and grid size")
    ap.add_argument("--only-selected", action="store_true", help="the table lists the --select kernels only")
    ap.add_argument("--unit-end", default=None,
                    help="with --units-regex: keep only whole units, from the first launch matching --units-regex "
                         "through the last launch matching this regex")
    a = ap.parse_args()
    launches = read_launches(a.csv, a.by_grid)
    if a.unit_end and a.units_regex:
        launches = complete_units(launches, a.units_regex, a.unit_end)
    table, traffic, units = summarise(launches, a.select, a.units_regex, a.short_names, a.only_selected)
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
