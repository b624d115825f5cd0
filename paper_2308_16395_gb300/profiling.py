"""Summaries of ncu CSV launch lists (``--csv --log-file``) of this library's kernels.

  python -m paper_2308_16395_gb300.profiling LAUNCHES.csv [--skip N] [--per U]

Prints, per kernel, the launches, total and average device time and its share; when the CSV
also holds ``dram__bytes_read.sum`` / ``dram__bytes_write.sum``, the DRAM bytes per launch.
``--skip N`` drops the first N launches (the initial ST-HOSVD); ``--per U`` divides totals by U
(e.g. the number of updates captured) for a per-update column.
"""

from __future__ import annotations

import argparse
import csv
import re
from collections import OrderedDict


def _short(name: str) -> str:
    name = re.sub(r"^void\s+", "", name)
    name = re.sub(r"\(.*$", "", name)
    return name


def read(path: str):
    """List of launches in order: dict(id, kernel, metrics{name: value})."""
    rows = OrderedDict()
    with open(path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        i = int(r["ID"])
        e = rows.setdefault(i, {"id": i, "kernel": _short(r["Kernel Name"]), "grid": r["Grid Size"],
                                "block": r["Block Size"], "metrics": {}})
        v = r["Metric Value"].replace(",", "")
        try:
            val = float(v)
        except ValueError:
            continue
        unit = r.get("Metric Unit", "")
        if unit in ("Kbyte", "KB"):
            val *= 1e3
        elif unit in ("Mbyte", "MB"):
            val *= 1e6
        elif unit in ("Gbyte", "GB"):
            val *= 1e9
        elif unit == "usecond":
            val *= 1e3
        elif unit == "msecond":
            val *= 1e6
        e["metrics"][r["Metric Name"]] = val
    return list(rows.values())


def summarize(launches, per: float = 1.0):
    agg = OrderedDict()
    for L in launches:
        a = agg.setdefault(L["kernel"], {"n": 0, "ns": 0.0, "rd": 0.0, "wr": 0.0})
        m = L["metrics"]
        a["n"] += 1
        a["ns"] += m.get("gpu__time_duration.sum", 0.0)
        a["rd"] += m.get("dram__bytes_read.sum", 0.0)
        a["wr"] += m.get("dram__bytes_write.sum", 0.0)
    total = sum(a["ns"] for a in agg.values()) or 1.0
    out = []
    for k, a in sorted(agg.items(), key=lambda kv: -kv[1]["ns"]):
        out.append(dict(kernel=k, launches=a["n"], total_us=a["ns"] / 1e3, avg_us=a["ns"] / 1e3 / a["n"],
                        share=a["ns"] / total, per_unit_us=a["ns"] / 1e3 / per,
                        dram_mb_per_launch=(a["rd"] + a["wr"]) / a["n"] / 1e6))
    return out, total / 1e3


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("--skip", type=int, default=0)
    ap.add_argument("--per", type=float, default=1.0)
    args = ap.parse_args()
    launches = read(args.csv)[args.skip:]
    rows, total = summarize(launches, args.per)
    has_dram = any("dram__bytes_read.sum" in L["metrics"] for L in launches)
    hdr = f"{'kernel':44s} {'launches':>8s} {'total_us':>10s} {'avg_us':>9s} {'share':>6s} {'per_unit_us':>11s}"
    if has_dram:
        hdr += f" {'dram_MB/launch':>14s}"
    print(hdr)
    for r in rows:
        line = (f"{r['kernel'][:44]:44s} {r['launches']:8d} {r['total_us']:10.1f} {r['avg_us']:9.1f} "
                f"{100 * r['share']:5.1f}% {r['per_unit_us']:11.1f}")
        if has_dram:
            line += f" {r['dram_mb_per_launch']:14.2f}"
        print(line)
    print(f"{'TOTAL':44s} {len(launches):8d} {total:10.1f}")


if __name__ == "__main__":
    main()
