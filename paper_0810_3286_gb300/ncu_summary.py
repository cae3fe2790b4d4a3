"""Summarise an Nsight Compute CSV log (``ncu --csv --log-file``) per kernel.

    python -m paper_0810_3286_gb300.ncu_summary launches.csv

For every kernel name: launches, total and average ``gpu__time_duration.sum`` and its share of
the total; when the log also holds ``dram__bytes_read.sum`` / ``dram__bytes_write.sum``, the
average DRAM bytes per launch.  ncu serialises launches and flushes caches between them, so
absolute times are cold-cache figures: compare shares, not absolutes.
"""
from __future__ import annotations

import collections
import csv
import sys

_TIME_SCALE = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3, "s": 1e6,
               "second": 1e6}
_BYTE_SCALE = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}


def summarize(path):
    rows = list(csv.reader(open(path, newline="")))
    hdr = None
    agg = collections.OrderedDict()
    for r in rows:
        if r and r[0] == "ID":
            hdr = r
            continue
        if not hdr or len(r) != len(hdr):
            continue
        d = dict(zip(hdr, r))
        name = d["Kernel Name"].split("(")[0].replace("void ", "").strip()
        key = (name, d["ID"])
        rec = agg.setdefault(key, {"time_us": None, "dram": 0.0, "has_dram": False})
        metric, unit = d["Metric Name"], d["Metric Unit"]
        value = float(d["Metric Value"].replace(",", ""))
        if metric == "gpu__time_duration.sum":
            rec["time_us"] = value * _TIME_SCALE.get(unit, 1.0)
        elif metric in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            rec["dram"] += value * _BYTE_SCALE.get(unit, 1.0)
            rec["has_dram"] = True
    per = collections.defaultdict(lambda: {"n": 0, "t": 0.0, "dram": 0.0, "nd": 0})
    for (name, _), rec in agg.items():
        p = per[name]
        p["n"] += 1
        if rec["time_us"] is not None:
            p["t"] += rec["time_us"]
        if rec["has_dram"]:
            p["dram"] += rec["dram"]
            p["nd"] += 1
    return per


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    per = summarize(argv[0])
    tot = sum(p["t"] for p in per.values()) or 1.0
    print("total device time %.1f us over %d launches" % (tot, sum(p["n"] for p in per.values())))
    print("%-40s %7s %12s %10s %7s %14s" % ("kernel", "launches", "total_us", "avg_us", "share", "dram_B/launch"))
    for name, p in sorted(per.items(), key=lambda kv: -kv[1]["t"]):
        dram = "%14.0f" % (p["dram"] / p["nd"]) if p["nd"] else "%14s" % "-"
        print("%-40s %7d %12.1f %10.2f %7.3f %s" % (name[:40], p["n"], p["t"], p["t"] / max(p["n"], 1),
                                                 p["t"] / tot, dram))


if __name__ == "__main__":
    main()
