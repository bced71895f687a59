"""Summaries of ncu CSV logs (``ncu --csv --log-file F --metrics ...``).

    python -m paper_1503_04359_b300.ncu_summary F.csv              # launches per kernel
    python -m paper_1503_04359_b300.ncu_summary F.csv --bu-levels  # DRAM bytes per bottom-up level

The launch table lists, per kernel, its launches, total gpu__time_duration
and share of the captured total. The bottom-up view groups the captured
launches into bottom-up levels (one k_bu launch in search mode plus the
k_bu_long launch that follows it; the k_bu launches of bitmap-output and
mixed levels, which are followed by a recovery-mode k_bu, are left out) and
reports DRAM bytes read + written per level, the figure bench.py compares
with the algorithmic bytes.
"""
from __future__ import annotations

import argparse
import collections
import csv
import io
import json
import re
import sys

_UNIT = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12,
         "nsecond": 1e-3, "usecond": 1.0, "msecond": 1e3, "second": 1e6, "ns": 1e-3, "us": 1.0, "ms": 1e3, "s": 1e6}


def read_launches(path: str) -> list[dict]:
    """[{id, name, metrics{name: value}}] in launch order; bytes in bytes, times in us."""
    with open(path) as f:
        text = f.read()
    lines = text.splitlines()
    start = next(i for i, ln in enumerate(lines) if ln.startswith('"ID"'))
    rows = list(csv.reader(io.StringIO("\n".join(lines[start:]))))
    h = rows[0]
    ix = {k: h.index(k) for k in ("ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value")}
    out = collections.OrderedDict()
    for r in rows[1:]:
        if len(r) < len(h):
            continue
        key = int(r[ix["ID"]])
        rec = out.setdefault(key, {"id": key, "name": r[ix["Kernel Name"]], "metrics": {}})
        v = float(r[ix["Metric Value"]].replace(",", ""))
        rec["metrics"][r[ix["Metric Name"]]] = v * _UNIT.get(r[ix["Metric Unit"]], 1.0)
    return list(out.values())


def short_name(name: str) -> str:
    s = name
    for p in ("void ", "(anonymous namespace)::", "<unnamed>::", "unnamed>::", "dobfs::"):
        s = s.replace(p, "")
    return s.split("(")[0].strip()


def launch_table(launches: list[dict]) -> list[tuple[str, int, float, float]]:
    agg = collections.defaultdict(lambda: [0, 0.0])
    for L in launches:
        a = agg[short_name(L["name"])]
        a[0] += 1
        a[1] += L["metrics"].get("gpu__time_duration.sum", 0.0)
    total = sum(a[1] for a in agg.values()) or 1.0
    return sorted(((k, a[0], a[1], a[1] / total) for k, a in agg.items()), key=lambda x: -x[2])


def bu_levels(launches: list[dict]) -> list[dict]:
    """Bottom-up levels: a k_bu<..., 0> (search) launch directly followed by
    k_bu_long. In a mixed level the search launch is followed by the parent
    recovery (k_bu<..., 1>) instead; such launches are not bottom-up levels."""
    levels = []
    pending = None
    for L in launches:
        n = short_name(L["name"])
        m = L["metrics"]
        dram = m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0)
        t = m.get("gpu__time_duration.sum", 0.0)
        if re.match(r"k_bu<[^,]+,\s*(0|false)>", n):
            pending = {"bytes": dram, "us": t, "launches": 1}
        elif n.startswith("k_bu_long") and pending is not None:
            pending["bytes"] += dram
            pending["us"] += t
            pending["launches"] += 1
            levels.append(pending)
            pending = None
        else:
            pending = None
    return levels


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("--bu-levels", action="store_true")
    args = ap.parse_args(argv)
    launches = read_launches(args.csv)
    if args.bu_levels:
        lv = bu_levels(launches)
        for i, x in enumerate(lv):
            print("level %2d: %10.1f us  %12.0f bytes  %7.0f GB/s" % (i, x["us"], x["bytes"],
                                                                       x["bytes"] / (x["us"] * 1e3) if x["us"] else 0))
        if lv:
            tot_b = sum(x["bytes"] for x in lv)
            print(json.dumps({"bu_levels": len(lv), "bytes_per_level": tot_b / len(lv),
                              "us_per_level": sum(x["us"] for x in lv) / len(lv)}))
        return 0
    total = sum(x[2] for x in launch_table(launches))
    print("%-40s %9s %14s %8s" % ("kernel", "launches", "total us", "share"))
    for k, c, t, sh in launch_table(launches):
        print("%-40s %9d %14.1f %7.2f%%" % (k[:40], c, t, 100 * sh))
    print("%-40s %9d %14.1f" % ("all captured", len(launches), total))
    return 0


if __name__ == "__main__":
    sys.exit(main())
