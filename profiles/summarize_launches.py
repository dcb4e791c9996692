"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) per kernel:
launches, total device time and share.  Usage: python summarize_launches.py launches.csv"""
import collections
import csv
import re
import sys


def short(name):
    name = re.sub(r"\(.*$", "", name).replace("void ", "").replace("<unnamed>", "")
    return name.split("::")[-1]


def main(path):
    rows = list(csv.reader(open(path)))
    h = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr, data = rows[h], rows[h + 1:]
    ki, vi, ui = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Unit")
    scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in data:
        if len(r) <= vi or not r[vi]:
            continue
        us = float(r[vi].replace(",", "")) * scale.get(r[ui], 1.0)
        agg[short(r[ki])][0] += 1
        agg[short(r[ki])][1] += us
    tot = sum(v[1] for v in agg.values())
    print(f"{'kernel':34s} {'launches':>8s} {'total_us':>12s} {'share':>7s}")
    for k, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"{k:34s} {n:8d} {t:12.1f} {100 * t / tot:6.1f}%")
    print(f"{'(all)':34s} {sum(v[0] for v in agg.values()):8d} {tot:12.1f}")


if __name__ == "__main__":
    main(sys.argv[1])
