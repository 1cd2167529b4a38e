"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) per kernel.

Usage: python -m paper_2506_00976_gb300.ncu_summary launches.csv [skip_first_n]
Prints launches, total device time and share per kernel (cold-cache,
serialised times: compare shares, not absolutes).
"""
import collections
import csv
import sys

SCALE = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3,
         "s": 1e6, "second": 1e6}


def main(path, skip=0):
    rows = list(csv.reader(open(path)))
    hi = [i for i, r in enumerate(rows) if r and r[0] == "ID"][0]
    h, data = rows[hi], rows[hi + 1:]
    ki, vi, ui = h.index("Kernel Name"), h.index("Metric Value"), h.index("Metric Unit")
    agg = collections.OrderedDict()
    for r in data[skip:]:
        name = r[ki].split("(")[0].replace("void ", "")
        v = float(r[vi].replace(",", "")) * SCALE[r[ui]]
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += v
    tot = sum(a[1] for a in agg.values())
    print(f"{'kernel':60s} {'launches':>8s} {'total_us':>12s} {'share':>7s}")
    for k, (n, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        print(f"{k[:60]:60s} {n:8d} {t:12.1f} {100 * t / tot:6.1f}%")
    print(f"{'total':60s} {sum(a[0] for a in agg.values()):8d} {tot:12.1f}")


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else 0)
