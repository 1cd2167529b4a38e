"""Summaries of ncu CSV output for the profile notes.

  python -m paper_2506_00976_gb300.ncu_summary launches.csv [skip_first_n]
      per kernel: launches, total device time and share, from a launch list
      taken with --metrics gpu__time_duration.sum --csv (cold-cache,
      serialised times: compare shares, not absolutes);
  python -m paper_2506_00976_gb300.ncu_summary metrics counters.csv
      every metric of every captured launch, one line each;
  python -m paper_2506_00976_gb300.ncu_summary traffic counters.csv REGEX SCALE OUT.json
      DRAM bytes (read + write) of the first launch whose kernel name matches
      REGEX, times SCALE (launch units of the full workload / those of the
      captured case), written with the SHA-256 of csrc/kernels.cu so that a
      reader can tell when the kernel has changed since.
"""
import collections
import csv
import hashlib
import json
import os
import re
import sys

SCALE = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3,
         "s": 1e6, "second": 1e6}
BYTES = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
HERE = os.path.dirname(os.path.abspath(__file__))


def _rows(path):
    rows = list(csv.reader(open(path)))
    hi = [i for i, r in enumerate(rows) if r and r[0] == "ID"][0]
    h = rows[hi]
    return [dict(zip(h, r)) for r in rows[hi + 1:]]


def launches(path, skip=0):
    agg = collections.OrderedDict()
    for r in _rows(path)[skip:]:
        name = r["Kernel Name"].split("(")[0].replace("void ", "")
        v = float(r["Metric Value"].replace(",", "")) * SCALE[r["Metric Unit"]]
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += v
    tot = sum(a[1] for a in agg.values())
    print(f"{'kernel':60s} {'launches':>8s} {'total_us':>12s} {'share':>7s}")
    for k, (n, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        print(f"{k[:60]:60s} {n:8d} {t:12.1f} {100 * t / tot:6.1f}%")
    print(f"{'total':60s} {sum(a[0] for a in agg.values()):8d} {tot:12.1f}")


def metrics(path):
    for r in _rows(path):
        print(f"{r['ID']:>3s} {r['Kernel Name'].split('(')[0][:48]:48s} {r['Metric Name']:70s} "
              f"{r['Metric Value']} {r.get('Metric Unit', '')}")


def traffic(path, regex, scale, out):
    by_id = collections.OrderedDict()
    for r in _rows(path):
        if re.search(regex, r["Kernel Name"]):
            by_id.setdefault(r["ID"], []).append(r)
    if not by_id:
        raise SystemExit(f"no launch matches {regex}")
    rec = next(iter(by_id.values()))
    total = 0.0
    for r in rec:
        if r["Metric Name"] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            total += float(r["Metric Value"].replace(",", "")) * BYTES.get(r["Metric Unit"], 1.0)
    with open(os.path.join(HERE, "csrc", "kernels.cu"), "rb") as fh:
        sha = hashlib.sha256(fh.read()).hexdigest()
    doc = {"kernel": rec[0]["Kernel Name"].split("(")[0].replace("void ", ""),
           "dram_bytes_captured_launch": total, "scale": scale,
           "dram_bytes_per_launch": total * scale, "kernel_source_sha256": sha,
           "source": os.path.basename(path)}
    with open(out, "w") as fh:
        json.dump(doc, fh, indent=1)
    print(json.dumps(doc))


if __name__ == "__main__":
    if sys.argv[1] == "metrics":
        metrics(sys.argv[2])
    elif sys.argv[1] == "traffic":
        traffic(sys.argv[2], sys.argv[3], float(sys.argv[4]), sys.argv[5])
    else:
        launches(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else 0)
