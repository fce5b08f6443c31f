"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) per kernel:
launches, total device time, share.  Usage: python -m paper_2011_05427_gb300.profiling FILE.csv"""
import collections
import csv
import sys

SCALE = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}


def summarize(path):
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
    hdr, data = rows[hi], rows[hi + 1:]
    ki, mi = hdr.index("Kernel Name"), hdr.index("Metric Name")
    vi, ui = hdr.index("Metric Value"), hdr.index("Metric Unit")
    tot, cnt = collections.defaultdict(float), collections.Counter()
    for r in data:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        us = float(r[vi].replace(",", "")) * SCALE[r[ui]]
        name = r[ki].split("(")[0].replace("void ", "")
        tot[name] += us
        cnt[name] += 1
    T = sum(tot.values())
    out = [f"| kernel | launches | total ms | share | mean us |", "|---|---|---|---|---|"]
    for k, v in sorted(tot.items(), key=lambda x: -x[1]):
        out.append(f"| `{k}` | {cnt[k]} | {v / 1e3:.2f} | {100 * v / T:.1f}% | {v / cnt[k]:.1f} |")
    out.append(f"| total | {sum(cnt.values())} | {T / 1e3:.2f} | 100% | |")
    return "\n".join(out)


if __name__ == "__main__":
    print(summarize(sys.argv[1]))
