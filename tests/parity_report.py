"""Tabulate the errors that the GPU parity tests measured against the FP64
oracle (and against central differences, brute force or the unbatched path,
where that is the reference).

    SCGR_PARITY_LOG=/tmp/parity.jsonl python -m pytest tests -m gpu -q
    python tests/parity_report.py /tmp/parity.jsonl

One row per measured quantity: how many checks measured it, the worst value
seen, its tolerance and the ratio of the two, and the test that saw the
worst value.  Not a test module (pytest does not collect it)."""
import json
import sys
from collections import OrderedDict


def main(path):
    rows = OrderedDict()
    for line in open(path):
        line = line.strip()
        if not line:
            continue
        r = json.loads(line)
        key = r["quantity"]
        cur = rows.get(key)
        if cur is None:
            rows[key] = {"n": 1, "worst": r["value"], "tol": r["tol"], "test": r["test"]}
        else:
            cur["n"] += 1
            if r["value"] > cur["worst"]:
                cur.update(worst=r["value"], test=r["test"])
            cur["tol"] = max(cur["tol"], r["tol"])
    print("| result | checks | worst measured | tolerance | worst / tolerance | worst in |")
    print("|---|---:|---:|---:|---:|---|")
    for key, v in rows.items():
        ratio = "-" if v["tol"] == 0 else f"{v['worst'] / v['tol']:.3g}"
        worst = f"{v['worst']:.3g}" if v["worst"] != int(v["worst"]) or abs(v["worst"]) < 1e-3 else f"{int(v['worst'])}"
        tol = f"{v['tol']:.3g}" if v["tol"] != 0 else "0"
        print(f"| {key} | {v['n']} | {worst} | {tol} | {ratio} | `{v['test'].split('::', 1)[-1]}` |")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "parity.jsonl")
