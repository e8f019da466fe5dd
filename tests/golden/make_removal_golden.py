"""Writes the stored expected results of whole removals at full size.

Every value written here comes from the CPU oracle (``oracle.run``, the
restatement of Sec. 3, Eq. 1-4) on the seeded synthetic inputs of
``paper_1403_4238_gb300.synth``; nothing is taken from the CUDA library.
The oracle needs about 15-20 minutes of one core for the 1920x1080 removal,
so the results are stored once and the GPU tests compare against them:

  removals.json          one entry per removal: generator call, sizes, the
                         SHA-256 of the input bytes (so a test can tell a
                         changed input from a wrong result), status,
                         iterations, exact evaluation count, SHA-256 of the
                         final RGB and of the trace
  trace_<name>.txt       the full per-iteration trace of the removals whose
                         trace is kept (one line per iteration:
                         px py qx qy ssd priority-bits confidence-bits filled
                         remaining n_known n_cand; the two doubles as 16 hex
                         digits of their IEEE bits)

Run from the repository root:  python tests/golden/make_removal_golden.py
(options: --only NAME[,NAME...] to recompute some entries, -j N processes).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# (entry name, generator expression evaluated in synth's namespace, keep full trace)
BATCH_PICK = (0, 3, 12, 47, 53, 58)     # of synth.batch_cases(64): sizes 283x484 ... 1221x703, r 4 and 5
SERVE_PICK = (1, 4, 12, 14, 26)          # of synth.serving_trace(2000): 385x720 ... 1605x261, r 4 and 5
CASES = [("hd_blob", "hd_blob()", True)]
CASES += [(f"batch64_{i}", f"batch_cases(64)[{i}]", False) for i in BATCH_PICK]
CASES += [(f"serve2000_{i}", f"serving_case(*serving_trace(2000)[{i}][1:])", False) for i in SERVE_PICK]

TRACE_FIELDS = ("px", "py", "qx", "qy", "ssd", "priority", "confidence", "filled", "remaining",
                "n_known", "n_cand")


def make_case(expr: str):
    from paper_1403_4238_gb300 import synth

    return eval(expr, {k: getattr(synth, k) for k in dir(synth) if not k.startswith("_")})


def sha(a) -> str:
    import numpy as np

    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def trace_lines(tr) -> list[str]:
    import numpy as np

    out = []
    for rec in tr:
        vals = []
        for f in TRACE_FIELDS:
            if f in ("priority", "confidence"):
                vals.append("%016x" % int(np.float64(rec[f]).view(np.uint64)))
            else:
                vals.append(str(int(rec[f])))
        out.append(" ".join(vals))
    return out


def compute(item):
    name, expr, keep = item
    import oracle

    case = make_case(expr)
    t0 = time.time()
    res = oracle.run(case.rgb, case.mask, case.r)
    dt = time.time() - t0
    lines = trace_lines(res.trace)
    entry = {
        "name": name,
        "generator": f"synth.{expr}",
        "case": case.name,
        "W": case.W,
        "H": case.H,
        "r": case.r,
        "rgb_sha256": sha(case.rgb),
        "mask_sha256": sha(case.mask),
        "unknown": int((case.mask != 0).sum()),
        "status": int(res.status),
        "iters": int(res.iters),
        "evals": int(res.evals),
        "result_sha256": sha(res.rgb),
        "trace_sha256": hashlib.sha256("\n".join(lines).encode()).hexdigest(),
        "trace_file": f"trace_{name}.txt" if keep else None,
        "oracle_seconds": round(dt, 1),
    }
    if keep:
        with open(os.path.join(HERE, entry["trace_file"]), "w") as f:
            f.write("# " + " ".join(TRACE_FIELDS) + "\n")
            f.write("\n".join(lines) + "\n")
    return entry


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default="")
    ap.add_argument("-j", type=int, default=max(1, min(len(CASES), os.cpu_count() or 1)))
    args = ap.parse_args()
    import oracle

    oracle.build()
    todo = CASES
    if args.only:
        keep = set(args.only.split(","))
        todo = [c for c in CASES if c[0] in keep]
    path = os.path.join(HERE, "removals.json")
    old = {}
    if os.path.exists(path):
        with open(path) as f:
            old = {e["name"]: e for e in json.load(f)["removals"]}
    # longest first, so the 1920x1080 removal starts at once
    with mp.get_context("spawn").Pool(args.j) as pool:
        for e in pool.imap_unordered(compute, todo):
            old[e["name"]] = e
            print(f"{e['name']}: {e['W']}x{e['H']} r={e['r']} iters={e['iters']} evals={e['evals']} "
                  f"({e['oracle_seconds']} s)", flush=True)
    order = [c[0] for c in CASES]
    doc = {
        "_about": ("Whole removals computed by the CPU oracle (Sec. 3, Eq. 1-4) on seeded synthetic "
                   "inputs; written by tests/golden/make_removal_golden.py, which calls only oracle/ "
                   "and the input generator."),
        "removals": [old[n] for n in order if n in old],
    }
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
