"""Patch-size / search-factor sweep (Sec. 5.3-5.4, Eq. 6-8, Fig. 9).

The paper shrinks the search area with a factor alpha (Eq. 6: the object's
bounding box w x h grown by alpha*w left and right and alpha*h up and down)
and argues with Eq. 8 that a larger patch P only pays off once the search
area is small, because more of the remaining candidates then overlap the
object.  This module measures that trend on the GB300: every Table-3-shaped
synthetic input (synth.TABLE3: WalkingMan, River, DivingMan, Hill sizes and
object shapes) is removed with 9x9, 13x13 and 17x17 patches over a range of
alpha, with the persistent engine, and each removal's time and exact
algorithmic work (valid candidates x known target pixels, summed over the
iterations) are reported next to Eq. 8's estimate.

This library's candidates must lie fully in the known region (the reading of
Eq. 3-4 used throughout), so a candidate that overlaps the object is not
evaluated at all; in Eq. 8's terms that is k = 0.  Eq. 8 is printed for the
paper's k = 0.5 and for k = 0.

    python -m paper_1403_4238_gb300.sweep --out sweep.md
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import api, synth

RADII = (4, 6, 8)                                  # P = 9, 13, 17
ALPHAS = (0.05, 0.1, 0.25, 0.5, 1.0, 2.0, -1.0)    # -1: every interior centre


def eq8_complexity(w: int, h: int, P: int, alpha: float, k: float = 0.5) -> float:
    """Eq. 8: w^2 h^2 ((2a+1)^2 - (1-k)(2(P-1)/w + 1)(2(P-1)/h + 1) - k)."""
    a2 = (2.0 * alpha + 1.0) ** 2
    overlap = (2.0 * (P - 1) / w + 1.0) * (2.0 * (P - 1) / h + 1.0)
    return float(w) ** 2 * float(h) ** 2 * (a2 - (1.0 - k) * overlap - k)


def object_box(mask: np.ndarray) -> tuple[int, int]:
    ys, xs = np.nonzero(mask)
    return int(xs.max() - xs.min() + 1), int(ys.max() - ys.min() + 1)


def run_point(case: synth.Case, alpha: float, reps: int = 3) -> dict:
    """Best-of-reps time of one whole removal (after one untimed run).  A
    search area with no fully known candidate ends the removal with
    NO_SOURCE (status "no_source", no time)."""
    import torch

    with api.Inpainter(case.rgb, case.mask, case.r, alpha=alpha, loop="engine") as ip:
        drgb = torch.from_numpy(case.rgb).cuda()
        dmask = torch.from_numpy(case.mask).cuda()
        best = float("inf")
        n = 0
        for rep in range(reps + 1):
            ip.reset(drgb, dmask)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                rc, n, _ = ip.run()
            except api.InpaintError as e:
                if e.code != -4:
                    raise
                return {"status": "no_source", "rect": list(ip.search_rect())}
            torch.cuda.synchronize()
            if rc != 0:
                raise RuntimeError(f"{case.name} alpha={alpha}: status {rc}")
            if rep:
                best = min(best, time.perf_counter() - t0)
        return {"status": "ok", "iterations": int(n), "evals": int(ip.info()["evals"]), "ms": 1e3 * best,
                "rect": list(ip.search_rect())}


def sweep(names=None, radii=RADII, alphas=ALPHAS, log=print) -> list[dict]:
    rows = []
    for name, W, H, kind, w, h, _, _ in synth.TABLE3:
        if names and name not in names:
            continue
        for r in radii:
            case = synth.table3_case(name, r)
            bw, bh = object_box(case.mask)
            for a in alphas:
                pt = run_point(case, a)
                P = 2 * r + 1
                row = {"image": name, "W": W, "H": H, "object": kind, "w": bw, "h": bh, "P": P, "alpha": a,
                       **pt}
                if a >= 0:
                    row["eq8_k05"] = eq8_complexity(bw, bh, P, a, 0.5)
                    row["eq8_k0"] = eq8_complexity(bw, bh, P, a, 0.0)
                rows.append(row)
                log(json.dumps(row))
    return rows


def table(rows: list[dict]) -> str:
    """Markdown: per image and alpha, time and work of P = 13, 17 relative to
    P = 9 (the normalisation of Fig. 9), and Eq. 8's ratio."""
    out = ["| image | alpha | P=9 ms | P=9 evals | t13/t9 | t17/t9 | evals13/evals9 | evals17/evals9 |"
           " Eq.8 (k=0.5) 13/9 | 17/9 |",
           "|---|---:|---:|---:|---:|---:|---:|---:|---:|---:|"]
    key = {(r["image"], r["alpha"], r["P"]): r for r in rows}
    for name, *_ in synth.TABLE3:
        for a in sorted({r["alpha"] for r in rows if r["image"] == name}, key=lambda v: (v < 0, v)):
            b = key.get((name, a, 9))
            if b is None:
                continue
            ok = lambda c: c is not None and c["status"] == "ok"
            if not ok(b):
                out.append(f"| {name} | {'all' if a < 0 else f'{a:g}'} | no source | | | | | | | |")
                continue
            cells = [name, "all" if a < 0 else f"{a:g}", f"{b['ms']:.2f}", f"{b['evals']:.3g}"]
            for P in (13, 17):
                c = key.get((name, a, P))
                cells.append(f"{c['ms'] / b['ms']:.2f}" if ok(c) else "no source")
            for P in (13, 17):
                c = key.get((name, a, P))
                cells.append(f"{c['evals'] / b['evals']:.2f}" if ok(c) and b["evals"] else "-")
            for P in (13, 17):
                c = key.get((name, a, P))
                if c and a >= 0 and b.get("eq8_k05", 0) > 0:
                    cells.append(f"{c['eq8_k05'] / b['eq8_k05']:.2f}")
                else:
                    cells.append("-")
            out.append("| " + " | ".join(cells) + " |")
    return "\n".join(out) + "\n"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None, help="markdown table file")
    ap.add_argument("--json", default=None, help="raw rows (JSON lines)")
    ap.add_argument("--images", default=None, help="comma-separated subset of " +
                    ",".join(t[0] for t in synth.TABLE3))
    args = ap.parse_args()
    names = args.images.split(",") if args.images else None
    rows = sweep(names)
    if args.json:
        with open(args.json, "w") as f:
            for r in rows:
                f.write(json.dumps(r) + "\n")
    md = table(rows)
    if args.out:
        with open(args.out, "w") as f:
            f.write(md)
    print(md)


if __name__ == "__main__":
    main()
