"""Autotuner for the engine's search batch shape.

The persistent engine stages search batches of 16 warps x rows x 128
candidate columns; rows per warp (1 or 2) trades staging reuse against how
many batches each CTA gets.  For each (patch radius, image-size bucket) this
times a bounded prefix of a synthetic removal with both shapes on the GPU at
hand and writes the winner to a tuning file, one line per bucket:
"radius max_pixels rows_per_warp".  The library reads it through
inpaint_options.tuning_file (single images, batches and the server).

    python -m paper_1403_4238_gb300.autotune --out tuning.txt --radii 4,5
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np

from . import api, synth

# pixel-count buckets and a representative 16:9-ish size for each
BUCKETS = [(160_000, (480, 320)), (400_000, (768, 512)), (1_000_000, (1280, 720)),
           (2_500_000, (1920, 1080)), (1 << 30, (2560, 1440))]


def time_shape(case, rows, iters, reps=3):
    """Evaluations per second of `iters` engine iterations of the case."""
    import torch

    best = math.inf
    evals = 0
    with api.Inpainter(case.rgb, case.mask, case.r, loop="engine", tile_rows=rows) as ip:
        drgb = torch.from_numpy(case.rgb).cuda()
        dmask = torch.from_numpy(case.mask).cuda()
        torch.cuda.synchronize()
        for _ in range(reps):
            ip.reset(drgb, dmask)
            t0 = time.perf_counter()
            ip.run(max_iters=iters)
            dt = time.perf_counter() - t0
            best = min(best, dt)
            evals = ip.info()["evals"]
    return evals / best


def tune(radii, buckets=BUCKETS, iters=48, seed=9, log=print):
    """Returns [(radius, max_pixels, rows_per_warp, {rows: evals/s})]."""
    table = []
    for r in radii:
        for max_px, (W, H) in buckets:
            case = synth.Case(f"tune_{W}x{H}_r{r}", synth.image(W, H, 12, 30.0, seed),
                              synth.ellipse_mask(W, H, 3, 0.05, 0.06, seed + 1), r)
            rates = {rows: time_shape(case, rows, iters) for rows in (1, 2)}
            best = max(rates, key=rates.get)
            table.append((r, max_px, best, rates))
            log(f"r={r} <= {max_px} px ({W}x{H}): " +
                ", ".join(f"rows {k}: {v:.3e} evals/s" for k, v in rates.items()) + f" -> {best}")
    return table


def write(table, path):
    with open(path, "w") as f:
        for r, max_px, rows, _ in table:
            f.write(f"{r} {max_px} {rows}\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--radii", default="4,5")
    ap.add_argument("--iters", type=int, default=48)
    ap.add_argument("--max-pixels", type=int, default=2_500_000)
    args = ap.parse_args()
    radii = [int(x) for x in args.radii.split(",")]
    buckets = [b for b in BUCKETS if b[0] <= args.max_pixels] or BUCKETS[:1]
    write(tune(radii, buckets, args.iters), args.out)


if __name__ == "__main__":
    main()
