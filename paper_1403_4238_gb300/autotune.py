"""Autotuner for the engine's search batch shape (streaming mode).

A search batch is 32 candidate rows (one per lane) x 16 warps x 4 * rows
candidate columns per lane: rows = 1 gives 64 columns (4 candidates per
lane), rows = 2 gives 128 (8 per lane: fewer loads per evaluation, but
batches twice as large, so fewer of them to spread over a team's CTAs).
Which is faster depends on how many pixels each CTA of a team works on, so
the table is keyed by radius and pixels per CTA, and measured in the batched
form itself: n copies of one synthetic image share the GPU's CTAs (teams of
about SMs / n CTAs), for several n, each shape timed over a bounded number
of iterations.  The table is a text file, one line per bucket:
"radius max_pixels_per_cta rows_per_warp"; the library reads it through
inpaint_options.tuning_file (single images, batches and the server).

    python -m paper_1403_4238_gb300.autotune --out tuning.txt --radii 4,5
"""
from __future__ import annotations

import argparse
import math
import time

from . import api, synth

IMAGE = (480, 320)          # tuning image size
COPIES = (1, 9, 38, 152)    # images per launch (scaled to the SM count)
ITERS = 24                  # iterations timed per run


def _rate(cases, rows, iters, reps=2):
    """Evaluations per second of `iters` iterations of every image of a batch."""
    import torch

    best = math.inf
    evals = 0
    with api.Batch(cases, tile_rows=rows) as b:
        for _ in range(reps):
            b.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.run(max_iters=iters)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        evals = sum(b.result(i)[2] for i in range(len(cases)))
    return evals / best


def tune(radii, iters=ITERS, seed=9, log=print):
    """Returns [(radius, max_pixels_per_cta, rows_per_warp, {rows: evals/s})]."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    W, H = IMAGE
    base = [synth.Case(f"tune{k}", synth.image(W, H, 12, 30.0, seed + k),
                       synth.ellipse_mask(W, H, 3, 0.05, 0.06, seed + 100 + k), 4) for k in range(4)]
    table = []
    for r in radii:
        points = []
        for c in COPIES:
            n = max(1, min(sms, round(c * sms / 152)))
            cases = [(base[i % 4].rgb, base[i % 4].mask, r) for i in range(n)]
            per_cta = W * H * n / sms
            rates = {rows: _rate(cases, rows, iters) for rows in (1, 2)}
            points.append((per_cta, max(rates, key=rates.get), rates))
            log(f"r={r} images={n} ({per_cta:.0f} px per CTA): " +
                ", ".join(f"rows {k}: {v:.3e} evals/s" for k, v in rates.items()))
        points.sort()
        for k, (px, rows, rates) in enumerate(points):
            bound = math.sqrt(px * points[k + 1][0]) if k + 1 < len(points) else float(1 << 40)
            table.append((r, int(bound), rows, rates))
    return table


def write(table, path):
    with open(path, "w") as f:
        for r, max_px, rows, _ in table:
            f.write(f"{r} {max_px} {rows}\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--radii", default="4,5")
    ap.add_argument("--iters", type=int, default=ITERS)
    args = ap.parse_args()
    radii = [int(x) for x in args.radii.split(",")]
    write(tune(radii, args.iters), args.out)


if __name__ == "__main__":
    main()
