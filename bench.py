"""Benchmark of exemplar-based object removal on GB300 (one JSON line on rank 0).

Workload (one "step"): one whole object removal of a 512x384 synthetic
image with a 3-ellipse mask covering 7.5-8.5 % of the pixels, 9x9 patches
(radius 4), exhaustive search -- initialisation from inputs already in HBM,
then the device-driven fill loop to an empty target region.  The metric is
candidate-pixel SSD evaluations per second (one evaluation = one valid
candidate x one known target pixel, all three channels), counted exactly by
the device loop; ms per removal is reported beside it.

--impl reference times the CPU oracle (the plain single-threaded C
restatement) on a bounded prefix of the same removal.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "candidate-pixel SSD evals/s (whole removal, 512x384, 9x9 patch, exhaustive search)"
UNIT = "evals/s"
WORKLOAD = "512x384 RGB, 3-ellipse mask 7.5-8.5%, r=4 (9x9), exhaustive search, plain form"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-iters", type=int, default=150,
                    help="oracle iterations per CPU sample (bounded prefix of the removal)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--json-out", default=None)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload():
    from paper_1403_4238_gb300 import synth

    return synth.walkingman_like()


def cpu_sample(case, iters):
    """Oracle on a bounded prefix of the removal: (evals/s, seconds, evals)."""
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    res = oracle.run(case.rgb, case.mask, case.r, max_iters=iters)
    dt = time.perf_counter() - t0
    return res.evals / dt, dt, res.evals, res.iters


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    case = workload()
    vals = []
    for i in range(args.warmup + args.steps):
        v, dt, ev, it = cpu_sample(case, max(1, args.cpu_iters // 5))
        if i >= args.warmup:
            vals.append((v, dt, ev, it))
    tot_ev = sum(x[2] for x in vals)
    tot_t = sum(x[1] for x in vals)
    value = tot_ev / tot_t
    sample = f"first {vals[0][3]} of the removal's iterations per step (oracle, 1 thread)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(vals),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/int32/f64",
        "data": "synthetic", "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def l2_flush(buf):
    buf.add_(1)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_1403_4238_gb300 import api

    case = workload()
    H, W = case.mask.shape
    dev_rgb = torch.from_numpy(case.rgb).cuda()
    dev_mask = torch.from_numpy(case.mask).cuda()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # 512 MB > L2
    ip = api.Inpainter(case.rgb, case.mask, case.r)
    stream = ip.stream
    torch.cuda.synchronize()

    def one_step():
        ip.reset(dev_rgb, dev_mask)
        rc, n, _ = ip.run()
        assert rc == 0, rc
        return n

    for _ in range(max(args.warmup, 3)):
        one_step()
    info = ip.info()
    evals_per_removal = info["evals"]
    iters = None

    # timed region: K removals, L2 flushed between them (outside the events)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            l2_flush(flush)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            iters = one_step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    total_ms = sum(ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = evals_per_removal * args.steps * world / (total_ms / 1e3)

    # end to end through the public API with host buffers (pinned), per removal
    pin_rgb = torch.from_numpy(case.rgb).pin_memory()
    pin_mask = torch.from_numpy(case.mask).pin_memory()
    out = np.zeros((H, W, 3), np.uint8)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ip.reset(pin_rgb.numpy(), pin_mask.numpy())
        ip.run()
        out = ip.result()
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_ms.append(1e3 * (t1 - t0))
    e2e_value = evals_per_removal * len(e2e_ms) * world / (sum(e2e_ms) / 1e3)
    launches_per_removal = 8 + 2 * iters

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8/int32/f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "W": W, "H": H, "r": case.r, "mask_px": int(case.mask.sum()),
                       "iterations": iters, "evals_per_removal": evals_per_removal,
                       "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas x{world}"},
            "ms_per_removal": total_ms / args.steps,
            "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_removal": statistics.mean(e2e_ms),
                    "h2d_bytes_per_step": 4 * W * H, "d2h_bytes_per_step": 3 * W * H},
            "gpu_launches": launches_per_removal * args.steps,
            "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline and world == 1:
            v, dt, ev, it = cpu_sample(case, args.cpu_iters)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"first {it} of {iters} iterations of the same removal "
                                              f"({ev} evals, {dt:.1f} s)"}
        print(json.dumps(line), flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                json.dump(line, f, indent=1)
    ip.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
