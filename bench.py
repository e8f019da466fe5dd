"""Benchmark of exemplar-based object removal on GB300 (one JSON line on rank 0).

Headline workload (one "step"): one whole object removal of a 512x384
synthetic image with a 3-ellipse mask covering 7.5-8.5 % of the pixels, 9x9
patches (radius 4), exhaustive search -- initialisation from inputs already
in HBM, then the device-driven fill loop (persistent engine, plain CUDA-core
search) to an empty target region.  The metric is candidate-pixel SSD
evaluations per second (one evaluation = one valid candidate x one known
target pixel, all three channels), counted exactly by the device loop; ms
per removal is reported beside it.

Beside the headline the same JSON line carries the other forms, each at
outputs identical to the plain form's:
  tc       the exact tensor-core search form on the same removal and on a
           1920x1080 removal with 13x13 patches (whole removal and the search
           kernel alone), as speedups over the plain form;
  batched  64 images of uneven sizes in one persistent launch (CUDA graph),
           images/s and the speedup over removing them one after another;
  serving  Poisson arrivals (200 req/s) through the continuous-batching
           server under a 40 GB HBM budget: p50/p99 latency and images/s.

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
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-iters", type=int, default=150,
                    help="oracle iterations per CPU sample (bounded prefix of the removal)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-extras", action="store_true",
                    help="headline only: no tensor-core, batched or serving sections")
    ap.add_argument("--serve-requests", type=int, default=300)
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
        self.first = 0

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
        # nvidia-smi takes a moment to start: wait (bounded) for its first
        # sample so that the samples span the whole timed region
        t0 = time.monotonic()
        while not self.lines and self.proc.poll() is None and time.monotonic() - t0 < 3.0:
            time.sleep(0.01)
        self.first = len(self.lines)  # samples taken before the timed region
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
        # the last sample before the region stands for its start
        for ln in self.lines[max(0, self.first - 1):]:
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


# Plain-search roofline: one evaluation is one byte-SIMD absolute difference
# (vabsdiffu4) plus one 4-way byte dot product (dp4a); each is a half-rate
# integer instruction (16 lanes per clock per SM sub-partition, 4 per SM) and
# the two go to different pipes, so an SM completes at most 64 evaluations
# per clock.
EVALS_PER_CLK_SM = 64

# DRAM bytes (read + write) of one k_engine launch on the headline workload,
# from an ncu capture of the current kernel (dram__bytes_read.sum +
# dram__bytes_write.sum: 2.350 MB + 2.198 MB); None once the kernel changes.
ENGINE_TRAFFIC_BYTES = 4547840


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def launches_init(H):
    # ctrl init, unpack, SAT rows / column chunks / chunk prefix (/ apply),
    # validity counts, priorities, two tile levels, first selection
    return 10 + (1 if H > 64 else 0)


def time_removals(ip, drgb, dmask, steps, warmup, flush):
    """ms per removal (reset from device inputs + run) and ms of run() alone."""
    import torch

    for _ in range(warmup):
        ip.reset(drgb, dmask)
        ip.run()
    tot, run = [], []
    for _ in range(steps):
        l2_flush(flush)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(ip.stream)
        ip.reset(drgb, dmask)
        ev[1].record(ip.stream)
        rc, n, _ = ip.run()
        ev[2].record(ip.stream)
        ev[2].synchronize()
        assert rc == 0, rc
        tot.append(ev[0].elapsed_time(ev[2]))
        run.append(ev[1].elapsed_time(ev[2]))
    return statistics.mean(tot), statistics.mean(run), n


def tc_section(api, case, flush, steps, peaks, plain_ms=None, plain_out=None):
    """Tensor-core form vs the plain form on one removal: whole removal and
    the search kernel alone (initial target), outputs compared."""
    import torch

    drgb = torch.from_numpy(case.rgb).cuda()
    dmask = torch.from_numpy(case.mask).cuda()
    out = {"workload": f"{case.mask.shape[1]}x{case.mask.shape[0]} r={case.r}"}
    res = {}
    for form, loop in (("plain", "auto"), ("plain", "graph"), ("tc", "graph")):
        if form == "plain" and loop == "auto" and plain_ms is not None:
            res[(form, loop)] = (plain_ms, plain_out)
            continue
        with api.Inpainter(case.rgb, case.mask, case.r, form=form, loop=loop) as ip:
            ms, _, n = time_removals(ip, drgb, dmask, steps, 1, flush)
            res[(form, loop)] = (ms, ip.result())
            out["iterations"] = n
    with api.Inpainter(case.rgb, case.mask, case.r, loop="graph") as ip:
        s_plain, k_plain, ev = ip.time_search("plain", 20)
        s_tc, k_tc, _ = ip.time_search("tc", 20)
    base_ms, base_img = res[("plain", "auto")]
    out.update({
        "ms_per_removal": {"plain_engine": base_ms, "plain_graph": res[("plain", "graph")][0],
                           "tc_graph": res[("tc", "graph")][0]},
        "speedup_vs_plain": base_ms / res[("tc", "graph")][0],
        "speedup_vs_plain_same_loop": res[("plain", "graph")][0] / res[("tc", "graph")][0],
        "identical_outputs": bool(np.array_equal(res[("tc", "graph")][1], base_img)
                                  and np.array_equal(res[("plain", "graph")][1], base_img)),
        "search_kernel_us": {"plain": 1e3 * s_plain, "tc": 1e3 * s_tc},
        "search_speedup": s_plain / s_tc,
        "search_same_key": bool(k_plain == k_tc),
        "search_evals": ev,
    })
    # algorithmic tensor work of one search: per evaluation 3 cross-term and
    # 2 square-term multiply-adds (BF16 in, FP32 accumulate)
    peak = peaks.get("bf16_tflops")
    ach = ev * 5 * 2 / (s_tc * 1e-3) / 1e12
    out["roofline"] = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                       "frac": (ach / peak) if peak else None, "traffic": None,
                       "peak_source": "measured bf16 burst" if peak else None}
    return out


# Initialisation (row a1), algorithmic bytes per pixel: the RGB + mask input
# read (4) and the state written: RGBA word 4, mask 1, grey 1, confidence 8,
# validity count 4, priority key 8, confidence of the last evaluation 8.
INIT_BYTES_PER_PX = 4 + 4 + 1 + 1 + 8 + 4 + 8 + 8


def init_section(api, cases, flush, reps, hbm_gbs):
    """Initialisation from device inputs (inpaint_reset: unpack, integral
    image, validity counts, priorities, tiles, first selection) against the
    HBM bandwidth its algorithmic bytes would need."""
    import torch

    out = []
    for case in cases:
        drgb = torch.from_numpy(case.rgb).cuda()
        dmask = torch.from_numpy(case.mask).cuda()
        with api.Inpainter(case.rgb, case.mask, case.r, loop="engine") as ip:
            ip.reset(drgb, dmask)
            ts = []
            for _ in range(reps):
                l2_flush(flush)
                torch.cuda.synchronize()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                ev[0].record(ip.stream)
                ip.reset(drgb, dmask)
                ev[1].record(ip.stream)
                ev[1].synchronize()
                ts.append(ev[0].elapsed_time(ev[1]))
        H, W = case.mask.shape
        ms = statistics.mean(ts)
        gbs = INIT_BYTES_PER_PX * W * H / (ms * 1e-3) / 1e9
        out.append({"workload": f"{W}x{H}", "us": 1e3 * ms, "bytes": INIT_BYTES_PER_PX * W * H,
                    "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s",
                                 "frac": gbs / hbm_gbs if hbm_gbs else None,
                                 "note": "a chain of small kernels: latency-bound at these sizes"}})
    return out


def overlap_section(api, case, flush, steps, peak_evals):
    """Partial-overlap search variant (Algorithm 1, Sec. 5.4) against the full
    search, both in the graph loop: whole removal, exact work, and the search
    kernel alone for the initial target."""
    import torch

    drgb = torch.from_numpy(case.rgb).cuda()
    dmask = torch.from_numpy(case.mask).cuda()
    out = {"workload": f"{case.mask.shape[1]}x{case.mask.shape[0]} r={case.r}, graph loop"}
    for name, ov in (("full", False), ("overlap", True)):
        with api.Inpainter(case.rgb, case.mask, case.r, loop="graph", overlap=ov) as ip:
            ms, _, n = time_removals(ip, drgb, dmask, steps, 1, flush)
            ev = ip.info()["evals"]
            ip.reset(drgb, dmask)
            s_ms, _, s_ev = ip.time_search("plain", 20)
        out[name] = {"ms_per_removal": ms, "iterations": n, "evals_per_removal": ev,
                     "evals_per_s": ev / (ms * 1e-3), "search_kernel_us": 1e3 * s_ms, "search_evals": s_ev,
                     "search_evals_per_s": s_ev / (s_ms * 1e-3)}
    ach = out["overlap"]["search_evals_per_s"]
    # the variant spends 5 instructions per evaluation (4 on the ALU pipe:
    # absolute difference, two shifts, mask) instead of 2: the 2-instruction
    # peak is an upper bound it cannot reach
    out["roofline"] = {"bound": "alu", "achieved": ach, "peak": peak_evals, "unit": "evals/s",
                       "frac": ach / peak_evals, "kernel": "k_search_overlap (one search)"}
    return out


def batch_section(api, flush, steps, log):
    import torch

    from paper_1403_4238_gb300 import autotune, synth

    cases = synth.batch_cases(64)
    import tempfile

    tf = os.path.join(tempfile.mkdtemp(prefix="inpaint_tune_"), "tuning_bench.txt")
    table = autotune.tune((4, 5), log=lambda *a: None)
    autotune.write(table, tf)
    items = [(c.rgb, c.mask, c.r) for c in cases]
    with api.Batch(items, tuning_file=tf) as b:
        b.reset()
        b.run()
        ms = []
        for _ in range(steps):
            l2_flush(flush)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(b.stream)
            b.reset()
            st = b.run()
            e1.record(b.stream)
            e1.synchronize()
            assert all(x in (0, 1) for x in st), st
            ms.append(e0.elapsed_time(e1))
        outs = [b.result(i)[0] for i in range(len(cases))]
        plan = b.plan()
    # the same images one after another (plain form, persistent engine)
    seq_ms, same = 0.0, True
    for c, o in zip(cases, outs):
        drgb, dmask = torch.from_numpy(c.rgb).cuda(), torch.from_numpy(c.mask).cuda()
        with api.Inpainter(c.rgb, c.mask, c.r, tuning_file=tf) as ip:
            t, _, _ = time_removals(ip, drgb, dmask, 1, 1, flush)
            seq_ms += t
            same = same and np.array_equal(ip.result(), o)
    bms = statistics.mean(ms)
    return {"images": len(cases), "images_per_s": len(cases) / (bms / 1e3), "ms_per_batch": bms,
            "ms_sequential": seq_ms, "speedup_vs_sequential": seq_ms / bms, "identical_outputs": bool(same),
            "teams": plan["teams"], "grid": plan["grid"], "graph": "reset and run captured in CUDA graphs",
            "autotune": [{"r": r, "max_pixels_per_cta": mp, "rows": rows} for r, mp, rows, _ in table]}


def serving_section(api, n_req, pool_n=24):
    import torch

    from paper_1403_4238_gb300 import synth

    trace = synth.serving_trace(n_req)
    pool = [synth.serving_case(*t[1:]) for t in trace[:pool_n]]
    alone = []
    for c in pool:
        with api.Inpainter(c.rgb, c.mask, c.r) as ip:
            ip.run()
            alone.append(ip.result())
    with api.Server(hbm_budget_bytes=40 << 30, max_slots=256, iters_per_tick=0) as srv:
        ids = []
        t0 = time.perf_counter()
        for i, t in enumerate(trace):
            now = time.perf_counter() - t0
            if t[0] > now:
                time.sleep(t[0] - now)
            c = pool[i % pool_n]
            ids.append((srv.submit(c.rgb, c.mask, c.r), i % pool_n))
        srv.wait_idle(600)
        lat, done, first, same, ok = [], [], None, True, 0
        for rid, k in ids:
            out, info = srv.poll(rid)
            ok += info["status"] == 0
            lat.append(1e3 * (info["t_done"] - info["t_submit"]))
            done.append(info["t_done"])
            first = info["t_submit"] if first is None else min(first, info["t_submit"])
            same = same and np.array_equal(out, alone[k])
        st = srv.stats()
    span = max(done) - first
    return {"requests": n_req, "rate_req_s": 200.0, "completed_ok": ok, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "images_per_s": n_req / span,
            "identical_to_alone": bool(same), "hbm_budget_gb": 40, "ticks": st["ticks"],
            "pool": f"{pool_n} distinct seeded cases from the trace, request i uses case i mod {pool_n}"}


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

    peaks = measured_peaks()
    case = workload()
    H, W = case.mask.shape
    dev_rgb = torch.from_numpy(case.rgb).cuda()
    dev_mask = torch.from_numpy(case.mask).cuda()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # 512 MB > L2
    ip = api.Inpainter(case.rgb, case.mask, case.r)
    stream = ip.stream
    torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        ip.reset(dev_rgb, dev_mask)
        assert ip.run()[0] == 0
    evals_per_removal = ip.info()["evals"]

    # timed region: K removals, L2 flushed between them (outside the events)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms, run_ms = [], []
    iters = 0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            l2_flush(flush)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            ip.reset(dev_rgb, dev_mask)
            ev[1].record(stream)
            rc, iters, _ = ip.run()
            ev[2].record(stream)
            ev[2].synchronize()
            assert rc == 0, rc
            ms.append(ev[0].elapsed_time(ev[2]))
            run_ms.append(ev[1].elapsed_time(ev[2]))
    torch.cuda.synchronize()
    from paper_1403_4238_gb300.dist import max_over_ranks

    total_ms = max_over_ranks(sum(ms))
    value = evals_per_removal * args.steps * world / (total_ms / 1e3)
    plain_out = ip.result()
    search_ns, update_ns, timed_iters = ip.loop_timing()

    # end to end through the public API with host buffers (pinned), per removal
    pin_rgb = torch.from_numpy(case.rgb).pin_memory()
    pin_mask = torch.from_numpy(case.mask).pin_memory()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ip.reset(pin_rgb.numpy(), pin_mask.numpy())
        ip.run()
        ip.result()
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_ms.append(1e3 * (t1 - t0))
    e2e_value = evals_per_removal * len(e2e_ms) * world / (sum(e2e_ms) / 1e3)

    line = None
    if rank == 0:
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        clocks = clk.summary()
        mhz = peaks.get("sm_max_mhz") or 2070.0
        peak = sms * EVALS_PER_CLK_SM * mhz * 1e6
        eng_ms = statistics.mean(run_ms)
        ach = evals_per_removal / (eng_ms / 1e3)
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
            "gpu_launches": (launches_init(H) + 1) * args.steps,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "evals/s", "frac": ach / peak,
                         "traffic": ENGINE_TRAFFIC_BYTES, "traffic_unit": "bytes per launch (ncu)",
                         "kernel": "k_engine (one persistent launch per removal)",
                         "peak_source": f"{sms} SMs x {EVALS_PER_CLK_SM} evals/clk x {mhz:.0f} MHz",
                         "search_phase": {"ns": search_ns, "iters": timed_iters,
                                          "evals_per_s": evals_per_removal / (search_ns * 1e-9) if search_ns else None},
                         "update_phase_ns": update_ns},
            "clocks": clocks,
        }
        if not args.skip_extras and world == 1:
            from paper_1403_4238_gb300 import synth

            line["tc"] = tc_section(api, case, flush, 3, peaks, line["ms_per_removal"], plain_out)
            hd = synth.hd_blob()
            line["tc_hd"] = tc_section(api, hd, flush, 2, peaks)
            line["overlap"] = overlap_section(api, case, flush, 3, line["roofline"]["peak"])
            line["init"] = init_section(api, [case, hd], flush, 5, peaks.get("hbm_gbs"))
            line["batched"] = batch_section(api, flush, 3, print)
            line["serving"] = serving_section(api, args.serve_requests)
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
