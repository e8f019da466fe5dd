"""Benchmark of exemplar-based object removal on GB300 (one JSON line on rank 0).

Headline workload (one "step"): one whole object removal of a 1920x1080
synthetic image with a random-walk blob mask covering about 5 % of the
pixels, 13x13 patches (radius 6), exhaustive search -- initialisation from
inputs already in HBM, then the device-driven fill loop (persistent engine
with the exact tensor-core search, --form plain for the CUDA-core search)
until the target region is empty.  The metric is candidate-pixel SSD
evaluations per second (one evaluation = one valid candidate x one known
target pixel, all three channels), counted exactly by the device loop; ms
per removal is reported beside it, and the line's "plain_engine" holds the
same removal with the plain form (time, roofline, and the speedup).

Beside the headline the same JSON line carries:
  walkingman  the 512x384 removal (3 ellipses, 8 %, 9x9 patches) with the
              headline's keys (value, e2e, roofline, cpu_baseline);
  tc, tc_hd  the exact tensor-core search form on both removals (whole
              removal in the engine and in the graph loop, and the search
              kernel alone), as speedups over the plain form, outputs compared;
  batched     64 images of uneven sizes in one persistent launch (CUDA
              graph), images/s and the speedup over one after another;
  serving     Poisson arrivals through the continuous-batching server under
              a 40 GB HBM budget: its capacity (closed loop), p50/p99
              latency at 0.5x and 0.9x of it and at 200 req/s;
  overlap, init, peaks  the partial-overlap search variant, the
              initialisation's bandwidth, the measured instruction rates.

--gpus N > 1 re-launches itself under torch.distributed.run with N ranks:
every rank runs the headline removal (replicas, weak scaling), and the
batched and serving workloads are split over the ranks by estimated work
(independent images: no collective on the data path).  --dry-run does the
rank set-up and the split on CPU (gloo) without a GPU.

--impl reference times the CPU oracle (the plain single-threaded C
restatement of the method) on a bounded sample of the same removal.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "candidate-pixel SSD evals/s (whole removal, 1920x1080, 13x13 patch, exhaustive search)"
UNIT = "evals/s"
WORKLOAD = ("1920x1080 RGB, random-walk blob mask 4.5% (93,336 px), r=6 (13x13), exhaustive search, "
            "{form} form, persistent engine")
FORM_NAMES = {"tc": "exact tensor-core", "plain": "plain CUDA-core"}
WORKLOAD2 = "512x384 RGB, 3-ellipse mask 7.5-8.5%, r=4 (9x9), exhaustive search, plain form, persistent engine"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--form", default="tc", choices=["tc", "plain"],
                    help="search form of the headline removal (the other one is timed beside it)")
    ap.add_argument("--cpu-iters", type=int, default=12,
                    help="oracle iterations of the CPU sample (a bounded prefix of the removal)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-extras", action="store_true",
                    help="headline only: no 512x384, tensor-core, batched or serving sections")
    ap.add_argument("--serve-seconds", type=float, default=8.0,
                    help="arrival span of each open-loop serving run")
    ap.add_argument("--dry-run", action="store_true",
                    help="rank set-up and work split only, on CPU (gloo); no GPU work")
    ap.add_argument("--json-out", default=None)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def relaunch(args) -> int:
    """--gpus N > 1 outside a launcher: run this script under torch.distributed.run."""
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


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

    return synth.hd_blob()


def workload2():
    from paper_1403_4238_gb300 import synth

    return synth.walkingman_like()


def cpu_sample(case, iters):
    """Oracle on a bounded prefix of the removal: (evals/s, seconds, evals, iterations)."""
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    res = oracle.run(case.rgb, case.mask, case.r, max_iters=iters)
    dt = time.perf_counter() - t0
    return res.evals / dt, dt, res.evals, res.iters


def run_reference(args):
    """The oracle as it stands, one iteration of the headline removal per step
    (each step continues from the state the previous one left)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    case = workload()
    rgb, om = case.rgb.copy(), (case.mask != 0).astype(np.uint8)
    conf = np.where(om != 0, 0.0, 1.0)
    vals = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        res = oracle.run_from_state(rgb, om, conf, case.r, max_iters=1)
        dt = time.perf_counter() - t0
        rgb, om, conf = res.rgb, res.mask, res.conf
        if i >= args.warmup:
            vals.append((dt, res.evals))
    tot_t = sum(v[0] for v in vals)
    value = sum(v[1] for v in vals) / tot_t
    sample = (f"iterations {args.warmup + 1}-{args.warmup + args.steps} of the 1920x1080 removal, "
              f"one per step, each continuing from the previous state (oracle, 1 thread)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(vals),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/int32/f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD.format(form=FORM_NAMES[args.form]), "W": int(case.rgb.shape[1]),
                   "H": int(case.rgb.shape[0]), "r": case.r, "mask_px": int(case.mask.sum()), "form": args.form,
                   "parallelism": "one host thread"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def l2_flush(buf):
    buf.add_(1)


# Plain-search roofline: one evaluation is one byte-SIMD absolute difference
# (vabsdiffu4, ALU pipe) plus one 4-way byte dot product (dp4a, FMA pipe),
# each occupying its pipe for two cycles per warp (16 lanes per clock per SM
# sub-partition), so an SM completes at most 64 evaluations per clock.  The
# algorithmic count of the method is 6 integer operations per evaluation
# (3 differences, 3 multiply-adds), reported as "effective INT32" against the
# measured scalar integer rate (64 lanes per clock per SM for IADD3 / IMAD).
EVALS_PER_CLK_SM = 64
INT32_LANES_PER_CLK_SM = 64
INT32_OPS_PER_EVAL = 6

# The committed ncu summary of the headline kernel: the DRAM bytes of one
# launch and the digest of the kernel sources the capture was taken on.
ENGINE_PROFILE = os.path.join(ROOT, "profiles", "k_engine_1920x1080.md")
ENGINE_TC_PROFILE = os.path.join(ROOT, "profiles", "k_engine_tc_1920x1080.md")
ENGINE_SOURCES = ("engine_impl.cuh", "engine_multi.cu", "update_fast.cuh", "inpaint_engine.h",
                  "inpaint_internal.cuh", "ptx.cuh", "gen_ssd_rows.py", "search_tc_engine.cuh")

# Tensor-core form, algorithmic work per evaluation: the im2col INT8 count
# of the expanded SSD, 3 weight sets x 3 channels = 9 MACs (18 FLOP); the
# exact BF16 form of this library does 5 useful MACs (3 colour products
# and the two halves of the squared source norm).  The MMAs it executes
# per tile follow from its geometry (Toeplitz target rows x 16 candidate
# rows x 8 shifts against N blocks of 8 candidate columns).
TC_ALGO_FLOP_PER_EVAL = 18
TC_USEFUL_FLOP_PER_EVAL = 10


def tc_mmas_per_iteration(W, H, r):
    """MMAs (128 x N x 16) one search of the engine's tensor-core form issues."""
    cx0, cx1, cy0, cy1 = r, W - 1 - r, r, H - 1 - r
    xs0 = (cx0 - r) & ~7
    wneed = cx1 - r - xs0 + 1
    ntx = (wneed + 1023) // 1024
    n = 64 if (wneed + 8 * ntx - 1) // (8 * ntx) <= 64 else 128
    nty = (cy1 - cy0 + 16) // 16
    p = 2 * r + 1
    nc = (p + 14) // 8
    per_tile = (16 + p - 1) * ((3 * nc + 1) // 2 + nc)
    return ntx * nty * per_tile, n


def engine_source_digest() -> str:
    h = hashlib.sha256()
    for f in ENGINE_SOURCES:
        with open(os.path.join(ROOT, "paper_1403_4238_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def engine_traffic(path=ENGINE_PROFILE):
    """(bytes per launch, note) from the committed capture, or (None, why)."""
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None, "no committed capture"
    vals = {}
    for line in text.splitlines():
        if line.startswith("traffic_bytes_per_launch:") or line.startswith("sources_digest:"):
            k, v = line.split(":", 1)
            vals[k] = v.strip()
    if "traffic_bytes_per_launch" not in vals:
        return None, "no traffic line in the capture"
    if vals.get("sources_digest") != engine_source_digest():
        return None, "kernel sources changed since the capture"
    return int(vals["traffic_bytes_per_launch"]), f"ncu capture, sources {vals['sources_digest']}"


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
    n = 0
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


def e2e_removals(ip, case, steps, warmup):
    """ms per removal through the public API from pinned host buffers: the
    host->device copy of the inputs, the removal and the device->host copy
    of the result inside the timed region."""
    import torch

    pin_rgb = torch.from_numpy(case.rgb).pin_memory()
    pin_mask = torch.from_numpy(case.mask).pin_memory()
    out = []
    for i in range(warmup + steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ip.reset(pin_rgb.numpy(), pin_mask.numpy())
        ip.run()
        ip.result()
        t1 = time.perf_counter()
        if i >= warmup:
            out.append(1e3 * (t1 - t0))
    return statistics.mean(out)


def roofline_plain(evals, run_ms, sms, mhz, peaks_probe, traffic):
    peak = sms * EVALS_PER_CLK_SM * mhz * 1e6
    ach = evals / (run_ms / 1e3)
    # scalar 32-bit integer peak: the measured rate of three-input adds and
    # multiply-adds when the probe ran, else 64 lanes per clock per SM
    if peaks_probe:
        i32 = max(peaks_probe["iadd3_per_s"], peaks_probe["imad_per_s"])
        i32_src = "measured (probe: max of IADD3 and IMAD rates)"
    else:
        i32 = sms * INT32_LANES_PER_CLK_SM * mhz * 1e6
        i32_src = f"{sms} SMs x {INT32_LANES_PER_CLK_SM} lanes/clk x {mhz:.0f} MHz"
    out = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "evals/s", "frac": ach / peak,
           "peak_source": f"{sms} SMs x {EVALS_PER_CLK_SM} evals/clk (two half-rate instructions on two "
                          f"pipes) x {mhz:.0f} MHz",
           "effective_int32": {"achieved": INT32_OPS_PER_EVAL * ach, "peak": i32,
                               "frac": INT32_OPS_PER_EVAL * ach / i32, "unit": "ops/s", "peak_source": i32_src,
                               "note": "6 scalar integer ops per evaluation (3 differences, 3 multiply-adds); "
                                       "the byte-SIMD pair does them 3 channels at a time, so this can exceed 1"}}
    if peaks_probe:
        pp = peaks_probe["ssd_evals_per_s"]
        out["peak_measured"] = pp
        out["frac_of_measured"] = ach / pp if pp else None
    out["traffic"], out["traffic_note"] = traffic
    return out


def roofline_tc(evals, iters, W, H, r, run_ms, peaks, traffic):
    """Tensor-bound roofline of the engine's tensor-core form."""
    peak = peaks.get("bf16_tflops")
    secs = run_ms / 1e3
    ach = evals * TC_ALGO_FLOP_PER_EVAL / secs / 1e12
    mmas, n = tc_mmas_per_iteration(W, H, r)
    executed = iters * mmas * 2 * 128 * n * 16 / secs / 1e12
    useful = evals * TC_USEFUL_FLOP_PER_EVAL / secs / 1e12
    out = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
           "frac": ach / peak if peak else None,
           "peak_source": "measured bf16 burst (MEASURED_PEAKS.json)" if peak else None,
           "algorithmic": f"{TC_ALGO_FLOP_PER_EVAL} FLOP per evaluation (9 MACs: 3 weight sets x 3 channels)",
           "useful_bf16": {"achieved": useful, "frac": useful / peak if peak else None,
                           "note": "5 MACs per evaluation: 3 colour products, 2 halves of the square norm"},
           "executed_mma": {"achieved": executed, "frac": executed / peak if peak else None,
                            "mmas_per_iteration": mmas, "shape": f"128x{n}x16",
                            "note": "MMA work issued, zero-padded Toeplitz rows included"}}
    out["traffic"], out["traffic_note"] = traffic
    return out


def single_section(api, case, flush, steps, warmup, peaks_probe, traffic, world, cpu_iters, sms, mhz):
    """One removal timed as the headline is: device-resident inputs, L2
    flushed between steps; the same metric end to end from host buffers;
    roofline of the engine; the oracle on a bounded prefix."""
    import torch

    H, W = case.mask.shape
    drgb, dmask = torch.from_numpy(case.rgb).cuda(), torch.from_numpy(case.mask).cuda()
    with api.Inpainter(case.rgb, case.mask, case.r) as ip:
        tot_ms, run_ms, iters = time_removals(ip, drgb, dmask, steps, warmup, flush)
        ev = ip.info()["evals"]
        s_ns, u_ns, it_t = ip.loop_timing()
        e2e_ms = e2e_removals(ip, case, max(2, steps // 2), 1)
        out_img = ip.result()
    res = {"value": ev / (tot_ms / 1e3), "unit": UNIT, "ms_per_removal": tot_ms, "iterations": iters,
           "evals_per_removal": ev, "W": W, "H": H, "r": case.r,
           "e2e": {"value": ev / (e2e_ms / 1e3), "unit": UNIT, "ms_per_removal": e2e_ms,
                   "h2d_bytes_per_step": 4 * W * H, "d2h_bytes_per_step": 3 * W * H},
           "roofline": roofline_plain(ev, run_ms, sms, mhz, peaks_probe, traffic),
           "phases_us_per_iteration": {"search": s_ns / 1e3 / max(it_t, 1), "update": u_ns / 1e3 / max(it_t, 1)}}
    if cpu_iters:
        v, dt, cev, cit = cpu_sample(case, cpu_iters)
        res["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"first {cit} of {iters} iterations of the same removal "
                                         f"({cev} evals, {dt:.1f} s)"}
    return res, out_img


def tc_section(api, case, flush, steps, peaks, known):
    """Tensor-core form vs the plain form on one removal: whole removal in
    the engine and in the graph loop, the search kernel alone (first
    target), outputs compared.  known: {(form, loop): (ms, image)} already
    timed by the caller."""
    import torch

    drgb = torch.from_numpy(case.rgb).cuda()
    dmask = torch.from_numpy(case.mask).cuda()
    out = {"workload": f"{case.mask.shape[1]}x{case.mask.shape[0]} r={case.r}"}
    res = dict(known)
    for form, loop in (("plain", "engine"), ("tc", "engine"), ("plain", "graph"), ("tc", "graph")):
        if (form, loop) in res:
            continue
        with api.Inpainter(case.rgb, case.mask, case.r, form=form, loop=loop) as ip:
            ms, _, n = time_removals(ip, drgb, dmask, steps, 1, flush)
            res[(form, loop)] = (ms, ip.result())
            out["iterations"] = n
    with api.Inpainter(case.rgb, case.mask, case.r, loop="graph") as ip:
        s_plain, k_plain, ev = ip.time_search("plain", 20)
        s_tc, k_tc, _ = ip.time_search("tc", 20)
    base_ms, base_img = res[("plain", "engine")]
    out.update({
        "ms_per_removal": {"plain_engine": base_ms, "tc_engine": res[("tc", "engine")][0],
                           "plain_graph": res[("plain", "graph")][0], "tc_graph": res[("tc", "graph")][0]},
        "speedup_vs_plain": base_ms / res[("tc", "engine")][0],
        "speedup_vs_plain_graph_loop": res[("plain", "graph")][0] / res[("tc", "graph")][0],
        "identical_outputs": bool(all(np.array_equal(v[1], base_img) for v in res.values())),
        "search_kernel_us": {"plain": 1e3 * s_plain, "tc": 1e3 * s_tc},
        "search_speedup": s_plain / s_tc,
        "search_same_key": bool(k_plain == k_tc),
        "search_evals": ev,
    })
    # the stand-alone (graph-loop) search kernel: 5 useful MACs per evaluation
    peak = peaks.get("bf16_tflops")
    ach = ev * 5 * 2 / (s_tc * 1e-3) / 1e12
    out["search_kernel_roofline"] = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                     "frac": (ach / peak) if peak else None, "traffic": None,
                                     "peak_source": "measured bf16 burst" if peak else None,
                                     "frac_at_9_macs_per_eval": (ach * 9 / 5 / peak) if peak else None}
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


def batch_work(c):
    """Estimated work of an image: candidate area x unknown pixels / patch area."""
    return float(c.mask.size) * float((c.mask != 0).sum()) / (2 * c.r + 1) ** 2


def batch_section(api, flush, steps, rank, world):
    """The 64 images split over the ranks by estimated work; each rank runs
    its share in one persistent launch (CUDA graph).  images/s counts every
    rank's images over the slowest rank's time."""
    import tempfile

    import torch

    from paper_1403_4238_gb300 import autotune, dist, synth

    cases = synth.batch_cases(64)
    mine = dist.my_share([batch_work(c) for c in cases], rank, world)
    sub = [cases[i] for i in mine]
    tf = os.path.join(tempfile.mkdtemp(prefix="inpaint_tune_"), "tuning_bench.txt")
    table = autotune.tune((4, 5), log=lambda *a: None)
    autotune.write(table, tf)
    items = [(c.rgb, c.mask, c.r) for c in sub]
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
        outs = [b.result(i)[0] for i in range(len(sub))]
        plan = b.plan()
    bms = dist.max_over_ranks(statistics.mean(ms))
    res = {"images": len(cases), "ranks": world, "images_per_s": len(cases) / (bms / 1e3), "ms_per_batch": bms,
           "graph": "reset and run captured in CUDA graphs", "teams": plan["teams"], "grid": plan["grid"],
           "autotune": [{"r": r, "max_pixels_per_cta": mp, "rows": rows} for r, mp, rows, _ in table]}
    if world == 1:
        # the same images one after another (plain form, persistent engine)
        seq_ms, same = 0.0, True
        for c, o in zip(sub, outs):
            drgb, dmask = torch.from_numpy(c.rgb).cuda(), torch.from_numpy(c.mask).cuda()
            with api.Inpainter(c.rgb, c.mask, c.r, tuning_file=tf) as ip:
                t, _, _ = time_removals(ip, drgb, dmask, 1, 1, flush)
                seq_ms += t
                same = same and np.array_equal(ip.result(), o)
        res.update({"ms_sequential": seq_ms, "speedup_vs_sequential": seq_ms / bms, "identical_outputs": bool(same)})
    return res


def serve_run(api, pool, arrivals, alone):
    """One open-loop run: request i arrives at arrivals[i] (seconds from the
    start; None = all at once) with pool case i mod len(pool).  Returns
    latencies (ms), span (s), identity with the solo results, completions."""
    with api.Server(hbm_budget_bytes=40 << 30, max_slots=256, iters_per_tick=0) as srv:
        ids = []
        t0 = time.perf_counter()
        for i, t in enumerate(arrivals):
            if t is not None:
                now = time.perf_counter() - t0
                if t > now:
                    time.sleep(t - now)
            c = pool[i % len(pool)]
            ids.append((srv.submit(c.rgb, c.mask, c.r), i % len(pool)))
        srv.wait_idle(600)
        lat, done, first, same, ok = [], [], None, True, 0
        for rid, k in ids:
            out, info = srv.poll(rid)
            ok += info["status"] == 0
            lat.append(1e3 * (info["t_done"] - info["t_submit"]))
            done.append(info["t_done"])
            first = info["t_submit"] if first is None else min(first, info["t_submit"])
            same = same and (alone is None or np.array_equal(out, alone[k]))
        ticks = srv.stats()["ticks"]
    return lat, max(done) - first, same, ok, ticks


def serving_section(api, rank, world, seconds, pool_n=24):
    """Continuous-batching server under a 40 GB budget.  Capacity: all of a
    block of requests submitted at once (closed loop), completions per
    second.  Then open-loop Poisson runs at 0.5x and 0.9x of that capacity
    and at 200 req/s, each over `seconds` of arrivals.  With several ranks,
    each rank serves every world-th request of each trace on its own GPU."""
    from paper_1403_4238_gb300 import dist, synth

    trace = synth.serving_trace(2000)
    pool = [synth.serving_case(*t[1:]) for t in trace[:pool_n]]
    alone = []
    for c in pool:
        with api.Inpainter(c.rgb, c.mask, c.r) as ip:
            ip.run()
            alone.append(ip.result())
    # closed loop: 4 x pool requests at once
    lat, span, same, ok, _ = serve_run(api, pool, [None] * (4 * pool_n), alone)
    cap = dist.max_over_ranks(span)
    capacity = 4 * pool_n * world / cap
    out = {"budget_gb": 40, "pool": f"{pool_n} distinct seeded cases from the trace, request i uses case i mod "
                                    f"{pool_n}", "capacity_req_s": capacity,
           "capacity_note": "closed loop: 96 requests submitted at once per rank, completions per second",
           "identical_to_alone": bool(same), "runs": []}

    rng = np.random.default_rng(5)
    for label, rate in (("0.5x capacity", 0.5 * capacity), ("0.9x capacity", 0.9 * capacity),
                        ("200 req/s", 200.0)):
        n = int(min(2000, max(world, round(rate * seconds))))
        arr = np.cumsum(rng.exponential(1.0 / rate, n))
        mine = [float(a) for i, a in enumerate(arr) if i % world == rank]
        lat, span, same_i, ok, ticks = serve_run(api, pool, mine, alone)
        span = dist.max_over_ranks(span)
        out["identical_to_alone"] = out["identical_to_alone"] and bool(same_i)
        out["runs"].append({"offered": label, "rate_req_s": rate, "requests": n, "completed_ok": ok,
                            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                            "images_per_s": n / span, "ticks": ticks})
    return out


def dry_run(args):
    """Rank set-up and work split on CPU (gloo): the JSON line carries the
    rank count and each rank's share, no timing."""
    import torch.distributed as tdist

    from paper_1403_4238_gb300 import dist, synth

    rank, world, _ = dist_env()
    if world > 1:
        tdist.init_process_group("gloo")
    cases = synth.batch_cases(64)
    mine = dist.my_share([batch_work(c) for c in cases], rank, world)
    shares = [None] * world
    if world > 1:
        tdist.all_gather_object(shares, mine)
    else:
        shares = [mine]
    if rank == 0:
        print(json.dumps({"dry_run": True, "n_gpus": world, "gpus_requested": args.gpus,
                          "batch_shares": shares, "metric": METRIC, "unit": UNIT}), flush=True)
    if world > 1:
        tdist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return relaunch(args)
    rank, world, local = dist_env()
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but the launcher started {world} ranks")
    if args.dry_run:
        return dry_run(args)
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_1403_4238_gb300 import api
    from paper_1403_4238_gb300.dist import max_over_ranks

    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = peaks.get("sm_max_mhz") or 2070.0
    probe = api.probe_peaks() if world == 1 else None
    case = workload()
    H, W = case.mask.shape
    dev_rgb = torch.from_numpy(case.rgb).cuda()
    dev_mask = torch.from_numpy(case.mask).cuda()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # 512 MB > L2
    ip = api.Inpainter(case.rgb, case.mask, case.r, form=args.form, loop="engine")
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
    if world > 1:
        torch.distributed.barrier()
    total_ms = max_over_ranks(sum(ms))
    value = evals_per_removal * args.steps * world / (total_ms / 1e3)
    head_out = ip.result()
    search_ns, update_ns, timed_iters = ip.loop_timing()
    tc_rounds = ip.tc_rounds()
    e2e_ms = max_over_ranks(e2e_removals(ip, case, args.steps, args.warmup))
    e2e_value = evals_per_removal * world / (e2e_ms / 1e3)
    ip.close()
    clocks = clk.summary()
    # the other form on the same removal (same timing rules, fewer steps)
    other = "plain" if args.form == "tc" else "tc"
    with api.Inpainter(case.rgb, case.mask, case.r, form=other, loop="engine") as ip2:
        o_tot, o_run, _ = time_removals(ip2, dev_rgb, dev_mask, max(3, args.steps // 2), 2, flush)
        o_s, o_u, o_it = ip2.loop_timing()
        other_out = ip2.result()

    line = None
    if rank == 0:
        if args.form == "tc":
            roof = roofline_tc(evals_per_removal, iters, W, H, case.r, statistics.mean(run_ms), peaks,
                               engine_traffic(ENGINE_TC_PROFILE))
            plain_ms, plain_run, p_s, p_u, p_it = o_tot, o_run, o_s, o_u, o_it
        else:
            roof = roofline_plain(evals_per_removal, statistics.mean(run_ms), sms, mhz, probe, engine_traffic())
            plain_ms, plain_run, p_s, p_u, p_it = total_ms / args.steps, statistics.mean(run_ms), search_ns, update_ns, timed_iters
        roof.update({"kernel": "k_engine (one persistent launch per removal)",
                     "phases_us_per_iteration": {"search": search_ns / 1e3 / max(timed_iters, 1),
                                                 "update": update_ns / 1e3 / max(timed_iters, 1)}})
        plain_roof = roofline_plain(evals_per_removal, plain_run, sms, mhz, probe, engine_traffic())
        plain_roof["phases_us_per_iteration"] = {"search": p_s / 1e3 / max(p_it, 1), "update": p_u / 1e3 / max(p_it, 1)}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "u8/bf16/f32/f64" if args.form == "tc" else "u8/int32/f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.format(form=FORM_NAMES[args.form]), "W": W, "H": H, "r": case.r,
                       "mask_px": int(case.mask.sum()), "iterations": iters, "evals_per_removal": evals_per_removal,
                       "form": args.form, "tc_rounds": tc_rounds,
                       "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas x{world}"},
            "ms_per_removal": total_ms / args.steps,
            "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_removal": e2e_ms,
                    "h2d_bytes_per_step": 4 * W * H, "d2h_bytes_per_step": 3 * W * H},
            # per removal: the initialisation kernels, (tensor-core form) the
            # planes, and one persistent engine launch
            "gpu_launches": (launches_init(H) + (2 if args.form == "tc" else 1)) * args.steps,
            "roofline": roof,
            "clocks": clocks,
            "plain_engine": {"ms_per_removal": plain_ms, "value": evals_per_removal / (plain_ms / 1e3),
                             "unit": UNIT, "roofline": plain_roof},
            "speedup_vs_plain": plain_ms / (total_ms / args.steps) if args.form == "tc" else 1.0,
            "identical_outputs_vs_other_form": bool(np.array_equal(head_out, other_out)),
        }
    if not args.skip_extras:
        if world == 1:
            case2 = workload2()
            sec2, out2 = single_section(api, case2, flush, max(args.steps, 20), args.warmup, probe, (None, "not captured"),
                                        world, 0 if args.no_cpu_baseline else 150, sms, mhz)
            sec2["workload"] = WORKLOAD2
            line["walkingman"] = sec2
            line["tc"] = tc_section(api, case2, flush, 3, peaks, {("plain", "engine"): (sec2["ms_per_removal"], out2)})
            known = {(args.form, "engine"): (line["ms_per_removal"], head_out),
                     (other, "engine"): (o_tot, other_out)}
            line["tc_hd"] = tc_section(api, case, flush, 2, peaks, known)
            line["overlap"] = overlap_section(api, case2, flush, 3, plain_roof["peak"])
            line["init"] = init_section(api, [case2, case], flush, 5, peaks.get("hbm_gbs"))
        bsec = batch_section(api, flush, 3, rank, world)
        ssec = serving_section(api, rank, world, args.serve_seconds)
        if rank == 0:
            line["batched"] = bsec
            line["serving"] = ssec
    if rank == 0:
        if probe:
            line["peaks"] = {k: probe[k] for k in ("ssd_evals_per_s", "imad_per_s", "iadd3_per_s", "dadd_per_s",
                                                    "sm_clock_mhz", "sm_count")}
        if not args.no_cpu_baseline and world == 1:
            v, dt, ev, it = cpu_sample(case, args.cpu_iters)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"first {it} of {iters} iterations of the same removal "
                                              f"({ev} evals, {dt:.1f} s)"}
        print(json.dumps(line), flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                json.dump(line, f, indent=1)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main() or 0)
