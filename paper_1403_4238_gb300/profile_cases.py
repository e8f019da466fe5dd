"""Small, self-contained GPU workloads for profiling the kernels one by one.

Each case runs a bounded number of launches of one kernel on a seeded
synthetic input, so that a profiler can be pointed at it with a kernel
filter and a launch count:

    python -m paper_1403_4238_gb300.profile_cases engine_512x384 --reps 4
    python -m paper_1403_4238_gb300.profile_cases search_tc_1080p --reps 3
    python -m paper_1403_4238_gb300.profile_cases search_plain_1080p --reps 3

engine_*   whole removals (one persistent k_engine launch each, plus the
           initialisation kernels), plain form (engine_tc_*: the tensor-core
           form); --iters N stops each launch after N iterations (a shorter
           launch for a full-counter capture);
search_*   the findBestPatch kernel of one form alone, for the first target
           of the removal (inpaint_time_search), after one untimed launch.
"""
from __future__ import annotations

import argparse

from . import api, synth

CASES = {
    "engine_512x384": (synth.walkingman_like, "engine", "plain"),
    "engine_1080p": (synth.hd_blob, "engine", "plain"),
    "engine_tc_512x384": (synth.walkingman_like, "engine", "tc"),
    "engine_tc_1080p": (synth.hd_blob, "engine", "tc"),
    "search_tc_512x384": (synth.walkingman_like, "search", "tc"),
    "search_plain_512x384": (synth.walkingman_like, "search", "plain"),
    "search_tc_1080p": (synth.hd_blob, "search", "tc"),
    "search_plain_1080p": (synth.hd_blob, "search", "plain"),
}


def run(name: str, reps: int, iters: int = 0):
    import torch

    make, kind, form = CASES[name]
    case = make()
    if kind == "engine":
        with api.Inpainter(case.rgb, case.mask, case.r, form=form, loop="engine") as ip:
            drgb, dmask = torch.from_numpy(case.rgb).cuda(), torch.from_numpy(case.mask).cuda()
            for _ in range(reps):
                ip.reset(drgb, dmask)
                rc, n, _ = ip.run(max_iters=iters)
                assert rc == 0, rc
            print(f"{name}: {reps} launches of {n} iterations, {ip.info()['evals']} evals each")
    else:
        with api.Inpainter(case.rgb, case.mask, case.r, loop="graph") as ip:
            ms, key, ev = ip.time_search(form, reps)
            print(f"{name}: {1e3 * ms:.2f} us per search, key {key:#x}, {ev} evals")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--iters", type=int, default=0, help="engine cases: iterations per launch (0: all)")
    a = ap.parse_args()
    run(a.case, a.reps, a.iters)


if __name__ == "__main__":
    main()
