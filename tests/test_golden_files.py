"""The stored full-size removal results (tests/golden/removals.json and the
trace files, written by make_removal_golden.py from the oracle) are
consistent with themselves and belong to the inputs the generator makes
today, so that the GPU tests comparing against them compare like with like."""
import functools
import hashlib
import json
import os

import numpy as np

from paper_1403_4238_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@functools.lru_cache(maxsize=None)
def _ns():
    # the generator's namespace; the list makers are cached (one call builds all 64 images)
    ns = {k: getattr(synth, k) for k in dir(synth) if not k.startswith("_")}
    ns["batch_cases"] = functools.lru_cache(maxsize=None)(synth.batch_cases)
    ns["serving_trace"] = functools.lru_cache(maxsize=None)(synth.serving_trace)
    return ns


def load():
    with open(os.path.join(GOLDEN, "removals.json")) as f:
        return json.load(f)["removals"]


def test_trace_files_match_their_digests_and_counts():
    for e in load():
        assert e["status"] == 0 and e["iters"] > 0 and e["evals"] > 0
        if not e["trace_file"]:
            continue
        lines = []
        with open(os.path.join(GOLDEN, e["trace_file"])) as f:
            for line in f:
                if not line.startswith("#"):
                    lines.append(line.rstrip("\n"))
        assert hashlib.sha256("\n".join(lines).encode()).hexdigest() == e["trace_sha256"]
        assert len(lines) == e["iters"]
        rows = [list(map(lambda v: int(v, 16) if len(v) == 16 else int(v), ln.split())) for ln in lines]
        filled = sum(r[7] for r in rows)
        assert filled == e["unknown"]          # every unknown pixel filled exactly once
        assert rows[-1][8] == 0                 # nothing remains
        # |Omega| shrinks by the filled count each iteration
        rem = e["unknown"]
        for r in rows:
            rem -= r[7]
            assert r[8] == rem
        # evaluations are the sum of candidates x known pixels
        assert sum(r[9] * r[10] for r in rows) == e["evals"]


def test_stored_inputs_are_the_generators_bytes():
    # the small entries only (the 1920x1080 input is checked by the GPU test)
    for e in load():
        if e["W"] * e["H"] > 600000:
            continue
        expr = e["generator"][len("synth."):]
        case = eval(expr, _ns())
        assert hashlib.sha256(np.ascontiguousarray(case.rgb).tobytes()).hexdigest() == e["rgb_sha256"]
        assert hashlib.sha256(np.ascontiguousarray(case.mask).tobytes()).hexdigest() == e["mask_sha256"]
        assert int((case.mask != 0).sum()) == e["unknown"]
