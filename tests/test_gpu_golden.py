"""Whole removals at full size against the oracle's stored results.

The 1920x1080 removal with 13x13 patches takes the oracle about 25 minutes
of one core, so its results were computed once by
tests/golden/make_removal_golden.py (which calls only oracle/) and stored:
the per-iteration trace (p^, q~, SSD, the bits of P(p^) and C(p^), counts)
and SHA-256 digests of the inputs and of the final image.  Here the CUDA
library runs the same removals -- every loop and search form of the single
image path, the batched form on six of the 64 batch images, and the server
on five requests of the Poisson trace -- and must match tolerance 0
(Sec. 3, Eq. 1-4 as restated by the oracle).
"""
import functools
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1403_4238_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FIELDS = ("px", "py", "qx", "qy", "ssd", "priority", "confidence", "filled", "remaining",
          "n_known", "n_cand")


@functools.lru_cache(maxsize=None)
def _ns():
    # the generator's namespace; the list makers are cached (one call builds all 64 images)
    ns = {k: getattr(synth, k) for k in dir(synth) if not k.startswith("_")}
    ns["batch_cases"] = functools.lru_cache(maxsize=None)(synth.batch_cases)
    ns["serving_trace"] = functools.lru_cache(maxsize=None)(synth.serving_trace)
    return ns


def removals():
    with open(os.path.join(GOLDEN, "removals.json")) as f:
        return {e["name"]: e for e in json.load(f)["removals"]}


def sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def make_case(entry):
    expr = entry["generator"][len("synth."):]
    case = eval(expr, _ns())
    # the stored results belong to exactly these input bytes
    assert sha(case.rgb) == entry["rgb_sha256"] and sha(case.mask) == entry["mask_sha256"], entry["name"]
    return case


def trace_rows(entry):
    rows = []
    with open(os.path.join(GOLDEN, entry["trace_file"])) as f:
        for line in f:
            if not line.startswith("#"):
                rows.append(line.split())
    return rows


def assert_trace_matches(tr, rows):
    assert len(tr) == len(rows)
    for i, (rec, row) in enumerate(zip(tr, rows)):
        for f, v in zip(FIELDS, row):
            if f in ("priority", "confidence"):
                got = "%016x" % int(np.float64(rec[f]).view(np.uint64))
            else:
                got = str(int(rec[f]))
            assert got == v, (i, f, got, v)


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4238_gb300 import api as _api
    return _api


@pytest.fixture(scope="module")
def hd():
    e = removals()["hd_blob"]
    return e, make_case(e), trace_rows(e)


@pytest.mark.parametrize("form,loop", [("plain", "engine"), ("plain", "graph"), ("tc", "engine"),
                                       ("tc", "graph")])
def test_full_hd_removal_equals_oracle(api, hd, form, loop):
    e, case, rows = hd
    with api.Inpainter(case.rgb, case.mask, case.r, form=form, loop=loop) as ip:
        rc, n, tr = ip.run(trace=True)
        out = ip.result()
        info = ip.info()
        tc_rounds = ip.tc_rounds()
    assert rc == 0 and n == e["iters"]
    # the engine's tensor-core form searched every iteration
    assert tc_rounds == (n if (form, loop) == ("tc", "engine") else 0)
    assert_trace_matches(tr, rows)
    assert sha(out) == e["result_sha256"]
    assert info["evals"] == e["evals"] and info["remaining"] == 0


def test_full_size_batch_images_equal_oracle(api):
    es = [v for k, v in removals().items() if k.startswith("batch64_")]
    cases = [make_case(e) for e in es]
    with api.Batch([(c.rgb, c.mask, c.r) for c in cases]) as b:
        st = b.run()
        for i, e in enumerate(es):
            out, iters, evals = b.result(i)
            assert st[i] == e["status"] == 0, e["name"]
            assert iters == e["iters"] and evals == e["evals"], e["name"]
            assert sha(out) == e["result_sha256"], e["name"]


def test_full_size_served_requests_equal_oracle(api):
    es = [v for k, v in removals().items() if k.startswith("serve2000_")]
    cases = [make_case(e) for e in es]
    with api.Server(hbm_budget_bytes=4 << 30, max_slots=8, iters_per_tick=0) as srv:
        ids = [srv.submit(c.rgb, c.mask, c.r) for c in cases]
        srv.wait_idle(600)
        for rid, e in zip(ids, es):
            out, info = srv.poll(rid)
            assert info["status"] == e["status"] == 0, e["name"]
            assert info["iterations"] == e["iters"] and info["evals"] == e["evals"], e["name"]
            assert sha(out) == e["result_sha256"], e["name"]
