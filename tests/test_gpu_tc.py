"""GPU parity of the exact tensor-core search form (INPAINT_FORM_TC).

The tcgen05 BF16 correlation form computes every SSD as an exact integer
(A2 - 2X + 256 hi + lo, Sec. 3 Eq. 4 expanded), so the whole fill must equal
the oracle's bit for bit: tolerance 0 on p^, q~, SSD, priority, confidence and
the final image.  Both loops: the persistent engine (its tensor-core tiles of
16 candidate rows, every iteration counted by tc_rounds()) and the graph loop
(the stand-alone tensor-core search kernel).
"""
import numpy as np
import pytest

import oracle
from paper_1403_4238_gb300 import synth

pytestmark = pytest.mark.gpu

FIELDS = ("px", "py", "qx", "qy", "ssd", "priority", "confidence", "filled", "remaining",
          "n_known", "n_cand")


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4238_gb300 import api as _api
    return _api


def assert_trace_equal(gpu, ora, n=None):
    n = len(ora) if n is None else n
    assert len(gpu) >= n and len(ora) >= n
    for i in range(n):
        for f in FIELDS:
            a, b = gpu[i][f], ora[i][f]
            if f in ("priority", "confidence"):
                assert np.float64(a).view(np.uint64) == np.float64(b).view(np.uint64), (i, f, a, b)
            else:
                assert a == b, (i, f, a, b)


LOOPS = ("engine", "graph")


def run_tc(api, case, loop, **kw):
    with api.Inpainter(case.rgb, case.mask, case.r, form="tc", loop=loop, **kw) as ip:
        rc, n, tr = ip.run(trace=True)
        # the engine searched every iteration in the tensor-core form
        assert ip.tc_rounds() == (n if loop == "engine" else 0)
        return rc, n, tr, ip.result(), ip.info()


@pytest.mark.parametrize("loop", LOOPS)
@pytest.mark.parametrize("W,H,r,seed", [
    (20, 16, 1, 1), (24, 20, 2, 2), (33, 27, 3, 3), (40, 31, 4, 4), (47, 35, 5, 5),
    (52, 45, 6, 6), (61, 50, 7, 7), (70, 58, 8, 8),
])
def test_tc_tiny_every_radius(api, W, H, r, seed, loop):
    case = synth.tiny(W, H, seed, r=r)
    ora = oracle.run(case.rgb, case.mask, case.r)
    rc, n, tr, out, info = run_tc(api, case, loop, debug=True)
    assert rc == 0 and n == ora.iters
    assert_trace_equal(tr, ora.trace)
    assert np.array_equal(out, ora.rgb)
    assert info["evals"] == ora.evals


@pytest.mark.parametrize("loop", LOOPS)
@pytest.mark.parametrize("W,H,r,seed", [(1100, 90, 4, 21), (1030, 70, 8, 22), (517, 61, 2, 23),
                                        (2500, 40, 3, 24)])
def test_tc_wide_images_span_several_tiles(api, W, H, r, seed, loop):
    # more than one tile per row (graph loop: 512-column plane tiles; engine:
    # 512 or 1024 candidate columns), ragged last tiles and rows
    case = synth.Case("wide", synth.image(W, H, 9, 35.0, seed),
                      synth.ellipse_mask(W, H, 2, 0.03, 0.05, seed + 1), r)
    ora = oracle.run(case.rgb, case.mask, case.r)
    rc, n, tr, out, info = run_tc(api, case, loop)
    assert rc == 0 and n == ora.iters
    assert_trace_equal(tr, ora.trace)
    assert np.array_equal(out, ora.rgb)


@pytest.mark.parametrize("loop", LOOPS)
def test_tc_border_holes_and_alpha(api, loop):
    W, H, r = 203, 77, 4
    rgb = synth.image(W, H, 5, 30.0, 77)
    mask = np.zeros((H, W), np.uint8)
    mask[0:9, 190:203] = 1
    mask[60:77, 0:6] = 1
    case = synth.Case("border", rgb, mask, r)
    for alpha in (-1.0, 0.5):
        ora = oracle.run(case.rgb, case.mask, case.r, alpha=alpha)
        rc, n, tr, out, info = run_tc(api, case, loop, alpha=alpha)
        assert_trace_equal(tr, ora.trace)
        assert np.array_equal(out, ora.rgb)


@pytest.mark.parametrize("loop", LOOPS)
def test_tc_walkingman_like_config(api, loop):
    case = synth.walkingman_like()
    ora = oracle.run(case.rgb, case.mask, case.r)
    rc, n, tr, out, info = run_tc(api, case, loop)
    assert rc == 0 and n == ora.iters
    assert_trace_equal(tr, ora.trace)
    assert np.array_equal(out, ora.rgb)
    assert info["evals"] == ora.evals


@pytest.mark.parametrize("loop", LOOPS)
def test_tc_equals_plain_on_hd_prefix(api, loop):
    # 1920 x 1080, r = 6: the first iterations against the oracle, a longer
    # prefix against the CUDA-core form (the whole removal: test_gpu_golden)
    case = synth.hd_blob()
    ora = oracle.run(case.rgb, case.mask, case.r, max_iters=3)
    outs = {}
    for form in ("tc", "plain"):
        with api.Inpainter(case.rgb, case.mask, case.r, form=form, loop=loop) as ip:
            rc, n, tr = ip.run(max_iters=60, trace=True)
            outs[form] = (n, tr, ip.result())
    assert outs["tc"][0] == outs["plain"][0] == 60
    assert_trace_equal(outs["tc"][1], ora.trace, n=3)
    assert_trace_equal(outs["tc"][1], outs["plain"][1])
    assert np.array_equal(outs["tc"][2], outs["plain"][2])


def test_tc_engine_resumes_across_launches(api):
    # run() in chunks: each chunk is one engine launch that rebuilds the
    # planes from the image and the validity bits from the counts
    case = synth.walkingman_like()
    ora = oracle.run(case.rgb, case.mask, case.r)
    with api.Inpainter(case.rgb, case.mask, case.r, form="tc", loop="engine") as ip:
        tr = []
        while True:
            rc, n, part = ip.run(max_iters=97, trace=True)
            tr.extend(part)
            if n < 97 or ip.info()["remaining"] == 0:
                break
        assert ip.tc_rounds() == len(tr) == ora.iters
        assert_trace_equal(tr, ora.trace)
        assert np.array_equal(ip.result(), ora.rgb)


def test_tc_step_by_step_equals_run(api):
    case = synth.small_rect(seed=11)
    ora = oracle.run(case.rgb, case.mask, case.r)
    with api.Inpainter(case.rgb, case.mask, case.r, form="tc") as ip:
        recs = []
        while True:
            rec = ip.step()
            if rec is None:
                break
            recs.append(rec)
        assert_trace_equal(recs, ora.trace)
        assert np.array_equal(ip.result(), ora.rgb)


def test_tc_rejects_unsupported(api):
    case = synth.tiny(40, 40, 3, r=9)
    for loop in ("engine", "graph"):
        with pytest.raises(api.InpaintError):
            api.Inpainter(case.rgb, case.mask, 9, form="tc", loop=loop)
