"""GPU parity: the CUDA library against the CPU oracle, bit for bit.

Tolerance 0 everywhere: the fill order (p^ per iteration), the chosen source
patch q~, its SSD, the priority and confidence bits, counts, and the final
image must equal the oracle's (Sec. 3, Eq. 1-4 as restated there).
"""
import numpy as np
import pytest

import oracle
from paper_1403_4238_gb300 import synth

pytestmark = pytest.mark.gpu

FIELDS = ("iter", "px", "py", "qx", "qy", "ssd", "priority", "confidence", "filled", "remaining",
          "n_known", "n_cand")


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4238_gb300 import api as _api
    return _api


def assert_trace_equal(gpu, ora, n=None, skip=()):
    n = len(ora) if n is None else n
    assert len(gpu) >= n and len(ora) >= n
    for i in range(n):
        for f in FIELDS:
            if f in skip:
                continue
            a, b = gpu[i][f], ora[i][f]
            if f in ("priority", "confidence"):
                assert np.float64(a).view(np.uint64) == np.float64(b).view(np.uint64), (i, f, a, b)
            else:
                assert a == b, (i, f, a, b)


def run_both(api, case, **kw):
    ora = oracle.run(case.rgb, case.mask, case.r, alpha=kw.get("alpha", -1.0))
    with api.Inpainter(case.rgb, case.mask, case.r, **kw) as ip:
        rc, n, tr = ip.run(trace=True)
        out, m = ip.result(with_mask=True)
        info = ip.info()
    return ora, (rc, n, tr, out, m, info)


LOOPS = ["engine", "graph"]


@pytest.mark.parametrize("loop", LOOPS)
@pytest.mark.parametrize("W,H,r,seed", [
    (20, 16, 1, 1), (24, 20, 2, 2), (33, 27, 3, 3), (40, 31, 4, 4), (47, 35, 5, 5),
    (52, 45, 6, 6), (61, 50, 7, 7), (70, 58, 8, 8), (75, 64, 9, 9), (90, 80, 12, 10),
    (240, 160, 32, 14),  # the largest radius (65 x 65 patches)
])
def test_tiny_full_runs_every_radius(api, W, H, r, seed, loop):
    if loop == "engine" and r > 8:
        loop = "auto"  # the engine covers r <= 8; larger radii use the graph loop
    case = synth.tiny(W, H, seed, r=r)
    ora, (rc, n, tr, out, m, info) = run_both(api, case, debug=True, loop=loop)
    assert ora.status == 0 and rc == 0
    assert n == ora.iters
    assert_trace_equal(tr, ora.trace)
    assert np.array_equal(out, ora.rgb)
    assert m.sum() == 0 and info["evals"] == ora.evals


@pytest.mark.parametrize("loop,tile_rows", [("engine", 1), ("engine", 2), ("graph", 0)])
def test_small_rect_config(api, loop, tile_rows):
    case = synth.small_rect()
    ora, (rc, n, tr, out, m, info) = run_both(api, case, debug=True, loop=loop, tile_rows=tile_rows)
    assert n == ora.iters == len(tr)
    assert_trace_equal(tr, ora.trace)
    assert np.array_equal(out, ora.rgb)
    assert info["evals"] == ora.evals


def test_step_by_step_equals_run(api):
    case = synth.small_rect(seed=11)
    ora = oracle.run(case.rgb, case.mask, case.r)
    with api.Inpainter(case.rgb, case.mask, case.r) as ip:
        recs = []
        while True:
            rec = ip.step()
            if rec is None:
                break
            recs.append(rec)
        assert_trace_equal(recs, ora.trace)
        assert np.array_equal(ip.result(), ora.rgb)
        assert ip.step() is None  # DONE afterwards


@pytest.mark.parametrize("loop", LOOPS)
def test_border_masks_and_ragged_tiles(api, loop):
    # candidate grid not a multiple of the 128 x 8 tile; hole on two borders
    rng = np.random.default_rng(5)
    W, H, r = 203, 77, 4
    rgb = synth.image(W, H, 5, 30.0, 77)
    mask = np.zeros((H, W), np.uint8)
    mask[0:9, 190:203] = 1
    mask[60:77, 0:6] = 1
    mask[30:40, 100:113] = rng.integers(0, 2, (10, 13)).astype(np.uint8)
    case = synth.Case("border", rgb, mask, r)
    ora, (rc, n, tr, out, m, info) = run_both(api, case, debug=True, loop=loop)
    assert_trace_equal(tr, ora.trace)
    assert np.array_equal(out, ora.rgb)


@pytest.fixture(scope="module")
def walkingman():
    case = synth.walkingman_like()
    return case, oracle.run(case.rgb, case.mask, case.r)


@pytest.mark.parametrize("loop", LOOPS)
def test_walkingman_like_config(api, walkingman, loop):
    case, ora = walkingman
    with api.Inpainter(case.rgb, case.mask, case.r, loop=loop) as ip:
        rc, n, tr = ip.run(trace=True)
        out = ip.result()
        info = ip.info()
    assert rc == 0 and n == ora.iters
    assert_trace_equal(tr, ora.trace)
    assert np.array_equal(out, ora.rgb)
    assert info["evals"] == ora.evals


def test_hd_blob_prefix_and_sampled_iterations(api):
    """1920x1080, r = 6: the oracle takes minutes for the whole run, so check
    the first iterations exactly, then sample later iterations from exported
    GPU states, and check the whole run's invariants."""
    case = synth.hd_blob()
    ora = oracle.run(case.rgb, case.mask, case.r, max_iters=2)
    with api.Inpainter(case.rgb, case.mask, case.r, loop="engine") as ip:
        rc, n, tr = ip.run(max_iters=2, trace=True)
        assert n == 2
        assert_trace_equal(tr, ora.trace)
        done_iters = 2
        for target in (150, 600):
            if ip.info()["remaining"] == 0:
                break
            ip.run(max_iters=target - done_iters)
            done_iters = target
            rgb, om, conf = ip.export_state()
            if om.sum() == 0:
                break
            ref = oracle.run_from_state(rgb, om, conf, case.r, max_iters=1)
            rc, n, tr1 = ip.run(max_iters=1, trace=True)
            done_iters += 1
            assert tr1[0]["iter"] == done_iters - 1
            assert_trace_equal(tr1, ref.trace, skip=("iter",))  # the oracle restarts at 0
            # the GPU state after that iteration equals the oracle's
            rgb2, om2, conf2 = ip.export_state()
            assert np.array_equal(rgb2, ref.rgb) and np.array_equal(om2, ref.mask)
            assert np.array_equal(conf2.view(np.uint64), ref.conf.view(np.uint64))
        rc, n, tr = ip.run(trace=False)
        out, m = ip.result(with_mask=True)
    om0 = case.mask != 0
    assert m.sum() == 0
    assert np.array_equal(out[~om0], case.rgb[~om0])


def test_status_codes(api):
    case = synth.tiny(20, 16, 3, r=2)
    empty = np.zeros_like(case.mask)
    with api.Inpainter(case.rgb, empty, 2) as ip:
        assert ip.run()[0] == 1  # DONE
        assert ip.step() is None
    with pytest.raises(api.InpaintError) as e:
        api.Inpainter(case.rgb, np.ones_like(case.mask), 2)
    assert e.value.code == -1
    m = np.ones((16, 20), np.uint8)
    m[0, 0] = 0
    with api.Inpainter(case.rgb, m, 2) as ip:
        with pytest.raises(api.InpaintError) as e:
            ip.run()
        assert e.value.code == -4
        # state unchanged: still every pixel but one unknown
        assert ip.info()["remaining"] == 16 * 20 - 1


@pytest.mark.parametrize("loop", LOOPS)
def test_search_alpha_matches_oracle(api, loop):
    case = synth.small_rect(seed=21)
    for alpha in (0.6, 1.5):
        ora = oracle.run(case.rgb, case.mask, case.r, alpha=alpha)
        with api.Inpainter(case.rgb, case.mask, case.r, alpha=alpha, loop=loop) as ip:
            assert ip.search_rect() == oracle.search_rect(case.mask, case.r, alpha)
            rc, n, tr = ip.run(trace=True)
            if ora.status == 0:
                assert_trace_equal(tr, ora.trace)
                assert np.array_equal(ip.result(), ora.rgb)
            else:
                assert rc == ora.status or ora.status == -4


def test_reset_from_device_tensors_matches_create(api):
    import torch
    a = synth.small_rect(seed=31)
    b = synth.small_rect(seed=32)
    ora_b = oracle.run(b.rgb, b.mask, b.r)
    with api.Inpainter(a.rgb, a.mask, a.r) as ip:
        ip.run()
        drgb, dmask = torch.from_numpy(b.rgb).cuda(), torch.from_numpy(b.mask).cuda()
        torch.cuda.synchronize()  # the copies ran on torch's stream, the library uses its own
        ip.reset(drgb, dmask)
        rc, n, tr = ip.run(trace=True)
        assert_trace_equal(tr, ora_b.trace)
        ip.reset(a.rgb, a.mask)  # host inputs again
        rc, n, tr = ip.run(trace=True)
        assert np.array_equal(ip.result(), oracle.run(a.rgb, a.mask, a.r).rgb)


def test_export_import_resume(api):
    case = synth.small_rect(seed=41)
    ora = oracle.run(case.rgb, case.mask, case.r)
    with api.Inpainter(case.rgb, case.mask, case.r) as ip:
        ip.run(max_iters=4)
        st = ip.export_state()
    with api.Inpainter(case.rgb, case.mask, case.r) as ip2:
        ip2.import_state(*st)
        rc, n, tr = ip2.run(trace=True)
        assert np.array_equal(ip2.result(), ora.rgb)
        assert n == ora.iters - 4


def test_deterministic_repeat(api):
    case = synth.small_rect(seed=51)
    outs = []
    for _ in range(2):
        with api.Inpainter(case.rgb, case.mask, case.r) as ip:
            rc, n, tr = ip.run(trace=True)
            outs.append((ip.result(), tr))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
