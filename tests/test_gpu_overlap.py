"""GPU parity of the partial-overlap search variant (Algorithm 1, Sec. 5.4)
against the oracle, bit for bit: every centre of the search rectangle is a
candidate (also overlapping Omega or crossing the border), the SSD runs over
the known target / known source pairs, and a candidate needs a known source
pixel under every pixel it fills."""
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


def assert_trace_equal(gpu, ora):
    assert len(gpu) >= len(ora)
    for i in range(len(ora)):
        for f in FIELDS:
            a, b = gpu[i][f], ora[i][f]
            if f in ("priority", "confidence"):
                assert np.float64(a).view(np.uint64) == np.float64(b).view(np.uint64), (i, f, a, b)
            else:
                assert a == b, (i, f, a, b)


def run_both(api, case, alpha=-1.0, **kw):
    ora = oracle.run(case.rgb, case.mask, case.r, alpha=alpha, overlap=True)
    with api.Inpainter(case.rgb, case.mask, case.r, alpha=alpha, overlap=True, **kw) as ip:
        assert ip.search_rect() == oracle.search_rect(case.mask, case.r, alpha, overlap=True)
        rc, n, tr = ip.run(trace=True)
        out = ip.result()
        info = ip.info()
    return ora, rc, n, tr, out, info


@pytest.mark.parametrize("W,H,r,seed", [
    (20, 16, 1, 31), (24, 20, 2, 32), (33, 27, 3, 33), (40, 31, 4, 34), (47, 35, 5, 35),
    (52, 45, 6, 36), (61, 50, 7, 37), (70, 58, 8, 38),
])
def test_tiny_runs_every_radius(api, W, H, r, seed):
    case = synth.tiny(W, H, seed, r=r)
    ora, rc, n, tr, out, info = run_both(api, case, debug=True)
    assert ora.status == 0 and rc == 0 and n == ora.iters
    assert_trace_equal(tr, ora.trace)
    assert np.array_equal(out, ora.rgb)
    assert info["evals"] == ora.evals


@pytest.mark.parametrize("alpha", [-1.0, 0.3, 1.0])
def test_small_rect_and_search_factor(api, alpha):
    case = synth.small_rect(seed=41)
    ora, rc, n, tr, out, info = run_both(api, case, alpha=alpha)
    assert ora.status == 0 and n == ora.iters
    assert_trace_equal(tr, ora.trace)
    assert np.array_equal(out, ora.rgb)
    assert info["evals"] == ora.evals


def test_border_holes_ragged_tiles(api):
    # holes on three borders, candidate grid not a multiple of the tile
    rng = np.random.default_rng(6)
    W, H, r = 203, 77, 4
    rgb = synth.image(W, H, 5, 30.0, 78)
    mask = np.zeros((H, W), np.uint8)
    mask[0:9, 190:203] = 1
    mask[60:77, 0:6] = 1
    mask[30:40, 100:113] = rng.integers(0, 2, (10, 13)).astype(np.uint8)
    case = synth.Case("border", rgb, mask, r)
    ora, rc, n, tr, out, info = run_both(api, case)
    assert ora.status == 0
    assert_trace_equal(tr, ora.trace)
    assert np.array_equal(out, ora.rgb)


def test_step_path_and_differs_from_full_search(api):
    case = synth.small_rect(seed=43)
    ora = oracle.run(case.rgb, case.mask, case.r, overlap=True)
    full = oracle.run(case.rgb, case.mask, case.r)
    assert ora.evals != full.evals  # the variant searches other candidates
    with api.Inpainter(case.rgb, case.mask, case.r, overlap=True) as ip:
        recs = []
        while (rec := ip.step()) is not None:
            recs.append(rec)
        assert_trace_equal(recs, ora.trace)
        assert np.array_equal(ip.result(), ora.rgb)


def test_no_admissible_candidate(api):
    # a 1-pixel-wide known border around a hole: no candidate can cover the
    # 5 x 5 unknown part of a target patch with known pixels
    W, H, r = 24, 20, 2
    rgb = synth.image(W, H, 3, 30.0, 5)
    mask = np.ones((H, W), np.uint8)
    mask[0, :] = 0
    ora = oracle.run(rgb, mask, r, overlap=True)
    assert ora.status == -4 and ora.iters == 0
    with api.Inpainter(rgb, mask, r, overlap=True) as ip:
        with pytest.raises(api.InpaintError) as e:
            ip.run()
        assert e.value.code == -4
