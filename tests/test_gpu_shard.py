"""One removal split over replicas by candidate rows, on the GPU.

findBestPatch (Sec. 3, Eq. 3-4) is a minimum over candidate centres; the
library's row-range search and key application let replicas search disjoint
row slabs and apply the minimum key.  On one GPU the ranks are emulated by
sequential calls (several contexts, or several slabs of one context); every
iteration and the final image must equal the oracle's, bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1403_4238_gb300 import dist as pdist
from paper_1403_4238_gb300 import synth

pytestmark = pytest.mark.gpu

FIELDS = ("iter", "px", "py", "qx", "qy", "ssd", "filled", "remaining", "n_known", "n_cand")


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4238_gb300 import api as _api
    return _api


def same(a, b):
    for f in FIELDS:
        assert a[f] == b[f], (f, a[f], b[f])
    for f in ("priority", "confidence"):
        assert np.float64(a[f]).view(np.uint64) == np.float64(b[f]).view(np.uint64), f


def lockstep(ips, slabs):
    """Every replica searches its slab, all apply the minimum key."""
    recs = []
    while True:
        keys = [ip.search_rows(lo, hi) for ip, (lo, hi) in zip(ips, slabs)]
        if keys[0] is None:
            assert all(k is None for k in keys)
            return recs
        g = min(keys)
        out = [ip.apply_key(g) for ip in {id(ip): ip for ip in ips}.values()]  # once per replica
        for o in out[1:]:
            same(o, out[0])
        recs.append(out[0])


@pytest.mark.parametrize("case,world,kw", [
    (synth.small_rect(seed=81), 3, {}),
    (synth.small_rect(seed=82), 2, {"alpha": 0.5}),
    (synth.tiny(75, 64, 9, r=9), 2, {}),          # r > 8: the generic search and update kernels
    (synth.tiny(33, 27, 3, r=3), 40, {}),         # more ranks than candidate rows: empty slabs
])
def test_slabs_of_one_context_equal_the_oracle(api, case, world, kw):
    ora = oracle.run(case.rgb, case.mask, case.r, alpha=kw.get("alpha", -1.0))
    with api.Inpainter(case.rgb, case.mask, case.r, loop="graph", **kw) as ip:
        _, _, y0, y1 = ip.search_rect()
        slabs = pdist.row_slabs(y0, y1, world)
        recs = lockstep([ip] * world, slabs)
        assert len(recs) == ora.iters
        for a, b in zip(recs, ora.trace):
            same(a, b)
        assert np.array_equal(ip.result(), ora.rgb)
        assert ip.info()["evals"] == ora.evals


def test_two_replicas_stay_identical(api):
    case = synth.walkingman_like(seed=83)
    ora = oracle.run(case.rgb, case.mask, case.r, max_iters=60)
    a = api.Inpainter(case.rgb, case.mask, case.r)
    b = api.Inpainter(case.rgb, case.mask, case.r)
    with a, b:
        _, _, y0, y1 = a.search_rect()
        slabs = pdist.row_slabs(y0, y1, 2)
        recs = []
        for _ in range(60):
            ka, kb = a.search_rows(*slabs[0]), b.search_rows(*slabs[1])
            g = min(ka, kb)
            ra, rb = a.apply_key(g), b.apply_key(g)
            same(ra, rb)
            recs.append(ra)
        for x, y in zip(recs, ora.trace):
            same(x, y)
        sa, sb = a.export_state(), b.export_state()
        assert all(np.array_equal(u, v) for u, v in zip(sa, sb))
        assert np.array_equal(sa[0], ora.rgb)


def test_driver_on_one_rank(api):
    case = synth.small_rect(seed=84)
    ora = oracle.run(case.rgb, case.mask, case.r)
    with api.Inpainter(case.rgb, case.mask, case.r) as ip:
        recs = pdist.run_row_sharded(ip)
        assert len(recs) == ora.iters
        for x, y in zip(recs, ora.trace):
            same(x, y)
        assert np.array_equal(ip.result(), ora.rgb)


def test_keys_checked_and_forms_refused(api):
    case = synth.small_rect(seed=85)
    with api.Inpainter(case.rgb, case.mask, case.r) as ip:
        before = ip.export_state()
        W = case.mask.shape[1]
        for bad in (0, 3 * W + 3, (5 << 32) | (case.mask.size + 7)):  # centre not interior
            with pytest.raises(api.InpaintError) as e:
                ip.apply_key(bad)
            assert e.value.code == -1
        with pytest.raises(api.InpaintError) as e:
            ip.search_rows(10, 5)
        assert e.value.code == -1
        assert all(np.array_equal(u, v) for u, v in zip(ip.export_state(), before))
        with pytest.raises(api.InpaintError) as e:
            ip.apply_key(pdist.KEY_NONE)  # no source anywhere: nothing applied
        assert e.value.code == -4
        assert all(np.array_equal(u, v) for u, v in zip(ip.export_state(), before))
    with api.Inpainter(case.rgb, case.mask, case.r, form="tc") as ip:
        with pytest.raises(api.InpaintError) as e:
            ip.search_rows(0, 10)
        assert e.value.code == -6
    with api.Inpainter(case.rgb, case.mask, case.r, overlap=True) as ip:
        with pytest.raises(api.InpaintError) as e:
            ip.apply_key(pdist.KEY_NONE)
        assert e.value.code == -6
