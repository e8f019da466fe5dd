"""Failure detection on the GPU without a fault: the persistent engine's
bounded waits.

The failure is injected on the host: one searcher CTA of the team is told not
to report its key.  The team's leader must give up waiting for the keys after
the short limit, apply nothing, and stop every CTA of the team; the call must
return INPAINT_ERR_TIMEOUT (-5) quickly, leave the removal state exactly as
it was before the interrupted iteration, and the same context must then
finish the removal bit for bit like the oracle (Sec. 3, Eq. 1-4).
"""
import ctypes
import time

import numpy as np
import pytest

import oracle
from paper_1403_4238_gb300 import synth

pytestmark = pytest.mark.gpu

TIMEOUT = -5
LIMIT_S = 0.05


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4238_gb300 import api as _api
    return _api


def withheld(ip, rank, limit_s=LIMIT_S, max_iters=0):
    done = ctypes.c_int(-1)
    t0 = time.perf_counter()
    rc = ip.lib.inpaint_run_withheld(ip.ctx, rank, limit_s, max_iters, ctypes.byref(done))
    return rc, done.value, time.perf_counter() - t0


def states_equal(a, b):
    return (np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and
            np.array_equal(a[2].view(np.uint64), b[2].view(np.uint64)))


@pytest.mark.parametrize("tile_rows", [1, 2])
def test_withheld_key_times_out_and_the_context_recovers(api, tile_rows):
    case = synth.small_rect(seed=51)
    ora = oracle.run(case.rgb, case.mask, case.r)
    k = 5
    with api.Inpainter(case.rgb, case.mask, case.r, loop="engine", tile_rows=tile_rows) as ip:
        rc, n, _ = ip.run(max_iters=k)
        assert rc == 0 and n == k
        before = ip.export_state()
        rc, done, dt = withheld(ip, 0)
        assert rc == TIMEOUT and done == 0
        assert dt < 2.0  # the 50 ms limit, not the normal 4 s one
        assert states_equal(ip.export_state(), before)
        # twice in a row: the limit and the reporting were restored in between
        rc, done, _ = withheld(ip, 0)
        assert rc == TIMEOUT and done == 0
        rc, n, tr = ip.run(trace=True)
        assert rc == 0 and k + n == ora.iters
        for i in range(n):
            g, o = tr[i], ora.trace[k + i]
            assert (g["iter"], g["px"], g["py"], g["qx"], g["qy"], g["ssd"]) == \
                (o["iter"], o["px"], o["py"], o["qx"], o["qy"], o["ssd"]), i
        assert np.array_equal(ip.result(), ora.rgb)
        assert ip.info()["evals"] == ora.evals


def test_rank_that_does_not_search_changes_nothing(api):
    case = synth.small_rect(seed=52)
    ora = oracle.run(case.rgb, case.mask, case.r)
    with api.Inpainter(case.rgb, case.mask, case.r, loop="engine") as ip:
        rc, done, _ = withheld(ip, 1 << 20, limit_s=2.0)
        assert rc == 0 and done == ora.iters
        assert np.array_equal(ip.result(), ora.rgb)


def test_withheld_needs_the_engine(api):
    case = synth.small_rect(seed=53)
    with api.Inpainter(case.rgb, case.mask, case.r, loop="graph") as ip:
        assert withheld(ip, 0)[0] == -6
        assert ip.lib.inpaint_run_withheld(ip.ctx, 0, 20.0, 0, None) == -1  # limit above 10 s
