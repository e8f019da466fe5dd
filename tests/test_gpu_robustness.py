"""Robustness of the CUDA path: allocation failures and the bytes under Omega.

* Every device allocation of a context goes through inpaint_options.dev_alloc
  when it is given.  Failing each one in turn must give INPAINT_ERR_NOMEM,
  free everything allocated so far (create) or leave a context that finishes
  the removal like the oracle once memory is available again (the engine's
  buffers, allocated at the first run), and leak nothing after destroy.
* The pixels of the target region are unknown (Sec. 3): the result must not
  depend on the bytes the input holds there, on the GPU as in the oracle.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1403_4238_gb300 import synth

pytestmark = pytest.mark.gpu

NOMEM = -2


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


class FailingAllocator:
    """dev_alloc/dev_free over PyTorch's caching allocator whose allocation
    number `fail_at` (0-based, counted from the last reset) returns NULL."""

    def __init__(self, torch):
        from paper_1403_4238_gb300 import _lib
        dev = torch.cuda.current_device()
        self.live, self.errors = {}, []
        self.calls, self.fail_at = 0, -1

        def alloc(nbytes, stream, user):
            k = self.calls
            self.calls += 1
            if k == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
            self.live[int(p)] = int(nbytes)
            return p

        def free(ptr, nbytes, stream, user):
            if self.live.pop(int(ptr), None) != int(nbytes):
                self.errors.append((ptr, nbytes))
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = _lib.ALLOC_FN(alloc)
        self.free = _lib.FREE_FN(free)

    def reset(self, fail_at=-1):
        self.calls, self.fail_at = 0, fail_at


def test_every_allocation_failure_is_reported_and_leaks_nothing(torch):
    from paper_1403_4238_gb300 import _lib
    lib = _lib.load()
    case = synth.small_rect(seed=61)
    ora = oracle.run(case.rgb, case.mask, case.r)
    H, W = case.mask.shape
    rgb = np.ascontiguousarray(case.rgb)
    mask = np.ascontiguousarray(case.mask)
    fa = FailingAllocator(torch)
    stream = torch.cuda.Stream()

    def create():
        opt = _lib.Options()
        lib.inpaint_options_default(ctypes.byref(opt))
        opt.cuda_stream = stream.cuda_stream
        opt.dev_alloc, opt.dev_free = fa.alloc, fa.free
        ctx = ctypes.c_void_p()
        rc = lib.inpaint_create(rgb.ctypes.data, W, H, 3 * W, mask.ctypes.data, W, case.r,
                                ctypes.byref(opt), ctypes.byref(ctx))
        return rc, ctx, opt

    def run(ctx):
        done = ctypes.c_int()
        return lib.inpaint_run(ctx, 0, ctypes.byref(done), None, 0)

    def result(ctx):
        out = np.zeros((H, W, 3), np.uint8)
        assert lib.inpaint_result(ctx, out.ctypes.data, 3 * W, None) == 0
        return out

    # count the allocations of create and of the first run (the engine's)
    fa.reset()
    rc, ctx, opt = create()
    assert rc == 0
    n_create = fa.calls
    assert run(ctx) == 0
    n_total = fa.calls
    assert np.array_equal(result(ctx), ora.rgb)
    lib.inpaint_destroy(ctx)
    assert n_create > 0 and n_total > n_create
    assert not fa.live and not fa.errors

    for k in range(n_total):
        fa.reset(k)
        rc, ctx, opt = create()
        if k < n_create:
            assert rc == NOMEM and not ctx.value, k
            assert not fa.live, k  # create released what it had
            continue
        assert rc == 0, k
        assert run(ctx) == NOMEM, k
        fa.reset()  # memory available again: the same context finishes the removal
        assert run(ctx) == 0, k
        assert np.array_equal(result(ctx), ora.rgb), k
        lib.inpaint_destroy(ctx)
        assert not fa.live, k
    assert not fa.errors


@pytest.mark.parametrize("loop", ["engine", "graph"])
def test_result_independent_of_bytes_under_the_mask(torch, loop):
    from paper_1403_4238_gb300 import api
    case = synth.small_rect(seed=62)
    hole = case.mask != 0
    noisy = case.rgb.copy()
    noisy[hole] = np.random.default_rng(63).integers(0, 256, (int(hole.sum()), 3), dtype=np.uint8)
    zero = case.rgb.copy()
    zero[hole] = 0
    ora = oracle.run(case.rgb, case.mask, case.r)
    outs = []
    for rgb in (noisy, zero):
        with api.Inpainter(rgb, case.mask, case.r, loop=loop) as ip:
            rc, n, tr = ip.run(trace=True)
            assert rc == 0 and n == ora.iters
            outs.append((ip.result(), tr))
    for out, tr in outs:
        assert np.array_equal(out, ora.rgb)
        assert np.array_equal(tr["ssd"], ora.trace["ssd"][: len(tr)])
        assert np.array_equal(tr["qx"], ora.trace["qx"][: len(tr)])
