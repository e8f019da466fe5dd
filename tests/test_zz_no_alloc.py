"""The allocation-free search entry point, inpaint_best_patch_noalloc.

It serves callers that cannot allocate device memory: their memory is
reserved up front by another framework's allocator, or they issue work while
a stream is captured into a graph with a fixed memory plan.  Its result must
be the best patch of the search as the oracle defines it (Sec. 3, Eq. 3-4):
the argmin of the oracle's SSD map over fully known in-image candidates,
lowest linear index on ties, packed as (SSD << 32 | index), or UINT64_MAX
when no candidate exists.  The cases cover one and several candidate tiles
per row, radii 4, 6 and 8, a target on the image border, a target without
any source, an image near the scratch limit, and two calls in a row (the
shared static scratch must carry nothing over).  This file is collected last
on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_1403_4238_gb300 import synth

pytestmark = pytest.mark.gpu

KEY_NONE = (1 << 64) - 1


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4238_gb300 import _lib, api
    return torch, _lib.load(), api


def noalloc_key(torch, lib, rgb, mask, r, px, py, prefill=-1):
    H, W = mask.shape
    d_rgb = torch.from_numpy(np.ascontiguousarray(rgb)).cuda()
    d_mask = torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    d_key = torch.full((1,), prefill, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.inpaint_best_patch_noalloc(d_rgb.data_ptr(), d_mask.data_ptr(), W, H, r, px, py,
                                        d_key.data_ptr(), stream)
    assert rc == 0, lib.inpaint_last_error()
    torch.cuda.synchronize()
    return int(d_key.cpu().numpy().view(np.uint64)[0])


def oracle_key(rgb, mask, r, px, py):
    """Argmin of the oracle's SSD map (invalid candidates hold UINT32_MAX)."""
    ssd, n_cand, _ = oracle.ssd_map(rgb, (mask != 0).astype(np.uint8), r, px, py)
    if n_cand == 0:
        return KEY_NONE
    flat = ssd.ravel().astype(np.uint64)
    valid = ssd.ravel() != np.uint32(0xFFFFFFFF)
    idx = int(np.flatnonzero(valid)[np.argmin(flat[valid])])  # first minimum: lowest index
    return (int(flat[idx]) << 32) | idx


def first_target(case):
    t = oracle.run(case.rgb, case.mask, case.r, max_iters=1).trace[0]
    return int(t["px"]), int(t["py"])


def ellipse_case(W, H, r, seed):
    return synth.Case(f"ell{W}x{H}_r{r}", synth.image(W, H, 8, 30.0, seed),
                      synth.ellipse_mask(W, H, 2, 0.03, 0.05, seed + 1), r)


@pytest.mark.parametrize("make", [
    lambda: synth.small_rect(seed=61),       # 128x96, r=4: one 128-column tile per row
    lambda: synth.walkingman_like(),         # 512x384, r=4: four tiles per row
    lambda: ellipse_case(300, 200, 6, 71),   # r=6
    lambda: ellipse_case(240, 180, 8, 73),   # r=8, the largest radius of the entry point
])
def test_noalloc_equals_oracle_argmin(env, make):
    torch, lib, _ = env
    case = make()
    px, py = first_target(case)
    assert noalloc_key(torch, lib, case.rgb, case.mask, case.r, px, py) == \
        oracle_key(case.rgb, case.mask, case.r, px, py)


def test_noalloc_target_on_the_border(env):
    torch, lib, _ = env
    case = synth.tiny(60, 44, 9, hole=(0, 0, 7, 5), r=4)
    for px, py in ((0, 0), (3, 0), (0, 4), (59, 43)):
        assert noalloc_key(torch, lib, case.rgb, case.mask, case.r, px, py) == \
            oracle_key(case.rgb, case.mask, case.r, px, py), (px, py)


def test_noalloc_without_any_source_writes_key_none(env):
    torch, lib, _ = env
    W, H, r = 96, 72, 4
    mask = np.zeros((H, W), np.uint8)
    mask[r::2 * r, r::2 * r] = 1  # every (2r+1)^2 patch holds an unknown pixel
    rgb = synth.image(W, H, 5, 30.0, 31)
    assert oracle_key(rgb, mask, r, 20, 20) == KEY_NONE
    # the output starts as another value: the kernel must write the result
    assert noalloc_key(torch, lib, rgb, mask, r, 20, 20, prefill=0x1234) == KEY_NONE


def test_noalloc_near_its_scratch_limit(env):
    torch, lib, _ = env
    # 2048 x 2048 with r = 4: 16 x 255 = 4080 candidate tiles of the 4096 allowed
    W = H = 2048
    rgb = synth.image(W, H, 6, 30.0, 81)
    mask = np.zeros((H, W), np.uint8)
    mask[1000:1012, 900:916] = 1
    px, py = 900, 1005
    assert noalloc_key(torch, lib, rgb, mask, 4, px, py) == oracle_key(rgb, mask, 4, px, py)


def test_noalloc_two_calls_in_a_row_match_the_regular_search(env):
    torch, lib, api = env
    case = synth.small_rect(seed=61)
    H, W = case.mask.shape
    with api.Inpainter(case.rgb, case.mask, case.r) as ip:
        before = ip.export_state()
        rec0 = ip.step()            # iteration 0 on the initial state
        mid = ip.export_state()
        rec1 = ip.step()            # iteration 1 on the state after one fill
    for state, rec in ((before, rec0), (mid, rec1)):   # two calls in a row
        rgb, om, _ = state
        key = noalloc_key(torch, lib, rgb, om, case.r, int(rec["px"]), int(rec["py"]))
        want = (int(rec["ssd"]) << 32) | (int(rec["qy"]) * W + int(rec["qx"]))
        assert key == want, (hex(key), hex(want))
        assert key == oracle_key(rgb, om, case.r, int(rec["px"]), int(rec["py"]))


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, lib, api = env
    d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    k = torch.zeros(1, dtype=torch.int64, device="cuda")
    # 4200 x 4200 needs more than 4096 candidate tiles: rejected before any launch
    rc = lib.inpaint_best_patch_noalloc(d.data_ptr(), d.data_ptr(), 4200, 4200, 4, 10, 10,
                                        k.data_ptr(), None)
    assert rc == -1
    assert b"scratch" in lib.inpaint_last_error()
