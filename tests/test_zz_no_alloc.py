"""The allocation-free search entry point against the library's own search.

inpaint_best_patch_noalloc serves callers that cannot allocate device memory
(their memory is reserved up front by another framework, or they issue work
while a stream is captured with a fixed memory plan).  Its result must be
the one the regular entry point finds for the same target: the source patch
and SSD that inpaint_step reports for its iteration, bit for bit.  Two calls
in a row check that the shared static scratch carries nothing over between
calls.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1403_4238_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4238_gb300 import _lib, api
    return torch, _lib.load(), api


def noalloc_key(torch, lib, rgb, mask, r, px, py):
    H, W = mask.shape
    d_rgb = torch.from_numpy(np.ascontiguousarray(rgb)).cuda()
    d_mask = torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    d_key = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.inpaint_best_patch_noalloc(d_rgb.data_ptr(), d_mask.data_ptr(), W, H, r, px, py,
                                        d_key.data_ptr(), stream)
    assert rc == 0, lib.inpaint_last_error()
    torch.cuda.synchronize()
    return int(d_key.cpu().numpy().view(np.uint64)[0])


def test_noalloc_matches_regular_search_two_calls(env):
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


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, lib, api = env
    d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    k = torch.zeros(1, dtype=torch.int64, device="cuda")
    # 4200 x 4200 needs more than 4096 candidate tiles: rejected before any launch
    rc = lib.inpaint_best_patch_noalloc(d.data_ptr(), d.data_ptr(), 4200, 4200, 4, 10, 10,
                                        k.data_ptr(), None)
    assert rc == -1
    assert b"scratch" in lib.inpaint_last_error()
