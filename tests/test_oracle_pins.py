"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Sec. 3 (Eq. 1-4) defines the method.  The paper prints no worked example,
so the oracle is pinned by:
  * hand-derived priorities on few-pixel fronts (tests/golden/priority_pins.json);
  * an independent numpy brute force (tests/brute.py) of the front, the SSD
    map, the argmin with lowest-index ties, and the whole loop on tiny images;
  * planted exact copies (SSD 0 at a unique place), periodic images (many
    SSD-0 ties resolved to the lowest index), special cases (single unknown
    pixel, flat image, mask on the border), and run invariants.
"""
import json
import math
import os

import numpy as np
import pytest

import brute
import oracle
from paper_1403_4238_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mk_gray(spec, W, H):
    ys, xs = np.mgrid[0:H, 0:W]
    if spec.startswith("flat"):
        return np.full((H, W), int(spec.split()[1]), np.int64)
    return eval(spec, {}, {"x": xs, "y": ys})  # recipes like "10*y", "7*x+3*y"


def _mk_omega(spec, W, H):
    ys, xs = np.mgrid[0:H, 0:W]
    if isinstance(spec, list):
        om = np.zeros((H, W), np.uint8)
        for x, y in spec:
            om[y, x] = 1
        return om
    return eval(spec, {}, {"x": xs, "y": ys}).astype(np.uint8)


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "priority_pins.json")))["cases"],
                         ids=lambda c: c["name"][:40])
def test_priority_hand_derived(case):
    W, H, r = case["W"], case["H"], case["r"]
    g = _mk_gray(case["gray"], W, H)
    om = _mk_omega(case["omega"], W, H)
    rgb = np.repeat(g[..., None], 3, axis=2).astype(np.uint8)
    gray = brute.luma(rgb)  # R=G=B=v has luma v
    assert np.array_equal(gray, g)
    conf = np.where(om == 1, 0.0, 1.0)
    x, y = case["p"]
    assert oracle.front(om)[y, x] == 1
    c = case["c_num"] / case["c_den"]
    nx, ny, gx, gy = case["nx"], case["ny"], case["gx"], case["gy"]
    nn = nx * nx + ny * ny
    d = 0.0 if nn == 0 else (abs(-gy * nx + gx * ny) / math.sqrt(nn)) / 510.0
    p, co, do = oracle.priority(gray.astype(np.uint8), conf, om, r, x, y)
    assert co == c and do == d and p == c * d, (p, co, do, c, d)
    # independent brute force agrees bit for bit as well
    pb, cb, db = brute.priority(gray, conf, om, r, x, y)
    assert (pb, cb, db) == (p, co, do)


def test_confidence_sum_row_major_hand_derived():
    # The summation order: row-major, dy outer, dx inner, one addition at a
    # time.  A 3x3 patch where it matters: row 0 = (1, u, u), row 1 =
    # (u, p, u), row 2 = (0, 0, 0), u = 2^-53.  Row-major: 1 + u is a tie
    # and rounds to even (1), and so does every later + u, so the sum is 1
    # and C = 1/9.  Summing each row first would give 1 + 2^-52 instead
    # (row 1 = 2u exactly).  |Psi_p| = 9 in-image pixels.
    u = 2.0 ** -53
    conf = np.array([[1.0, u, u], [u, 0.0, u], [0.0, 0.0, 0.0]])
    om = np.zeros((3, 3), np.uint8)
    om[1, 1] = 1
    gray = np.zeros((3, 3), np.uint8)
    assert oracle.front(om)[1, 1] == 1
    _, c, _ = oracle.priority(gray, conf, om, 1, 1, 1)
    assert c == 1.0 / 9.0
    assert c != (1.0 + 2.0 ** -52) / 9.0  # the rows-first value
    _, cb, _ = brute.priority(gray.astype(np.int64), conf, om, 1, 1, 1)
    assert cb == c


def test_confidence_sum_fractional_against_brute_and_bound():
    # fractional confidences (as after fills): the oracle and the brute force
    # agree bit for bit, and the sum is within the recursive-summation bound
    # (n - 1) eps sum|c| of the exact sum (math.fsum), which a dropped or
    # doubled term or a wrong index would break
    rng = np.random.default_rng(17)
    eps = 2.0 ** -53
    for r in (1, 4, 6, 8):
        H, W = 3 * r + 5, 3 * r + 7
        for _ in range(40):
            conf = rng.random((H, W)) ** 3
            om = (rng.random((H, W)) < 0.35).astype(np.uint8)
            gray = rng.integers(0, 256, (H, W)).astype(np.uint8)
            x, y = int(rng.integers(0, W)), int(rng.integers(0, H))
            _, c, _ = oracle.priority(gray, conf, om, r, x, y)
            _, cb, _ = brute.priority(gray.astype(np.int64), conf, om, r, x, y)
            assert c == cb
            vals = [float(conf[yy, xx]) for yy in range(max(0, y - r), min(H, y + r + 1))
                    for xx in range(max(0, x - r), min(W, x + r + 1)) if not om[yy, xx]]
            n_in = (min(W - 1, x + r) - max(0, x - r) + 1) * (min(H - 1, y + r) - max(0, y - r) + 1)
            exact = math.fsum(vals)
            bound = (len(vals) + 1) * eps * exact + 1e-300
            assert abs(c * n_in - exact) <= bound + eps * n_in * c


def test_gray_bt601_values():
    # 0.299*255 = 76.2, 0.587*255 = 149.7, 0.114*255 = 29.1 rounded to nearest
    assert oracle.gray(255, 0, 0) == 76
    assert oracle.gray(0, 255, 0) == 150
    assert oracle.gray(0, 0, 255) == 29
    assert oracle.gray(255, 255, 255) == 255
    assert oracle.gray(0, 0, 0) == 0
    rng = np.random.default_rng(0)
    px = rng.integers(0, 256, (500, 3))
    for rr, gg, bb in px:
        assert oracle.gray(rr, gg, bb) == int(round(0.299 * rr + 0.587 * gg + 0.114 * bb + 1e-9))


@pytest.mark.parametrize("seed", range(6))
def test_front_matches_bruteforce(seed):
    c = synth.tiny(17, 13, seed)
    om = c.mask.copy()
    om[0, :] |= (np.arange(17) % 3 == 0).astype(np.uint8)  # touch the border
    assert np.array_equal(oracle.front(om), brute.front(om))


@pytest.mark.parametrize("seed,r,W,H", [(0, 1, 8, 8), (1, 2, 16, 12), (2, 1, 24, 16), (3, 2, 19, 23),
                                         (4, 3, 20, 18), (5, 1, 9, 30)])
def test_ssd_map_matches_bruteforce(seed, r, W, H):
    c = synth.tiny(W, H, seed, r=r)
    om = c.mask
    ys, xs = np.nonzero(brute.front(om))
    for k in range(0, len(xs), max(1, len(xs) // 5)):
        px, py = int(xs[k]), int(ys[k])
        a, nc_a, nk_a = oracle.ssd_map(c.rgb, om, r, px, py)
        b, nc_b, nk_b = brute.ssd_map(c.rgb, om, r, px, py)
        assert np.array_equal(a, b)
        assert (nc_a, nk_a) == (nc_b, nk_b)


@pytest.mark.parametrize("seed,r,W,H", [(10, 1, 8, 8), (11, 2, 16, 12), (12, 1, 24, 16), (13, 2, 19, 23),
                                         (14, 3, 20, 18), (15, 1, 9, 30)])
def test_ssd_map_overlap_matches_bruteforce(seed, r, W, H):
    # partial-overlap variant (Alg. 1, Sec. 5.4): candidates may overlap Omega
    # and cross the image border
    c = synth.tiny(W, H, seed, r=r)
    om = c.mask
    ys, xs = np.nonzero(brute.front(om))
    for k in range(0, len(xs), max(1, len(xs) // 5)):
        px, py = int(xs[k]), int(ys[k])
        for rect in (None, (2, W - 3, 1, H - 2)):
            a, nc_a, nk_a = oracle.ssd_map(c.rgb, om, r, px, py, rect=rect, overlap=True)
            b, nc_b, nk_b = brute.ssd_map_overlap(c.rgb, om, r, px, py, rect=rect)
            assert np.array_equal(a, b)
            assert (nc_a, nk_a) == (nc_b, nk_b)


def test_overlap_variant_admits_exactly_the_covering_candidates():
    # 12 x 10 image, r = 1, one unknown pixel at (5, 5); target p^ = (5, 5)
    rng = np.random.default_rng(3)
    rgb = rng.integers(0, 256, (10, 12, 3)).astype(np.uint8)
    om = np.zeros((10, 12), np.uint8)
    om[5, 5] = 1
    out, nc, nk = oracle.ssd_map(rgb, om, 1, 5, 5, overlap=True)
    assert nk == 8
    # every centre but the unknown pixel itself covers it with a known pixel
    assert nc == 12 * 10 - 1 and out[5, 5] == 2**32 - 1
    # a candidate next to the hole compares 7 pairs (its own (5, 5) pixel is unknown)
    qx, qy = 6, 5
    want = 0
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if (dx, dy) == (0, 0) or (qx + dx, qy + dy) == (5, 5):
                continue
            d = rgb[5 + dy, 5 + dx].astype(np.int64) - rgb[qy + dy, qx + dx].astype(np.int64)
            want += int((d * d).sum())
    assert out[qy, qx] == want
    # a corner centre compares only the in-image pairs
    d = rgb[5:7, 5:7].astype(np.int64) - rgb[0:2, 0:2].astype(np.int64)
    d[0, 0] = 0  # target (5, 5) is unknown
    assert out[0, 0] == int((d * d).sum())
    # the default variant keeps only interior, fully known candidates
    out0, nc0, _ = oracle.ssd_map(rgb, om, 1, 5, 5)
    assert nc0 == 10 * 8 - 9 and out0[0, 0] == 2**32 - 1


def test_overlap_variant_loop_invariants():
    c = synth.small_rect(seed=5)
    res = oracle.run(c.rgb, c.mask, c.r, overlap=True)
    assert res.status == 0 and res.mask.sum() == 0
    assert np.array_equal(res.rgb[c.mask == 0], c.rgb[c.mask == 0])  # known pixels never change
    # each fill copies pixels that were known at that time: replaying the trace
    # on the input reproduces the result
    img = c.rgb.copy()
    om = c.mask.astype(bool).copy()
    r = c.r
    for t in res.trace:
        px, py, qx, qy = int(t["px"]), int(t["py"]), int(t["qx"]), int(t["qy"])
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                tx, ty = px + dx, py + dy
                if 0 <= tx < c.W and 0 <= ty < c.H and om[ty, tx]:
                    assert not om[qy + dy, qx + dx]
                    img[ty, tx] = img[qy + dy, qx + dx]
                    om[ty, tx] = False
    assert np.array_equal(img, res.rgb)


def test_planted_copy_found_exactly():
    rng = np.random.default_rng(7)
    W, H, r = 40, 30, 2
    rgb = rng.integers(0, 256, (H, W, 3)).astype(np.uint8)
    om = np.zeros((H, W), np.uint8)
    om[10:14, 10:14] = 1
    px, py = 10, 12  # on the front
    qx, qy = 31, 22
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            if not om[py + dy, px + dx]:
                rgb[qy + dy, qx + dx] = rgb[py + dy, px + dx]
    ssd, nc, nk = oracle.ssd_map(rgb, om, r, px, py)
    assert ssd[qy, qx] == 0
    assert brute.argmin_lowest(ssd.astype(np.int64)) == qy * W + qx
    assert np.count_nonzero(ssd == 0) == 1


def test_periodic_ties_go_to_lowest_index():
    # period-4 tile pattern: every candidate shifted by a multiple of 4 ties
    W, H, r = 32, 24, 1
    rng = np.random.default_rng(3)
    tile = rng.integers(0, 256, (4, 4, 3)).astype(np.uint8)
    rgb = np.tile(tile, (H // 4, W // 4, 1))
    om = np.zeros((H, W), np.uint8)
    om[12:15, 16:19] = 1
    px, py = 16, 13
    ssd, _, _ = oracle.ssd_map(rgb, om, r, px, py)
    zeros = np.flatnonzero(ssd.reshape(-1) == 0)
    assert len(zeros) > 5
    q = brute.argmin_lowest(ssd.astype(np.int64))
    assert q == zeros[0]
    res = oracle.run(rgb, om, r, max_iters=1)
    t = res.trace[0]
    ssd1, _, _ = brute.ssd_map(rgb, om, r, int(t["px"]), int(t["py"]))
    assert int(t["qy"]) * W + int(t["qx"]) == int(np.flatnonzero(ssd1.reshape(-1) == 0)[0])
    assert t["ssd"] == 0


def test_ssd_is_exact_at_the_bound():
    # all-255 target against all-0 source: SSD = |K| * 3 * 255^2 exactly
    W, H, r = 30, 30, 6
    rgb = np.zeros((H, W, 3), np.uint8)
    rgb[:, :15] = 255
    om = np.zeros((H, W), np.uint8)
    om[12:18, 6:9] = 1
    ssd, nc, nk = oracle.ssd_map(rgb, om, r, 6, 15)
    # candidate centred at x = 23 lies wholly in the black half
    assert ssd[15, 23] == nk * 3 * 255 * 255
    assert nk == 13 * 13 - 3 * 6 - 0  # 13x13 patch minus the in-patch hole part


@pytest.mark.parametrize("seed,W,H,r", [(10, 12, 10, 1), (11, 14, 12, 2), (12, 16, 12, 1),
                                         (13, 18, 14, 2), (14, 20, 16, 1), (15, 13, 17, 2)])
def test_whole_loop_matches_bruteforce(seed, W, H, r):
    c = synth.tiny(W, H, seed, r=r)
    res = oracle.run(c.rgb, c.mask, r)
    st, img, om, conf, tr = brute.run(c.rgb, c.mask, r)
    assert res.status == st
    assert len(tr) == res.iters
    for a, b in zip(res.trace, tr):
        for k, v in b.items():
            assert a[k] == v, (k, a[k], v)
    assert np.array_equal(res.rgb, img)
    assert np.array_equal(res.mask, om)
    assert np.array_equal(res.conf, conf)


def test_single_unknown_pixel_is_one_iteration():
    c = synth.tiny(15, 11, 21, hole=(7, 5, 1, 1), r=2)
    res = oracle.run(c.rgb, c.mask, 2)
    assert res.status == 0 and res.iters == 1
    t = res.trace[0]
    assert (t["px"], t["py"], t["filled"], t["remaining"]) == (7, 5, 1, 0)
    assert res.rgb[5, 7].tolist() == c.rgb[t["qy"], t["qx"]].tolist()


def test_flat_image_fill_order_is_lowest_index():
    W, H, r = 20, 16, 2
    rgb = np.full((H, W, 3), 90, np.uint8)
    om = np.zeros((H, W), np.uint8)
    om[5:9, 6:11] = 1
    res = oracle.run(rgb, om, r)
    f = brute.front(om)
    first = int(np.flatnonzero(f.reshape(-1))[0])
    assert res.trace[0]["priority"] == 0.0
    assert res.trace[0]["py"] * W + res.trace[0]["px"] == first
    # every SSD is 0, so the lowest valid candidate index wins each time
    assert all(int(t["ssd"]) == 0 for t in res.trace)


def test_mask_touching_border():
    c = synth.tiny(24, 18, 31, hole=(0, 0, 5, 4), r=2)
    res = oracle.run(c.rgb, c.mask, 2)
    st, img, om, conf, tr = brute.run(c.rgb, c.mask, 2)
    assert res.status == st == 0
    assert np.array_equal(res.rgb, img)
    assert [t["px"] for t in res.trace] == [t["px"] for t in tr]


def test_status_codes():
    c = synth.tiny(12, 12, 1, r=1)
    empty = np.zeros_like(c.mask)
    assert oracle.run(c.rgb, empty, 1).status == oracle.DONE
    full = np.ones_like(c.mask)
    assert oracle.run(c.rgb, full, 1).status == oracle.ERR_ARG
    assert oracle.run(c.rgb[:2, :2], c.mask[:2, :2], 1).status == oracle.ERR_ARG
    # hole so large that no fully-known 5x5 patch exists
    m = np.ones((12, 12), np.uint8)
    m[0, 0] = 0
    res = oracle.run(c.rgb, m, 2)
    assert res.status == oracle.ERR_NO_SOURCE and res.iters == 0


def _invariants(case, res):
    W = case.W
    om0 = case.mask != 0
    # known pixels never altered
    assert np.array_equal(res.rgb[~om0], case.rgb[~om0])
    assert res.mask.sum() == 0
    rem = [int(t["remaining"]) for t in res.trace]
    assert all(a > b for a, b in zip([int(om0.sum())] + rem, rem))  # strictly shrinking
    assert res.iters <= int(om0.sum())
    assert sum(int(t["filled"]) for t in res.trace) == int(om0.sum())
    assert res.evals == sum(int(t["n_cand"]) * int(t["n_known"]) for t in res.trace)


def test_invariants_config_small_rect():
    case = synth.small_rect()
    res = oracle.run(case.rgb, case.mask, case.r)
    assert res.status == 0
    _invariants(case, res)
    # replay: each filled pixel equals its source pixel and each SSD is the
    # minimum of an independent brute-force map of the pre-iteration state
    img = case.rgb.copy()
    om = (case.mask != 0).astype(np.uint8)
    r = case.r
    for t in res.trace:
        ssd, nc, nk = brute.ssd_map(img, om, r, int(t["px"]), int(t["py"]))
        q = brute.argmin_lowest(ssd.astype(np.int64))
        assert q == int(t["qy"]) * case.W + int(t["qx"])
        assert int(ssd.reshape(-1)[q]) == int(t["ssd"]) and nc == t["n_cand"] and nk == t["n_known"]
        px, py, qx, qy = (int(t[k]) for k in ("px", "py", "qx", "qy"))
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                x, y = px + dx, py + dy
                if 0 <= x < case.W and 0 <= y < case.H and om[y, x]:
                    img[y, x] = img[qy + dy, qx + dx]
                    om[y, x] = 0
                    assert res.rgb[y, x].tolist() == img[y, x].tolist()
    assert np.array_equal(img, res.rgb)


def test_result_independent_of_bytes_under_mask():
    case = synth.small_rect()
    a = oracle.run(case.rgb, case.mask, case.r)
    scrambled = case.rgb.copy()
    rng = np.random.default_rng(99)
    sel = case.mask != 0
    scrambled[sel] = rng.integers(0, 256, (int(sel.sum()), 3)).astype(np.uint8)
    b = oracle.run(scrambled, case.mask, case.r)
    assert np.array_equal(a.rgb, b.rgb)
    assert np.array_equal(a.trace, b.trace)


def test_run_from_state_continues_a_run():
    case = synth.small_rect()
    full = oracle.run(case.rgb, case.mask, case.r)
    part = oracle.run(case.rgb, case.mask, case.r, max_iters=5)
    rest = oracle.run_from_state(part.rgb, part.mask, part.conf, case.r)
    assert np.array_equal(rest.rgb, full.rgb)
    got = [(int(t["px"]), int(t["py"]), int(t["qx"]), int(t["qy"])) for t in rest.trace]
    want = [(int(t["px"]), int(t["py"]), int(t["qx"]), int(t["qy"])) for t in full.trace[5:]]
    assert got == want


def test_search_rect_alpha():
    m = np.zeros((60, 80), np.uint8)
    m[20:30, 30:50] = 1  # w = 20, h = 10
    assert oracle.search_rect(m, 4, -1.0) == (4, 75, 4, 55)
    # floor(0.25*20) = 5, floor(0.25*10) = 2
    assert oracle.search_rect(m, 4, 0.25) == (25, 54, 18, 31)
    assert oracle.search_rect(m, 4, 10.0) == (4, 75, 4, 55)  # clamped to the interior
    c = synth.tiny(30, 24, 5, hole=(12, 9, 5, 5), r=2)
    rect = oracle.search_rect(c.mask, 2, 0.6)
    a, nca, _ = oracle.ssd_map(c.rgb, c.mask, 2, 12, 10, rect)
    b, ncb, _ = brute.ssd_map(c.rgb, c.mask, 2, 12, 10, rect)
    assert np.array_equal(a, b) and nca == ncb
