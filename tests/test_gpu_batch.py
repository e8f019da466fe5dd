"""Batched form: one persistent launch over many images of mixed sizes and
radii gives, for every image, exactly the single-image result (which the
parity tests tie to the oracle), and the oracle's result on small images."""
import numpy as np
import pytest

import oracle
from paper_1403_4238_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4238_gb300 import api as _api
    return _api


def mixed_cases(n, seed, wmax=200, hmax=150):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        W = int(rng.integers(40, wmax))
        H = int(rng.integers(36, hmax))
        r = int(rng.integers(1, 9))
        r = min(r, (min(W, H) - 1) // 4)
        c = synth.tiny(W, H, int(rng.integers(0, 2**31)), r=max(r, 1))
        out.append((c.rgb, c.mask, c.r))
    return out


def test_batch_equals_oracle_mixed_radii(api):
    cases = mixed_cases(12, 7)
    with api.Batch(cases) as b:
        st = b.run()
        for i, (rgb, mask, r) in enumerate(cases):
            ref = oracle.run(rgb, mask, r)
            out, iters, evals = b.result(i)
            assert st[i] == 0 and iters == ref.iters
            assert evals == ref.evals
            assert np.array_equal(out, ref.rgb), i


def test_batch_equals_solo_runs_and_reset(api):
    cases = [(c.rgb, c.mask, c.r) for c in synth.batch_cases(6, seed=11)]
    solo = []
    for rgb, mask, r in cases:
        with api.Inpainter(rgb, mask, r) as ip:
            ip.run()
            solo.append(ip.result())
    with api.Batch(cases) as b:
        plan = b.plan()
        assert sum(set(zip(plan["team"], plan["team_size"])) and plan["team_size"]) >= 1
        for rep in range(2):  # second pass after a device-side reset
            if rep:
                b.reset()
            st = b.run()
            assert all(v == 0 for v in st)
            for i in range(len(cases)):
                out, _, _ = b.result(i)
                assert np.array_equal(out, solo[i]), (rep, i)


def test_batch_more_images_than_ctas(api):
    # more images than CTAs: every CTA is a team working through a list
    cases = []
    for i in range(170):
        c = synth.tiny(20 + i % 7, 18 + i % 5, 1000 + i, r=1 + i % 2)
        cases.append((c.rgb, c.mask, c.r))
    with api.Batch(cases) as b:
        plan = b.plan()
        assert plan["teams"] == plan["grid"] and plan["grid"] < len(cases)
        st = b.run()
        assert all(v == 0 for v in st)
        for i in range(0, len(cases), 17):
            rgb, mask, r = cases[i]
            assert np.array_equal(b.result(i)[0], oracle.run(rgb, mask, r).rgb), i


def test_batch_iteration_limit_and_resume(api):
    cases = mixed_cases(5, 3)
    refs = [oracle.run(rgb, m, r) for rgb, m, r in cases]
    with api.Batch(cases) as b:
        b.run(max_iters=3)
        for i in range(len(cases)):
            assert b.result(i)[1] == min(3, refs[i].iters)
        b.run()
        for i in range(len(cases)):
            out, iters, _ = b.result(i)
            assert iters == refs[i].iters and np.array_equal(out, refs[i].rgb)


def test_batch_small_teams_with_searching_leaders(api):
    # 40 images on the GPU's CTAs: teams of a few CTAs, each with many search
    # batches, so the team leader searches its share besides the update
    rng = np.random.default_rng(21)
    cases = []
    for i in range(40):
        W, H = int(rng.integers(360, 480)), int(rng.integers(260, 340))
        s = int(rng.integers(0, 2**31))
        cases.append((synth.image(W, H, 8, 30.0, s), synth.ellipse_mask(W, H, 2, 0.01, 0.02, s + 1), 4))
    with api.Batch(cases) as b:
        plan = b.plan()
        assert plan["teams"] == 40 and max(plan["team_size"]) >= 2
        st = b.run()
        assert all(x == 0 for x in st), st
        outs = [b.result(i) for i in range(len(cases))]
    for i, (rgb, mask, r) in enumerate(cases):
        if i % 5:
            continue  # every fifth image against a single-image run, two against the oracle
        with api.Inpainter(rgb, mask, r) as ip:
            ip.run()
            assert np.array_equal(outs[i][0], ip.result()), i
            assert outs[i][2] == ip.info()["evals"], i
        if i in (0, 20):
            ref = oracle.run(rgb, mask, r)
            assert np.array_equal(outs[i][0], ref.rgb) and outs[i][1] == ref.iters, i


def test_batch_more_images_than_ctas_mixed_radii(api):
    # more images than CTAs, radii 1..8 mixed: single-CTA teams, some running
    # two images in turn
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    n = sms + 12
    cases = mixed_cases(n, 33, wmax=72, hmax=60)
    with api.Batch(cases) as b:
        plan = b.plan()
        assert plan["teams"] == plan["grid"] and max(plan["team_size"]) == 1
        st = b.run()
        assert all(x in (0, 1) for x in st), st
        for i in range(0, n, 17):
            rgb, mask, r = cases[i]
            ref = oracle.run(rgb, mask, r)
            out, iters, evals = b.result(i)
            assert iters == ref.iters and evals == ref.evals
            assert np.array_equal(out, ref.rgb), i


def lattice_case(W=96, H=72, r=4, seed=21):
    """Unknown pixels on a lattice of pitch 2r: every (2r+1)^2 patch holds
    one, so no candidate is fully known and the first search finds none."""
    rgb = synth.image(W, H, 5, 30.0, seed)
    mask = np.zeros((H, W), np.uint8)
    mask[r::2 * r, r::2 * r] = 1
    return rgb, mask, r


def test_batch_image_without_source_fails_alone(api):
    cases = [(c.rgb, c.mask, c.r) for c in synth.batch_cases(4, seed=12)]
    bad = lattice_case()
    assert oracle.run(*bad).status == -4
    cases.insert(2, bad)
    solo = {}
    for i, (rgb, mask, r) in enumerate(cases):
        if i != 2:
            with api.Inpainter(rgb, mask, r) as ip:
                ip.run()
                solo[i] = ip.result()
    with api.Batch(cases) as b:
        st = b.run()
        assert st[2] == -4
        for i in solo:
            assert st[i] == 0, i
            assert np.array_equal(b.result(i)[0], solo[i]), i


def test_one_shot_batch_run_equals_oracle(api):
    # the one-shot C entry point (create, run, results, destroy in one call)
    cases = mixed_cases(6, 41)
    outs, st = api.batch_run(cases)
    assert st == [0] * len(cases)
    for i, (rgb, mask, r) in enumerate(cases):
        assert np.array_equal(outs[i], oracle.run(rgb, mask, r).rgb), i
    # an image without a source fails alone inside the one-shot call
    bad = lattice_case()
    outs, st = api.batch_run(cases[:2] + [bad])
    assert st[:2] == [0, 0] and st[2] == -4
    assert np.array_equal(outs[1], oracle.run(*cases[1]).rgb)
