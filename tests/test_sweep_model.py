"""Host logic of the patch-size / search-factor sweep (Sec. 5.3-5.4).

Eq. 8 is pinned by hand-evaluated values and by its special cases; the
Table-3-shaped inputs by the sizes and object boxes printed in Table 3.
"""
import numpy as np
import pytest

from paper_1403_4238_gb300 import sweep, synth


def test_eq8_hand_value():
    # w = h = 10, P = 3, alpha = 1, k = 0.5:
    # 10^2 * 10^2 * (3^2 - 0.5 * (2*2/10 + 1)^2 - 0.5) = 10^4 * (9 - 0.98 - 0.5) = 75200
    assert sweep.eq8_complexity(10, 10, 3, 1.0, 0.5) == pytest.approx(75200.0, rel=1e-12)
    # k = 0: 10^4 * (9 - 1.96) = 70400
    assert sweep.eq8_complexity(10, 10, 3, 1.0, 0.0) == pytest.approx(70400.0, rel=1e-12)


def test_eq8_special_cases():
    w, h = 78, 126
    # k = 1: every candidate costs P^2 -> w^2 h^2 ((2a+1)^2 - 1) = wh * SA (Eq. 7), P-free
    for P in (9, 13, 17):
        assert sweep.eq8_complexity(w, h, P, 0.5, 1.0) == pytest.approx(w * h * ((2 * 0.5 + 1) ** 2 - 1) * w * h)
    # k < 1: a larger patch lowers the estimate, by the same absolute amount for every alpha
    d1 = sweep.eq8_complexity(w, h, 9, 0.1) - sweep.eq8_complexity(w, h, 17, 0.1)
    d2 = sweep.eq8_complexity(w, h, 9, 2.0) - sweep.eq8_complexity(w, h, 17, 2.0)
    assert d1 > 0 and d1 == pytest.approx(d2)
    # so the relative gain of a larger patch shrinks as alpha grows (the trend of Fig. 9)
    r_small = sweep.eq8_complexity(w, h, 17, 0.1) / sweep.eq8_complexity(w, h, 9, 0.1)
    r_big = sweep.eq8_complexity(w, h, 17, 2.0) / sweep.eq8_complexity(w, h, 9, 2.0)
    assert r_small < r_big < 1.0


@pytest.mark.parametrize("name,W,H,w,h", [
    ("walkingman", 512, 384, 78, 126), ("river", 480, 639, 59, 93),
    ("divingman", 576, 384, 155, 186), ("hill", 1024, 550, 1024, 10),
])
def test_table3_shapes(name, W, H, w, h):
    c = synth.table3_case(name, 4)
    assert c.rgb.shape == (H, W, 3) and c.mask.shape == (H, W)
    assert sweep.object_box(c.mask) == (w, h)
    c2 = synth.table3_case(name, 4)
    assert np.array_equal(c.rgb, c2.rgb) and np.array_equal(c.mask, c2.mask)  # seeded
