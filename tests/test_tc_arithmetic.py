"""The exactness argument of the tensor-core search form, checked on the CPU.

The form computes each SSD of Eq. 4 as A2 - 2X + S: A2 = sum over the known
target pixels of |t - 128|^2, X = sum of (t - 128)(s - 128) per channel, and
S = sum over the same offsets of |s - 128|^2, split as 256 hi + lo with
hi, lo in [0, 255].  The operands are BF16, the accumulators FP32, and the
read-back takes fl(fl(S - 2X) + A2), falling back to integers when that is
not below 2^24.  These tests pin each step with numpy: BF16 holds every
operand exactly, the expansion equals the direct SSD, every FP32 partial
sum stays below 2^24 (so the accumulation is exact in any order), and the
read-back is exact below 2^24 and never below it otherwise.
"""
import numpy as np

R_MAX = 8
P_MAX = 2 * R_MAX + 1
TWO24 = float(1 << 24)


def to_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to BF16 (nearest, ties to even), back as float32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32)


def test_bf16_holds_every_operand():
    d = np.arange(-128, 128, dtype=np.float32)  # shifted channel values
    assert np.array_equal(to_bf16(d), d)
    sq = np.arange(0, 3 * 128 * 128 + 1)  # squared norms of shifted RGB
    hi = (sq & ~255).astype(np.float32)
    lo = (sq & 255).astype(np.float32)
    assert np.array_equal(to_bf16(hi), hi) and np.array_equal(to_bf16(lo), lo)
    assert np.array_equal(hi + lo, sq.astype(np.float32))
    assert np.array_equal(to_bf16(np.array([0.0, 1.0], np.float32)), [0.0, 1.0])  # the mask


def test_expansion_equals_direct_ssd():
    rng = np.random.default_rng(7)
    for P in (3, 9, 13, 17):
        for _ in range(200):
            t = rng.integers(0, 256, (P, P, 3))
            s = rng.integers(0, 256, (P, P, 3))
            m = rng.random((P, P)) < 0.6
            direct = int((((t - s) ** 2).sum(axis=-1) * m).sum())
            a = t - 128
            b = s - 128
            a2 = int(((a ** 2).sum(axis=-1) * m).sum())
            x = int(((a * b).sum(axis=-1) * m).sum())
            sq = (b ** 2).sum(axis=-1)
            S = int(((sq & ~255) * m).sum() + ((sq & 255) * m).sum())
            assert a2 - 2 * x + S == direct


def test_accumulators_stay_below_two_to_24():
    # largest magnitudes any partial sum can reach at the largest patch
    n = P_MAX * P_MAX
    x_max = 3 * n * 128 * 128          # |sum of (t-128)(s-128)| over 3 channels
    s_max = n * 3 * 128 * 128          # sum of |s - 128|^2
    a2_max = n * 3 * 128 * 128
    assert max(x_max, s_max, a2_max) < TWO24
    # so the integer-valued partial sums are exact in FP32 whatever the order
    rng = np.random.default_rng(8)
    vals = rng.integers(-128 * 128, 128 * 128 + 1, 3 * n).astype(np.float32)
    acc = np.float32(0)
    for v in rng.permutation(vals):
        acc = np.float32(acc + v)
    assert int(acc) == int(vals.astype(np.int64).sum())


def test_readback_is_exact_below_two_to_24_and_routes_the_rest():
    # S - 2X = SSD - A2 with 0 <= A2 <= a2_max and SSD >= 0; for every SSD
    # near and across 2^24 and any A2, the FP32 read-back equals SSD when
    # SSD < 2^24 and is not below 2^24 otherwise
    n = P_MAX * P_MAX
    a2_max = n * 3 * 128 * 128
    rng = np.random.default_rng(9)
    ssd = np.concatenate([np.arange((1 << 24) - 4096, (1 << 24) + 4096),
                          rng.integers(0, 1 << 24, 20000), rng.integers(1 << 24, 3 << 24, 5000)])
    a2 = rng.integers(0, a2_max + 1, ssd.size)
    # the accumulators hold S and X exactly; one FMA gives fl(S - 2X)
    fsx = (ssd - a2).astype(np.float64).astype(np.float32)
    v = (fsx + a2.astype(np.float32)).astype(np.float32)  # fl(fl(S - 2X) + A2)
    below = ssd < (1 << 24)
    assert np.array_equal(v[below].astype(np.int64), ssd[below])
    assert np.all(v[~below] >= TWO24)
