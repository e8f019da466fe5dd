"""The update kernel's data term without a division instruction.

D = (dot / sqrt(nn)) / 510 (Eq. 2 with alpha = 255 and the factor 2 of the
central difference) takes only the 14 squared normal lengths nn a Sobel
normal of a binary mask can have and dot in [0, 2040].  The kernel divides
by each known divisor b with Markstein's method from y = RN(1/b):
q0 = RN(a y), r = a - q0 b (exact, one FMA), q = RN(q0 + r y).  That is not
correctly rounded for every a and b in general, so this test checks it
against the correctly rounded quotients for every input the kernel can see,
with each operation's rounding computed exactly from rationals.
"""
import math
from fractions import Fraction

NN = (1, 2, 4, 5, 8, 9, 10, 13, 16, 17, 18, 20, 25, 32)  # nx, ny in [-4, 4]


def rn(x: Fraction) -> float:
    return float(x)  # Fraction -> float rounds to nearest, ties to even


def div_known(a: float, b: float, y: float) -> float:
    q0 = rn(Fraction(a) * Fraction(y))
    r = rn(Fraction(a) - Fraction(q0) * Fraction(b))  # exact: one FMA on the device
    return rn(Fraction(r) * Fraction(y) + Fraction(q0))


def test_every_sobel_normal_length_is_covered():
    # the Sobel normal of the Omega indicator (replicated borders: still a
    # 3x3 binary neighbourhood): every length it can take is one of the 14
    seen = set()
    for m in range(512):
        b = [(m >> k) & 1 for k in range(9)]
        g = [b[0:3], b[3:6], b[6:9]]
        nx = (g[0][2] + 2 * g[1][2] + g[2][2]) - (g[0][0] + 2 * g[1][0] + g[2][0])
        ny = (g[2][0] + 2 * g[2][1] + g[2][2]) - (g[0][0] + 2 * g[0][1] + g[0][2])
        if nx or ny:
            seen.add(nx * nx + ny * ny)
    assert seen <= set(NN)


def test_data_term_by_known_divisors_is_correctly_rounded():
    y510 = 1.0 / 510.0
    for nn in NN:
        s = math.sqrt(float(nn))
        ys = 1.0 / s
        for dot in range(2041):
            q1 = div_known(float(dot), s, ys)
            assert q1 == float(dot) / s, (nn, dot)
            assert div_known(q1, 510.0, y510) == (float(dot) / s) / 510.0, (nn, dot)
