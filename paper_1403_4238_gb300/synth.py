"""Seeded synthetic inputs shaped like the paper's mobile-camera workloads.

The paper's photos (Table 3: WalkingMan 512x384, River 480x639, DivingMan
576x384, Hill 1024x550) are not available; these generators stand in for
them.  This module holds none of the inpainting arithmetic: it only makes
images and masks, and both the CUDA library's callers and the oracle consume
the same bytes.

Random numbers come from numpy's PCG64 bit generator (a documented, platform-
stable stream), seeded per input.

Image recipe: Voronoi regions (seeds uniform in the image, flat RGB colour per
region uniform in 0..255, nearest seed by squared Euclidean distance, ties to
the lowest seed) + three oriented sinusoidal gratings A*sin(2*pi*(x cos t +
y sin t)/lambda + phi) added to every channel (t ~ U[0, pi), lambda ~ U[8, 48]
pixels, phi ~ U[0, 2 pi)) + Gaussian noise sigma 4 per channel (Box-Muller),
rounded half up and clamped to [0, 255].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def image(W: int, H: int, regions: int, amplitude: float, seed: int, sigma: float = 4.0) -> np.ndarray:
    """(H, W, 3) uint8 synthetic image."""
    g = _rng(seed)
    sx = g.uniform(0, W, regions)
    sy = g.uniform(0, H, regions)
    colours = g.integers(0, 256, size=(regions, 3)).astype(np.float64)
    theta = g.uniform(0, math.pi, 3)
    lam = g.uniform(8.0, 48.0, 3)
    phi = g.uniform(0, 2 * math.pi, 3)

    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    label = np.zeros((H, W), np.int64)
    best = np.full((H, W), np.inf)
    for k in range(regions):  # strict < keeps the lowest seed on ties
        d = (xs - sx[k]) ** 2 + (ys - sy[k]) ** 2
        closer = d < best
        best = np.where(closer, d, best)
        label = np.where(closer, k, label)
    out = colours[label]  # (H, W, 3)
    grating = np.zeros((H, W))
    for t, l, p in zip(theta, lam, phi):
        grating += amplitude * np.sin(2 * math.pi * (xs * math.cos(t) + ys * math.sin(t)) / l + p)
    out += grating[..., None]
    u1 = g.uniform(np.finfo(np.float64).tiny, 1.0, (H, W, 3))
    u2 = g.uniform(0.0, 1.0, (H, W, 3))
    out += sigma * np.sqrt(-2.0 * np.log(u1)) * np.cos(2 * math.pi * u2)
    return np.clip(np.floor(out + 0.5), 0, 255).astype(np.uint8)


def rect_mask(W: int, H: int, w: int, h: int, seed: int) -> np.ndarray:
    """Axis-aligned w x h rectangle at a uniform position inside the image."""
    g = _rng(seed)
    x0 = int(g.integers(0, W - w + 1))
    y0 = int(g.integers(0, H - h + 1))
    m = np.zeros((H, W), np.uint8)
    m[y0:y0 + h, x0:x0 + w] = 1
    return m


def ellipse_mask(W: int, H: int, n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Union of n seeded rotated ellipses, rescaled until the covered fraction
    lies in [lo, hi]."""
    g = _rng(seed)
    cx = g.uniform(0.15 * W, 0.85 * W, n)
    cy = g.uniform(0.15 * H, 0.85 * H, n)
    ax = g.uniform(0.5, 1.5, n)
    ay = g.uniform(0.5, 1.5, n)
    rot = g.uniform(0, math.pi, n)
    target = g.uniform(lo, hi)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)

    def build(scale):
        # each ellipse is evaluated on its bounding box only (plus a margin);
        # pixels outside it are farther than scale * max(ax, ay) from the centre
        m = np.zeros((H, W), bool)
        for i in range(n):
            ext = scale * max(ax[i], ay[i]) + 2.0
            x0, x1 = max(0, int(cx[i] - ext)), min(W, int(cx[i] + ext) + 2)
            y0, y1 = max(0, int(cy[i] - ext)), min(H, int(cy[i] + ext) + 2)
            if x0 >= x1 or y0 >= y1:
                continue
            dx, dy = xs[y0:y1, x0:x1] - cx[i], ys[y0:y1, x0:x1] - cy[i]
            u = dx * math.cos(rot[i]) + dy * math.sin(rot[i])
            v = -dx * math.sin(rot[i]) + dy * math.cos(rot[i])
            m[y0:y1, x0:x1] |= (u / (scale * ax[i])) ** 2 + (v / (scale * ay[i])) ** 2 <= 1.0
        return m

    a, b = 0.5, 0.5 * math.hypot(W, H)
    m = build(b)
    for _ in range(60):
        s = 0.5 * (a + b)
        m = build(s)
        f = m.mean()
        if lo <= f <= hi and abs(f - target) < 0.002:
            break
        if f < target:
            a = s
        else:
            b = s
    return m.astype(np.uint8)


def blob_mask(W: int, H: int, frac: float, seed: int, tol: float = 0.005) -> np.ndarray:
    """Union of discs along a seeded random walk, grown until the covered
    fraction reaches frac (the last disc is shrunk to stay within tol)."""
    g = _rng(seed)
    m = np.zeros((H, W), bool)
    ys, xs = np.mgrid[0:H, 0:W]
    x, y = g.uniform(0.3 * W, 0.7 * W), g.uniform(0.3 * H, 0.7 * H)
    base = 0.04 * min(W, H)
    while m.mean() < frac - tol:
        rad = base * g.uniform(0.6, 1.4)
        disc = (xs - x) ** 2 + (ys - y) ** 2 <= rad * rad
        cand = m | disc
        while cand.mean() > frac + tol and rad > 1.0:
            rad *= 0.8
            disc = (xs - x) ** 2 + (ys - y) ** 2 <= rad * rad
            cand = m | disc
        m = cand
        ang = g.uniform(0, 2 * math.pi)
        x = float(np.clip(x + 0.8 * base * math.cos(ang), 0.1 * W, 0.9 * W))
        y = float(np.clip(y + 0.8 * base * math.sin(ang), 0.1 * H, 0.9 * H))
    return m.astype(np.uint8)


@dataclass
class Case:
    name: str
    rgb: np.ndarray   # (H, W, 3) uint8
    mask: np.ndarray  # (H, W) uint8, nonzero = remove
    r: int

    @property
    def W(self):
        return self.rgb.shape[1]

    @property
    def H(self):
        return self.rgb.shape[0]


def small_rect(seed: int = 1) -> Case:
    """128x96, 6 regions, amplitude 30, 20x16 rectangle, 9x9 patches."""
    return Case("rect128x96_r4", image(128, 96, 6, 30.0, seed), rect_mask(128, 96, 20, 16, seed + 1000), 4)


def walkingman_like(seed: int = 2) -> Case:
    """512x384, 12 regions, amplitude 30, 3 ellipses covering 7.5-8.5 %, 9x9."""
    return Case("ell512x384_r4", image(512, 384, 12, 30.0, seed),
                ellipse_mask(512, 384, 3, 0.075, 0.085, seed + 1000), 4)


def hd_blob(seed: int = 3) -> Case:
    """1920x1080, 40 regions, amplitude 40, random-walk blob of ~5 %, 13x13."""
    return Case("blob1920x1080_r6", image(1920, 1080, 40, 40.0, seed),
                blob_mask(1920, 1080, 0.05, seed + 1000), 6)


def batch_cases(n: int = 64, seed: int = 4):
    """n images, W ~ U[256, 1280], H ~ U[256, 720], ellipse-union masks over
    3-10 % of the area, patch radius 4 or 5."""
    g = _rng(seed)
    out = []
    for i in range(n):
        W = int(g.integers(256, 1281))
        H = int(g.integers(256, 721))
        r = int(g.integers(4, 6))
        lo = float(g.uniform(0.03, 0.095))
        s = int(g.integers(0, 2**31))
        out.append(Case(f"batch{i}_{W}x{H}_r{r}", image(W, H, 12, 30.0, s),
                        ellipse_mask(W, H, 3, lo, lo + 0.005, s + 1), r))
    return out


def serving_trace(n: int = 2000, rate: float = 200.0, seed: int = 5):
    """Open-loop Poisson arrivals: (arrival time s, W, H, r, mask lo, seed)."""
    g = _rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate, n))
    reqs = []
    for i in range(n):
        W = int(g.integers(320, 1921))
        H = int(g.integers(240, 1081))
        r = int(g.integers(4, 6))
        lo = float(g.uniform(0.02, 0.115))
        reqs.append((float(t[i]), W, H, r, lo, int(g.integers(0, 2**31))))
    return reqs


def serving_case(W, H, r, lo, s) -> Case:
    return Case(f"req_{W}x{H}_r{r}", image(W, H, 12, 30.0, s), ellipse_mask(W, H, 3, lo, lo + 0.005, s + 1), r)


def box_shape_mask(W: int, H: int, w: int, h: int, kind: str, seed: int) -> np.ndarray:
    """A w x h object at a seeded position inside the image, with bounding box
    exactly w x h: "blob" = the inscribed ellipse, "random" = a seeded union
    of discs inside the box (four of them centred on its edge midpoints, so
    that the shape spans the box), "strip" = the full box."""
    g = _rng(seed)
    x0 = int(g.integers(0, W - w + 1))
    y0 = int(g.integers(0, H - h + 1))
    m = np.zeros((H, W), bool)
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    if kind == "strip":
        box = np.ones((h, w), bool)
    elif kind == "blob":
        cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
        box = ((xs - cx) / (w / 2.0)) ** 2 + ((ys - cy) / (h / 2.0)) ** 2 <= 1.0
    elif kind == "random":
        rad0 = 0.12 * min(w, h)
        centres = [((w - 1) / 2.0, 0.0), ((w - 1) / 2.0, h - 1.0), (0.0, (h - 1) / 2.0), (w - 1.0, (h - 1) / 2.0)]
        radii = [rad0] * 4
        for _ in range(24):
            centres.append((g.uniform(0, w - 1), g.uniform(0, h - 1)))
            radii.append(g.uniform(0.5, 1.5) * 2.0 * rad0)
        box = np.zeros((h, w), bool)
        for (cx, cy), rad in zip(centres, radii):
            box |= (xs - cx) ** 2 + (ys - cy) ** 2 <= rad * rad
    else:
        raise ValueError(kind)
    m[y0:y0 + h, x0:x0 + w] = box
    return m.astype(np.uint8)


# Test images of Table 3: (name, W, H, object kind, object w, object h,
# image regions, grating amplitude).  Object kinds: blob, small blob, big /
# random shape, long strip.
TABLE3 = (
    ("walkingman", 512, 384, "blob", 78, 126, 12, 30.0),
    ("river", 480, 639, "blob", 59, 93, 16, 40.0),
    ("divingman", 576, 384, "random", 155, 186, 8, 40.0),
    ("hill", 1024, 550, "strip", 1024, 10, 12, 30.0),
)


def table3_case(name: str, r: int = 4, seed: int = 7) -> Case:
    """Synthetic stand-in for one test image of Table 3 (its size, object
    type and object size), with patch radius r."""
    for k, (nm, W, H, kind, w, h, regions, amp) in enumerate(TABLE3):
        if nm == name:
            s = seed + 100 * k
            return Case(f"{nm}{W}x{H}_r{r}", image(W, H, regions, amp, s),
                        box_shape_mask(W, H, w, h, kind, s + 1), r)
    raise KeyError(name)


def tiny(W: int, H: int, seed: int, hole: tuple | None = None, r: int = 1) -> Case:
    """Small random case for brute-force checks: noise image plus a hole."""
    g = _rng(seed)
    rgb = g.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    m = np.zeros((H, W), np.uint8)
    if hole is None:
        w = int(g.integers(1, max(2, W // 3)))
        h = int(g.integers(1, max(2, H // 3)))
        x0 = int(g.integers(0, W - w + 1))
        y0 = int(g.integers(0, H - h + 1))
        hole = (x0, y0, w, h)
    x0, y0, w, h = hole
    m[y0:y0 + h, x0:x0 + w] = 1
    return Case(f"tiny{W}x{H}_s{seed}", rgb, m, r)
