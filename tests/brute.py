"""Independent numpy brute force used to pin the oracle on tiny inputs.

Written separately from oracle/inpaint_oracle.c and in a different style
(whole-array numpy slicing instead of per-pixel loops), so that a dropped
term, wrong sign, wrong index or transposed operand in either shows up as a
disagreement.  Same readings of the paper (Sec. 3, Eq. 1-4).
"""
from __future__ import annotations

import math

import numpy as np


def luma(rgb):
    rgb = rgb.astype(np.int64)
    return ((299 * rgb[..., 0] + 587 * rgb[..., 1] + 114 * rgb[..., 2] + 500) // 1000).astype(np.int64)


def front(omega):
    om = omega.astype(bool)
    phi = ~om
    pad = np.zeros((om.shape[0] + 2, om.shape[1] + 2), bool)  # outside = not known
    pad[1:-1, 1:-1] = phi
    nb = pad[:-2, 1:-1] | pad[2:, 1:-1] | pad[1:-1, :-2] | pad[1:-1, 2:]
    return (om & nb).astype(np.uint8)


def sobel_normal(omega, x, y):
    m = np.pad(omega.astype(np.int64) != 0, 1, mode="edge").astype(np.int64)
    win = m[y:y + 3, x:x + 3]  # centred on (x, y) in the padded frame
    kx = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]])
    return int((win * kx).sum()), int((win * kx.T).sum())


def priority(gray, conf, omega, r, x, y):
    """(P, C, D) as Python floats (IEEE double), summing C row-major."""
    H, W = omega.shape
    om = omega.astype(bool)
    total = 0.0
    count = 0
    for yy in range(y - r, y + r + 1):
        for xx in range(x - r, x + r + 1):
            if 0 <= xx < W and 0 <= yy < H:
                count += 1
                if not om[yy, xx]:
                    total += float(conf[yy, xx])
    c = total / count
    nx, ny = sobel_normal(omega, x, y)
    g = gray.astype(np.int64)
    best = None
    for yy in range(y - r, y + r + 1):
        for xx in range(x - r, x + r + 1):
            pts = [(xx, yy), (xx - 1, yy), (xx + 1, yy), (xx, yy - 1), (xx, yy + 1)]
            if all(0 <= a < W and 0 <= b < H and not om[b, a] for a, b in pts):
                gx = int(g[yy, xx + 1] - g[yy, xx - 1])
                gy = int(g[yy + 1, xx] - g[yy - 1, xx])
                if best is None or gx * gx + gy * gy > best[0]:
                    best = (gx * gx + gy * gy, gx, gy)
    gx, gy = (0, 0) if best is None else best[1:]
    dot = abs(-gy * nx + gx * ny)
    nn = nx * nx + ny * ny
    d = 0.0 if nn == 0 else (dot / math.sqrt(nn)) / 510.0
    return c * d, c, d


def ssd_map(rgb, omega, r, px, py, rect=None):
    """SSD map by whole-array shifts; invalid candidates get 2**32 - 1."""
    H, W = omega.shape
    om = omega.astype(bool)
    img = rgb.astype(np.int64)
    P = 2 * r + 1
    if rect is None:
        rect = (r, W - 1 - r, r, H - 1 - r)
    # unknown count of every patch via a sliding-window sum
    u = om.astype(np.int64)
    cnt = np.zeros((H - P + 1, W - P + 1), np.int64)
    for dy in range(P):
        for dx in range(P):
            cnt += u[dy:dy + H - P + 1, dx:dx + W - P + 1]
    ssd = np.zeros((H - P + 1, W - P + 1), np.int64)
    nk = 0
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            tx, ty = px + dx, py + dy
            if not (0 <= tx < W and 0 <= ty < H) or om[ty, tx]:
                continue
            nk += 1
            src = img[r + dy:r + dy + H - P + 1, r + dx:r + dx + W - P + 1, :]
            ssd += ((src - img[ty, tx, :]) ** 2).sum(axis=-1)
    out = np.full((H, W), 2**32 - 1, np.int64)
    valid = cnt == 0
    ys, xs = np.mgrid[r:H - r, r:W - r]
    valid &= (xs >= rect[0]) & (xs <= rect[1]) & (ys >= rect[2]) & (ys <= rect[3])
    inner = out[r:H - r, r:W - r]
    inner[valid] = ssd[valid]
    return out.astype(np.uint32), int(valid.sum()), nk


def ssd_map_overlap(rgb, omega, r, px, py, rect=None):
    """Partial-overlap variant (Alg. 1, Sec. 5.4) by whole-array shifts of a
    padded frame: every centre of the image is a candidate if every unknown
    in-image target pixel has a known in-image source pixel under it; the SSD
    runs over the target/source pairs that are both known and in the image."""
    H, W = omega.shape
    P = 2 * r + 1
    if rect is None:
        rect = (0, W - 1, 0, H - 1)
    # padded copies: outside the image = not known
    kn = np.zeros((H + 2 * r, W + 2 * r), bool)
    kn[r:r + H, r:r + W] = ~omega.astype(bool)
    img = np.zeros((H + 2 * r, W + 2 * r, 3), np.int64)
    img[r:r + H, r:r + W] = rgb
    ssd = np.zeros((H, W), np.int64)
    ok = np.ones((H, W), bool)
    nk = 0
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            tx, ty = px + dx, py + dy
            if not (0 <= tx < W and 0 <= ty < H):
                continue
            src_known = kn[r + dy:r + dy + H, r + dx:r + dx + W]  # known(q + d) for every centre q
            if omega[ty, tx]:
                ok &= src_known
                continue
            nk += 1
            src = img[r + dy:r + dy + H, r + dx:r + dx + W, :]
            ssd += np.where(src_known, ((src - rgb[ty, tx, :].astype(np.int64)) ** 2).sum(axis=-1), 0)
    ys, xs = np.mgrid[0:H, 0:W]
    ok &= (xs >= rect[0]) & (xs <= rect[1]) & (ys >= rect[2]) & (ys <= rect[3])
    out = np.where(ok, ssd, 2**32 - 1)
    return out.astype(np.uint32), int(ok.sum()), nk


def argmin_lowest(a):
    """Index of the smallest entry; the lowest flat index among equals."""
    flat = a.reshape(-1)
    return int(np.flatnonzero(flat == flat.min())[0])


def run(rgb, mask, r, max_iters=0, rect=None):
    """Whole loop on a tiny image; returns (status, rgb, omega, conf, trace)."""
    H, W = mask.shape
    img = rgb.copy()
    om = (mask != 0).astype(np.uint8)
    conf = np.where(om == 1, 0.0, 1.0)
    trace = []
    if om.sum() == 0:
        return 1, img, om, conf, trace
    it = 0
    while om.sum() > 0 and (max_iters <= 0 or it < max_iters):
        gray = luma(img)
        f = front(om)
        best = None
        for i in np.flatnonzero(f.reshape(-1)):
            y, x = divmod(int(i), W)
            p, c, _ = priority(gray, conf, om, r, x, y)
            if best is None or p > best[0]:
                best = (p, c, x, y)
        p, c, px, py = best
        ssd, nc, nk = ssd_map(img, om, r, px, py, rect)
        if nc == 0:
            return -4, img, om, conf, trace
        q = argmin_lowest(ssd.astype(np.int64))
        qy, qx = divmod(q, W)
        filled = 0
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                tx, ty = px + dx, py + dy
                if 0 <= tx < W and 0 <= ty < H and om[ty, tx]:
                    img[ty, tx] = img[qy + dy, qx + dx]
                    conf[ty, tx] = c
                    om[ty, tx] = 0
                    filled += 1
        trace.append(dict(iter=it, px=px, py=py, qx=qx, qy=qy, ssd=int(ssd[qy, qx]), priority=p,
                          confidence=c, filled=filled, remaining=int(om.sum()), n_known=nk,
                          n_cand=nc))
        it += 1
    return 0, img, om, conf, trace
