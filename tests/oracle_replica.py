"""A rank's replica of one removal computed by the CPU oracle, with the
interface of the row-sharded driver (search_rect, search_rows, apply_key).

The search of a row range is the oracle's iteration with its search
rectangle limited to those rows (its state is discarded), and applying a key
is the oracle's iteration with the rectangle reduced to that key's centre,
so each replica follows the oracle's own fill loop (Sec. 3) step by step.
"""
import numpy as np

import oracle

KEY_NONE = (1 << 64) - 1
NO_SOURCE = -4


class OracleReplica:
    def __init__(self, rgb, mask, r):
        self.r = r
        self.W = mask.shape[1]
        self.rgb = np.array(rgb, np.uint8)
        self.om = (np.asarray(mask) != 0).astype(np.uint8)
        self.conf = np.where(self.om != 0, 0.0, 1.0)  # C = 1 on Phi, 0 on Omega
        self.rect = oracle.search_rect(mask, r)      # (x0, x1, y0, y1), inclusive

    def search_rect(self):
        return self.rect

    def search_rows(self, y0, y1):
        if not self.om.any():
            return None
        x0, x1, ry0, ry1 = self.rect
        lo, hi = max(ry0, y0), min(ry1, y1 - 1)
        if lo > hi:
            return KEY_NONE
        res = oracle.run_from_state(self.rgb, self.om, self.conf, self.r, rect=(x0, x1, lo, hi), max_iters=1)
        if res.status == NO_SOURCE:
            return KEY_NONE
        assert res.status == 0 and res.iters == 1
        t = res.trace[0]
        return (int(t["ssd"]) << 32) | (int(t["qy"]) * self.W + int(t["qx"]))

    def apply_key(self, key):
        assert key != KEY_NONE, "no source anywhere"
        q = key & 0xffffffff
        qx, qy = q % self.W, q // self.W
        res = oracle.run_from_state(self.rgb, self.om, self.conf, self.r, rect=(qx, qx, qy, qy), max_iters=1)
        assert res.status == 0 and res.iters == 1
        assert (int(res.trace[0]["ssd"]) << 32 | q) == key
        self.rgb, self.om, self.conf = res.rgb, res.mask, res.conf
        return res.trace[0]
