"""CPU oracle for exemplar-based object removal (paper Sec. 3, Eq. 1-4).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain single-threaded C program
(``inpaint_oracle.c``) that restates the algorithm step by step; this module
builds it with gcc and exposes it to Python through ctypes.  Only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.
It shares no code with the CUDA library and never imports it.

Parity pins (tests/test_oracle_*.py): an independent numpy brute force of the
SSD map and argmin, hand-computed priorities on few-pixel fronts, planted
exact copies, and run invariants.  The fill loop as a whole has no printed
reference values in the paper; it is pinned only through those pieces.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "inpaint_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libinpaint_oracle.so")
_lock = threading.Lock()
_lib = None

OK, DONE, ERR_ARG, ERR_NO_SOURCE = 0, 1, -1, -4


class Trace(ctypes.Structure):
    _fields_ = [
        ("iter", ctypes.c_int32),
        ("px", ctypes.c_int32),
        ("py", ctypes.c_int32),
        ("qx", ctypes.c_int32),
        ("qy", ctypes.c_int32),
        ("ssd", ctypes.c_uint32),
        ("priority", ctypes.c_double),
        ("confidence", ctypes.c_double),
        ("filled", ctypes.c_int32),
        ("remaining", ctypes.c_int32),
        ("n_known", ctypes.c_int32),
        ("n_cand", ctypes.c_int32),
    ]


TRACE_DTYPE = np.dtype(
    [
        ("iter", np.int32),
        ("px", np.int32),
        ("py", np.int32),
        ("qx", np.int32),
        ("qy", np.int32),
        ("ssd", np.uint32),
        ("priority", np.float64),
        ("confidence", np.float64),
        ("filled", np.int32),
        ("remaining", np.int32),
        ("n_known", np.int32),
        ("n_cand", np.int32),
    ],
    align=True,
)
assert TRACE_DTYPE.itemsize == ctypes.sizeof(Trace)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2 -ffp-contract=off) into oracle/_build."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (
        not force
        and os.path.exists(_LIB_PATH)
        and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC[:-1] + "h"))
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = [
        "gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
        "-Wall", "-Wextra", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm",
    ]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        f64p = ctypes.POINTER(ctypes.c_double)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        lib.oracle_gray.restype = ctypes.c_uint8
        lib.oracle_gray.argtypes = [ctypes.c_uint8] * 3
        lib.oracle_front.restype = None
        lib.oracle_front.argtypes = [u8p, c_int, c_int, u8p]
        lib.oracle_priority.restype = c_double
        lib.oracle_priority.argtypes = [u8p, f64p, u8p, c_int, c_int, c_int, c_int, c_int, f64p, f64p]
        lib.oracle_ssd_map.restype = c_int
        lib.oracle_ssd_map.argtypes = [u8p, u8p, c_int, c_int, c_int, c_int, c_int,
                                       c_int, c_int, c_int, c_int, u32p, i32p]
        lib.oracle_search_rect.restype = None
        lib.oracle_search_rect.argtypes = [u8p, c_int, c_int, c_int, c_double, i32p, i32p, i32p, i32p]
        lib.oracle_run.restype = c_int
        lib.oracle_run.argtypes = [u8p, u8p, c_int, c_int, c_int, c_double, c_int, u8p, u8p, f64p,
                                   ctypes.POINTER(Trace), c_int, i32p, u64p]
        lib.oracle_run_from_state.restype = c_int
        lib.oracle_run_from_state.argtypes = [u8p, u8p, f64p, c_int, c_int, c_int, c_int, c_int,
                                              c_int, c_int, c_int, ctypes.POINTER(Trace), c_int,
                                              i32p, u64p]
        lib.oracle_ssd_map_overlap.restype = c_int
        lib.oracle_ssd_map_overlap.argtypes = lib.oracle_ssd_map.argtypes
        lib.oracle_search_rect2.restype = None
        lib.oracle_search_rect2.argtypes = [u8p, c_int, c_int, c_int, c_double, c_int, i32p, i32p, i32p,
                                            i32p]
        lib.oracle_run2.restype = c_int
        lib.oracle_run2.argtypes = [u8p, u8p, c_int, c_int, c_int, c_double, c_int, c_int, u8p, u8p,
                                    f64p, ctypes.POINTER(Trace), c_int, i32p, u64p]
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ct):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ct))


def gray(r: int, g: int, b: int) -> int:
    return int(_load().oracle_gray(r, g, b))


def front(omega: np.ndarray) -> np.ndarray:
    H, W = omega.shape
    om = np.ascontiguousarray(omega, dtype=np.uint8)
    out = np.zeros((H, W), np.uint8)
    _load().oracle_front(_ptr(om, ctypes.c_uint8), W, H, _ptr(out, ctypes.c_uint8))
    return out


def priority(gray_img, conf, omega, r, x, y):
    """Returns (P, C, D) of pixel (x, y)."""
    H, W = omega.shape
    g = np.ascontiguousarray(gray_img, dtype=np.uint8)
    c = np.ascontiguousarray(conf, dtype=np.float64)
    om = np.ascontiguousarray(omega, dtype=np.uint8)
    co, do = ctypes.c_double(), ctypes.c_double()
    p = _load().oracle_priority(_ptr(g, ctypes.c_uint8), _ptr(c, ctypes.c_double),
                                _ptr(om, ctypes.c_uint8), W, H, r, x, y,
                                ctypes.byref(co), ctypes.byref(do))
    return p, co.value, do.value


def search_rect(mask, r, alpha=-1.0, overlap=False):
    H, W = mask.shape
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    v = [ctypes.c_int32() for _ in range(4)]
    _load().oracle_search_rect2(_ptr(m, ctypes.c_uint8), W, H, r, float(alpha), int(bool(overlap)),
                                *[ctypes.byref(x) for x in v])
    return tuple(x.value for x in v)


def ssd_map(rgb, omega, r, px, py, rect=None, overlap=False):
    """SSD of every candidate centre (UINT32_MAX where invalid), n_cand, |K|
    (overlap: the partial-overlap variant)."""
    H, W = omega.shape
    img = np.ascontiguousarray(rgb, dtype=np.uint8)
    om = np.ascontiguousarray(omega, dtype=np.uint8)
    if rect is None:
        rect = (0, W - 1, 0, H - 1) if overlap else (r, W - 1 - r, r, H - 1 - r)
    out = np.zeros((H, W), np.uint32)
    nk = ctypes.c_int32()
    fn = _load().oracle_ssd_map_overlap if overlap else _load().oracle_ssd_map
    nc = fn(_ptr(img, ctypes.c_uint8), _ptr(om, ctypes.c_uint8), W, H, r,
            px, py, *rect, _ptr(out, ctypes.c_uint32), ctypes.byref(nk))
    return out, int(nc), int(nk.value)


class Result:
    def __init__(self, status, rgb, mask, conf, trace, iters, evals):
        self.status = status
        self.rgb = rgb
        self.mask = mask
        self.conf = conf
        self.trace = trace
        self.iters = iters
        self.evals = evals


def run(rgb, mask, r, alpha=-1.0, max_iters=0, trace_cap=None, overlap=False) -> Result:
    """The whole removal loop.  rgb: (H, W, 3) uint8, mask: (H, W) nonzero = remove;
    overlap: the partial-overlap search variant (Alg. 1, Sec. 5.4)."""
    H, W = mask.shape
    img = np.ascontiguousarray(rgb, dtype=np.uint8)
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    if trace_cap is None:
        trace_cap = int(np.count_nonzero(m)) + 1
    rgb_out = np.zeros((H, W, 3), np.uint8)
    mask_out = np.zeros((H, W), np.uint8)
    conf_out = np.zeros((H, W), np.float64)
    tr = np.zeros(max(trace_cap, 1), TRACE_DTYPE)
    iters = ctypes.c_int32()
    evals = ctypes.c_uint64()
    st = _load().oracle_run2(_ptr(img, ctypes.c_uint8), _ptr(m, ctypes.c_uint8), W, H, r,
                             float(alpha), int(bool(overlap)), int(max_iters),
                             _ptr(rgb_out, ctypes.c_uint8), _ptr(mask_out, ctypes.c_uint8),
                             _ptr(conf_out, ctypes.c_double), tr.ctypes.data_as(ctypes.POINTER(Trace)),
                             trace_cap, ctypes.byref(iters), ctypes.byref(evals))
    n = iters.value
    return Result(st, rgb_out, mask_out, conf_out, tr[: min(n, trace_cap)].copy(), n,
                  int(evals.value))


def run_from_state(rgb, omega, conf, r, rect=None, max_iters=0, trace_cap=None) -> Result:
    """Continue the loop from an explicit (rgb, omega, conf) state."""
    H, W = omega.shape
    img = np.array(rgb, dtype=np.uint8, order="C", copy=True)
    om = np.array(omega, dtype=np.uint8, order="C", copy=True)
    cf = np.array(conf, dtype=np.float64, order="C", copy=True)
    if rect is None:
        rect = (r, W - 1 - r, r, H - 1 - r)
    if trace_cap is None:
        trace_cap = int(np.count_nonzero(om)) + 1
    tr = np.zeros(max(trace_cap, 1), TRACE_DTYPE)
    iters = ctypes.c_int32()
    evals = ctypes.c_uint64()
    st = _load().oracle_run_from_state(_ptr(img, ctypes.c_uint8), _ptr(om, ctypes.c_uint8),
                                       _ptr(cf, ctypes.c_double), W, H, r, *rect,
                                       int(max_iters), tr.ctypes.data_as(ctypes.POINTER(Trace)),
                                       trace_cap, ctypes.byref(iters), ctypes.byref(evals))
    n = iters.value
    return Result(st, img, om, cf, tr[: min(n, trace_cap)].copy(), n, int(evals.value))
