"""Build and load libinpaint (the CUDA library behind include/inpaint.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  There is no fallback; if the library cannot be built or
loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libinpaint.so")

ARCH = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_FLAGS = [
    ARCH, "-O3", "-lineinfo", "--fmad=false", "-std=c++17", "-rdc=true", "-maxrregcount=128",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC, "-I", OUT_DIR,
]
GENERATED = {"ssd_rows.cuh": "gen_ssd_rows.py"}  # headers written into OUT_DIR by csrc scripts

_lock = threading.Lock()
_lib = None


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libinpaint cannot be built")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h", ".py"))]
    hdrs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return sources() + hdrs + [os.path.abspath(__file__)]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every csrc/*.cu for sm_103a (in parallel) and link libinpaint.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _deps())
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    nvcc = _nvcc()
    objs = []
    for hdr, script in GENERATED.items():
        p = subprocess.run([sys.executable, os.path.join(CSRC, script)], capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"{script} failed:\n{p.stderr}")
        with open(os.path.join(OUT_DIR, hdr), "w") as f:
            f.write(p.stdout)

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *NVCC_FLAGS, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{p.stdout}\n{p.stderr}")
        if verbose:
            print(p.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [nvcc, ARCH, "-rdc=true", "-shared", "-o", tmp, *objs]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stdout}\n{p.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class StepInfo(ctypes.Structure):
    _fields_ = [
        ("iter", ctypes.c_int32), ("px", ctypes.c_int32), ("py", ctypes.c_int32),
        ("qx", ctypes.c_int32), ("qy", ctypes.c_int32), ("ssd", ctypes.c_uint32),
        ("priority", ctypes.c_double), ("confidence", ctypes.c_double),
        ("filled", ctypes.c_int32), ("remaining", ctypes.c_int32),
        ("n_known", ctypes.c_int32), ("n_cand", ctypes.c_int32),
    ]


class Peaks(ctypes.Structure):
    _fields_ = [("ssd_evals_per_s", ctypes.c_double), ("imad_per_s", ctypes.c_double),
                ("iadd3_per_s", ctypes.c_double), ("dadd_per_s", ctypes.c_double),
                ("sm_clock_mhz", ctypes.c_double), ("sm_count", ctypes.c_int)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("status", ctypes.c_int), ("iterations", ctypes.c_int), ("evals", ctypes.c_uint64),
                ("width", ctypes.c_int), ("height", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64), ("ticks", ctypes.c_uint64),
                ("queued", ctypes.c_int), ("active", ctypes.c_int), ("hbm_used", ctypes.c_size_t),
                ("hbm_budget", ctypes.c_size_t), ("busy_s", ctypes.c_double)]


STEP_DTYPE = np.dtype(
    [("iter", np.int32), ("px", np.int32), ("py", np.int32), ("qx", np.int32), ("qy", np.int32),
     ("ssd", np.uint32), ("priority", np.float64), ("confidence", np.float64),
     ("filled", np.int32), ("remaining", np.int32), ("n_known", np.int32), ("n_cand", np.int32)],
    align=True,
)
assert STEP_DTYPE.itemsize == ctypes.sizeof(StepInfo)

KEY_NONE = (1 << 64) - 1  # INPAINT_KEY_NONE: no candidate in the searched rows

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [
        ("form", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("debug_checks", ctypes.c_int),
        ("search_alpha", ctypes.c_double), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
        ("alloc_user", ctypes.c_void_p), ("loop_mode", ctypes.c_int), ("tile_rows", ctypes.c_int),
        ("tuning_file", ctypes.c_char_p), ("search_variant", ctypes.c_int),
    ]


class Image(ctypes.Structure):
    _fields_ = [
        ("rgb", ctypes.c_void_p), ("width", ctypes.c_int), ("height", ctypes.c_int),
        ("rgb_stride_bytes", ctypes.c_int), ("mask", ctypes.c_void_p),
        ("mask_stride_bytes", ctypes.c_int), ("patch_radius", ctypes.c_int),
    ]


# Exported symbols declared in include/inpaint.h, with their ctypes signatures.
_P = ctypes.c_void_p
_U8P = ctypes.POINTER(ctypes.c_uint8)
_I = ctypes.c_int
SIGNATURES = {
    "inpaint_options_default": (None, [ctypes.POINTER(Options)]),
    "inpaint_create": (_I, [_P, _I, _I, _I, _P, _I, _I, ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "inpaint_reset": (_I, [_P, _P, _I, _P, _I, _I]),
    "inpaint_step": (_I, [_P, ctypes.POINTER(StepInfo)]),
    "inpaint_run": (_I, [_P, _I, ctypes.POINTER(ctypes.c_int), _P, _I]),
    "inpaint_result": (_I, [_P, _P, _I, _P]),
    "inpaint_export_state": (_I, [_P, _P, _P, _P]),
    "inpaint_import_state": (_I, [_P, _P, _P, _P]),
    "inpaint_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                          ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_uint64)]),
    "inpaint_search_rect": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                 ctypes.POINTER(_I)]),
    "inpaint_destroy": (None, [_P]),
    "inpaint_status_str": (ctypes.c_char_p, [_I]),
    "inpaint_last_error": (ctypes.c_char_p, []),
    "inpaint_probe_peaks": (_I, [ctypes.POINTER(Peaks)]),
    "inpaint_time_search": (_I, [_P, _I, _I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64),
                                 ctypes.POINTER(ctypes.c_uint64)]),
    "inpaint_search_rows": (_I, [_P, _I, _I, ctypes.POINTER(ctypes.c_uint64)]),
    "inpaint_apply_key": (_I, [_P, ctypes.c_uint64, _P]),
    "inpaint_run_withheld": (_I, [_P, _I, ctypes.c_double, _I, ctypes.POINTER(_I)]),
    "inpaint_best_patch_noalloc": (_I, [_P, _P, _I, _I, _I, _I, _I, _P, _P]),
    "inpaint_batch_create": (_I, [ctypes.POINTER(Image), _I, ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "inpaint_batch_reset": (_I, [_P]),
    "inpaint_batch_run_ctx": (_I, [_P, _I, _P]),
    "inpaint_batch_run": (_I, [_I, _P, _P, _P, _P, _P, ctypes.POINTER(Options), _P, _P]),
    "inpaint_batch_result": (_I, [_P, _I, _P, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_uint64)]),
    "inpaint_batch_plan": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), _P, _P, _P]),
    "inpaint_batch_destroy": (None, [_P]),
    "inpaint_server_create": (_I, [ctypes.c_size_t, _I, _I, ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "inpaint_server_submit": (_I, [_P, ctypes.POINTER(Image), ctypes.POINTER(ctypes.c_uint64)]),
    "inpaint_server_poll": (_I, [_P, ctypes.c_uint64, _P, _I, ctypes.POINTER(RequestInfo)]),
    "inpaint_server_wait_idle": (_I, [_P, ctypes.c_double]),
    "inpaint_server_stats_get": (_I, [_P, ctypes.POINTER(ServerStats)]),
    "inpaint_server_clock": (ctypes.c_double, [_P]),
    "inpaint_server_destroy": (None, [_P]),
    "inpaint_loop_timing": (_I, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                 ctypes.POINTER(_I)]),
    "inpaint_search_form_rounds": (_I, [_P, ctypes.POINTER(_I)]),
}


def load():
    """Build if needed and load the library; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class InpaintError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.inpaint_status_str(code).decode()
        detail = lib.inpaint_last_error().decode()
        super().__init__(f"{where}: {msg} ({code}){': ' + detail if detail else ''}")
        self.code = code


STATUS = {
    "OK": 0, "DONE": 1, "PENDING": 2, "ERR_ARG": -1, "ERR_NOMEM": -2, "ERR_CUDA": -3, "ERR_NO_SOURCE": -4,
    "ERR_TIMEOUT": -5, "ERR_UNSUPPORTED": -6, "ERR_INTERNAL": -7,
}
