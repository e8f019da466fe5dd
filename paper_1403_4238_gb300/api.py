"""Python binding of libinpaint with the same entry points as include/inpaint.h.

Argument marshalling only.  PyTorch provides the CUDA stream and, through the
allocator hooks of inpaint_options, the device memory (its caching
allocator); every step of the method runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import STEP_DTYPE, InpaintError, Options, StepInfo

FORMS = {"plain": 0, "tc": 1}
LOOPS = {"auto": 0, "engine": 1, "graph": 2}


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("libinpaint needs a CUDA GPU; none is visible")
    return torch


class _TorchAllocator:
    """inpaint_options.dev_alloc/dev_free backed by PyTorch's caching allocator."""

    def __init__(self, device: int):
        torch = _torch()
        self.device = device

        def alloc(nbytes, stream, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
            except Exception:  # noqa: BLE001 - reported to C as NULL (INPAINT_ERR_NOMEM)
                return None

        def free(ptr, nbytes, stream, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = _lib.ALLOC_FN(alloc)
        self.free = _lib.FREE_FN(free)


def _check(code: int, where: str) -> int:
    if code < 0:
        raise InpaintError(code, where)
    return code


def _host_u8(a, shape_tail=()):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a


class Inpainter:
    """One object-removal job (a context of the C library).

    rgb: (H, W, 3) uint8 array; mask: (H, W), nonzero = remove; r: patch
    radius (patch side 2r+1).  form: "plain" or "tc".  alpha: search factor
    of Eq. 6 (negative = exhaustive).  loop: "auto", "engine" (persistent
    kernel) or "graph" (conditional CUDA graph).  tile_rows: engine search
    unit height (0 = library choice); tuning_file: autotuner table
    (paper_1403_4238_gb300.autotune) consulted when tile_rows is 0.  overlap:
    the partial-overlap search variant of Algorithm 1 / Sec. 5.4 (graph loop,
    r <= 8).  Inputs may be numpy arrays (host) or CUDA torch tensors (device,
    uint8, contiguous).
    """

    def __init__(self, rgb, mask, r: int, *, form: str = "plain", alpha: float = -1.0,
                 debug: bool = False, stream=None, torch_memory: bool = True,
                 loop: str = "auto", tile_rows: int = 0, tuning_file: str | None = None,
                 overlap: bool = False):
        torch = _torch()
        self.lib = _lib.load()
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self._alloc = _TorchAllocator(self.device) if torch_memory else None
        opt = Options()
        self.lib.inpaint_options_default(ctypes.byref(opt))
        opt.form = FORMS[form]
        opt.cuda_stream = self.stream.cuda_stream
        opt.debug_checks = int(debug)
        opt.search_alpha = float(alpha)
        opt.loop_mode = LOOPS[loop]
        opt.tile_rows = int(tile_rows)
        opt.search_variant = 1 if overlap else 0
        self._tf = tuning_file.encode() if tuning_file else None
        opt.tuning_file = self._tf
        if self._alloc is not None:
            opt.dev_alloc = self._alloc.alloc
            opt.dev_free = self._alloc.free
        self._opt = opt
        rgb_h = _host_u8(rgb.cpu().numpy() if hasattr(rgb, "cpu") else rgb)
        mask_h = _host_u8(mask.cpu().numpy() if hasattr(mask, "cpu") else mask)
        H, W = mask_h.shape
        assert rgb_h.shape == (H, W, 3)
        self.W, self.H, self.r = W, H, r
        ctx = ctypes.c_void_p()
        _check(self.lib.inpaint_create(rgb_h.ctypes.data, W, H, 3 * W, mask_h.ctypes.data, W, r,
                                       ctypes.byref(opt), ctypes.byref(ctx)), "inpaint_create")
        self.ctx = ctx

    # -- lifetime -------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.inpaint_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- loop -----------------------------------------------------------
    def reset(self, rgb, mask):
        """New inputs of the same size: numpy (host) or CUDA uint8 tensors (device)."""
        if hasattr(rgb, "is_cuda") and rgb.is_cuda:
            assert rgb.is_contiguous() and mask.is_contiguous()
            return _check(self.lib.inpaint_reset(self.ctx, rgb.data_ptr(), 3 * self.W,
                                                 mask.data_ptr(), self.W, 1), "inpaint_reset")
        rgb_h, mask_h = _host_u8(rgb), _host_u8(mask)
        return _check(self.lib.inpaint_reset(self.ctx, rgb_h.ctypes.data, 3 * self.W,
                                             mask_h.ctypes.data, self.W, 0), "inpaint_reset")

    def step(self):
        """One iteration; returns its record (numpy structured scalar) or None when done."""
        info = StepInfo()
        rc = _check(self.lib.inpaint_step(self.ctx, ctypes.byref(info)), "inpaint_step")
        if rc == 1:
            return None
        out = np.zeros(1, STEP_DTYPE)
        ctypes.memmove(out.ctypes.data, ctypes.byref(info), STEP_DTYPE.itemsize)
        return out[0]

    def run(self, max_iters: int = 0, trace: bool = False, trace_cap: int | None = None):
        """Iterate on the device; returns (status, iterations, trace array or None)."""
        done = ctypes.c_int()
        tr = None
        ptr, cap = None, 0
        if trace:
            cap = trace_cap if trace_cap is not None else self.info()["remaining"] + 1
            tr = np.zeros(max(cap, 1), STEP_DTYPE)
            ptr = tr.ctypes.data
        rc = _check(self.lib.inpaint_run(self.ctx, int(max_iters), ctypes.byref(done), ptr, cap),
                    "inpaint_run")
        n = done.value
        if tr is not None:
            tr = tr[: min(n, cap)].copy()
        return rc, n, tr

    def result(self, with_mask: bool = False):
        rgb = np.zeros((self.H, self.W, 3), np.uint8)
        m = np.zeros((self.H, self.W), np.uint8) if with_mask else None
        _check(self.lib.inpaint_result(self.ctx, rgb.ctypes.data, 3 * self.W,
                                       m.ctypes.data if m is not None else None), "inpaint_result")
        return (rgb, m) if with_mask else rgb

    def export_state(self):
        rgb = np.zeros((self.H, self.W, 3), np.uint8)
        om = np.zeros((self.H, self.W), np.uint8)
        conf = np.zeros((self.H, self.W), np.float64)
        _check(self.lib.inpaint_export_state(self.ctx, rgb.ctypes.data, om.ctypes.data,
                                             conf.ctypes.data), "inpaint_export_state")
        return rgb, om, conf

    def import_state(self, rgb, omega, conf):
        rgb = np.ascontiguousarray(rgb, np.uint8)
        omega = np.ascontiguousarray(omega, np.uint8)
        conf = np.ascontiguousarray(conf, np.float64)
        return _check(self.lib.inpaint_import_state(self.ctx, rgb.ctypes.data, omega.ctypes.data,
                                                    conf.ctypes.data), "inpaint_import_state")

    def info(self):
        w, h, r, rem = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ev = ctypes.c_uint64()
        _check(self.lib.inpaint_info(self.ctx, ctypes.byref(w), ctypes.byref(h), ctypes.byref(r),
                                     ctypes.byref(rem), ctypes.byref(ev)), "inpaint_info")
        return dict(width=w.value, height=h.value, r=r.value, remaining=rem.value, evals=ev.value)

    def loop_timing(self):
        """Engine phase clocks since create/reset: (search_ns, update_ns, iterations)."""
        a, b, n = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int()
        _check(self.lib.inpaint_loop_timing(self.ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)),
               "inpaint_loop_timing")
        return a.value, b.value, n.value

    def tc_rounds(self):
        """Iterations since create/reset whose engine search ran in the tensor-core form."""
        n = ctypes.c_int()
        _check(self.lib.inpaint_search_form_rounds(self.ctx, ctypes.byref(n)), "inpaint_search_form_rounds")
        return n.value

    def time_search(self, form: str = "plain", reps: int = 20):
        """Isolated timing of one search of `form` for the current target:
        (ms per search, best key (SSD << 32 | idx), evaluations)."""
        ms, key, ev = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(self.lib.inpaint_time_search(self.ctx, FORMS[form], int(reps), ctypes.byref(ms), ctypes.byref(key),
                                            ctypes.byref(ev)), "inpaint_time_search")
        return ms.value, key.value, ev.value

    def search_rect(self):
        v = [ctypes.c_int() for _ in range(4)]
        _check(self.lib.inpaint_search_rect(self.ctx, *[ctypes.byref(x) for x in v]),
               "inpaint_search_rect")
        return tuple(x.value for x in v)

    # -- row-sharded iterations (one removal over several replicas) -------
    def search_rows(self, y0: int, y1: int):
        """Smallest packed key (SSD << 32 | y*W + x) among the candidate
        centres of rows [y0, y1) for the current target; _lib.KEY_NONE if
        those rows hold none; None once the removal is done."""
        key = ctypes.c_uint64()
        rc = _check(self.lib.inpaint_search_rows(self.ctx, int(y0), int(y1), ctypes.byref(key)),
                    "inpaint_search_rows")
        return None if rc == 1 else key.value

    def apply_key(self, key: int):
        """Complete the iteration with the global minimum key; returns its
        record (None if the removal was already done)."""
        info = StepInfo()
        rc = _check(self.lib.inpaint_apply_key(self.ctx, ctypes.c_uint64(int(key)), ctypes.byref(info)),
                    "inpaint_apply_key")
        if rc == 1:
            return None
        out = np.zeros(1, STEP_DTYPE)
        ctypes.memmove(out.ctypes.data, ctypes.byref(info), STEP_DTYPE.itemsize)
        return out[0]


def remove_object(rgb, mask, r: int, **kw):
    """Convenience: create, run to completion, return (rgb_out, trace)."""
    with Inpainter(rgb, mask, r, **kw) as ip:
        rc, n, tr = ip.run(trace=True)
        return ip.result(), tr


def probe_peaks() -> dict:
    """Measured instruction-rate peaks of the current GPU (inpaint_probe_peaks)."""
    _torch()
    lib = _lib.load()
    pk = _lib.Peaks()
    _check(lib.inpaint_probe_peaks(ctypes.byref(pk)), "inpaint_probe_peaks")
    return {f: getattr(pk, f) for f, _ in _lib.Peaks._fields_}


class Batch:
    """Many independent removals in one persistent launch (inpaint_batch_*).

    cases: iterable of (rgb (H, W, 3) uint8, mask (H, W), patch radius).
    Results are identical to running each image alone.
    """

    def __init__(self, cases, *, tile_rows: int = 0, tuning_file: str | None = None, stream=None,
                 torch_memory: bool = True):
        torch = _torch()
        self.lib = _lib.load()
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self._alloc = _TorchAllocator(self.device) if torch_memory else None
        opt = Options()
        self.lib.inpaint_options_default(ctypes.byref(opt))
        opt.cuda_stream = self.stream.cuda_stream
        opt.tile_rows = int(tile_rows)
        self._tf = tuning_file.encode() if tuning_file else None
        opt.tuning_file = self._tf
        if self._alloc is not None:
            opt.dev_alloc = self._alloc.alloc
            opt.dev_free = self._alloc.free
        self._opt = opt
        self._keep = []
        imgs = []
        self.shapes = []
        for rgb, mask, r in cases:
            rgb = np.ascontiguousarray(rgb, np.uint8)
            mask = np.ascontiguousarray(mask, np.uint8)
            H, W = mask.shape
            self._keep += [rgb, mask]
            imgs.append(_lib.Image(rgb.ctypes.data, W, H, 3 * W, mask.ctypes.data, W, int(r)))
            self.shapes.append((H, W))
        self.n = len(imgs)
        arr = (_lib.Image * self.n)(*imgs)
        b = ctypes.c_void_p()
        _check(self.lib.inpaint_batch_create(arr, self.n, ctypes.byref(opt), ctypes.byref(b)),
               "inpaint_batch_create")
        self.b = b
        self._keep = []  # inputs were copied

    def close(self):
        if getattr(self, "b", None):
            self.lib.inpaint_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reset(self):
        return _check(self.lib.inpaint_batch_reset(self.b), "inpaint_batch_reset")

    def run(self, max_iters: int = 0):
        st = (ctypes.c_int * self.n)()
        _check(self.lib.inpaint_batch_run_ctx(self.b, int(max_iters), st), "inpaint_batch_run_ctx")
        return list(st)

    def result(self, i: int):
        H, W = self.shapes[i]
        out = np.zeros((H, W, 3), np.uint8)
        it, ev = ctypes.c_int(), ctypes.c_uint64()
        _check(self.lib.inpaint_batch_result(self.b, i, out.ctypes.data, 3 * W, ctypes.byref(it),
                                             ctypes.byref(ev)), "inpaint_batch_result")
        return out, it.value, ev.value

    def plan(self):
        g, t = ctypes.c_int(), ctypes.c_int()
        team = (ctypes.c_int * self.n)()
        size = (ctypes.c_int * self.n)()
        rows = (ctypes.c_int * self.n)()
        _check(self.lib.inpaint_batch_plan(self.b, ctypes.byref(g), ctypes.byref(t), team, size, rows),
               "inpaint_batch_plan")
        return dict(grid=g.value, teams=t.value, team=list(team), team_size=list(size), rows=list(rows))


def batch_run(cases, *, tile_rows: int = 0, tuning_file: str | None = None, stream=None):
    """One-shot batched removal (inpaint_batch_run): cases is a sequence of
    (rgb (H, W, 3) uint8, mask (H, W), patch radius); returns (list of result
    images, list of per-image statuses)."""
    torch = _torch()
    lib = _lib.load()
    stream = stream if stream is not None else torch.cuda.Stream(torch.cuda.current_device())
    opt = Options()
    lib.inpaint_options_default(ctypes.byref(opt))
    opt.cuda_stream = stream.cuda_stream
    opt.tile_rows = int(tile_rows)
    tf = tuning_file.encode() if tuning_file else None
    opt.tuning_file = tf
    rgbs, masks, outs = [], [], []
    for rgb, mask, _ in cases:
        m = np.ascontiguousarray(mask, np.uint8)
        rgbs.append(np.ascontiguousarray(rgb, np.uint8))
        masks.append(m)
        outs.append(np.zeros((m.shape[0], m.shape[1], 3), np.uint8))
    n = len(cases)
    ptrs = lambda arrs: (ctypes.c_void_p * n)(*[a.ctypes.data for a in arrs])  # noqa: E731
    ints = lambda vals: (ctypes.c_int * n)(*vals)  # noqa: E731
    st = (ctypes.c_int * n)()
    _check(lib.inpaint_batch_run(n, ptrs(rgbs), ptrs(masks), ints([m.shape[1] for m in masks]),
                                 ints([m.shape[0] for m in masks]), ints([int(c[2]) for c in cases]),
                                 ctypes.byref(opt), ptrs(outs), st), "inpaint_batch_run")
    return outs, list(st)


class Server:
    """Continuous-batching object-removal server (inpaint_server_*).

    A worker thread inside the library admits queued requests into device
    slots (HBM budget, slot limit) between scheduler ticks; each tick is one
    persistent launch over all active slots.  submit() returns an id at once;
    poll(id) returns None while pending, else (rgb, info dict).
    """

    def __init__(self, hbm_budget_bytes: int = 40 << 30, max_slots: int = 256, iters_per_tick: int = 0,
                 *, tile_rows: int = 0, tuning_file: str | None = None):
        torch = _torch()
        self.lib = _lib.load()
        torch.cuda.current_device()
        opt = Options()
        self.lib.inpaint_options_default(ctypes.byref(opt))
        opt.tile_rows = int(tile_rows)
        self._tf = tuning_file.encode() if tuning_file else None
        opt.tuning_file = self._tf
        self._opt = opt
        s = ctypes.c_void_p()
        _check(self.lib.inpaint_server_create(int(hbm_budget_bytes), int(max_slots), int(iters_per_tick),
                                              ctypes.byref(opt), ctypes.byref(s)), "inpaint_server_create")
        self.s = s
        self.shapes = {}

    def close(self):
        if getattr(self, "s", None):
            self.lib.inpaint_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, rgb, mask, r: int) -> int:
        rgb = np.ascontiguousarray(rgb, np.uint8)
        mask = np.ascontiguousarray(mask, np.uint8)
        H, W = mask.shape
        im = _lib.Image(rgb.ctypes.data, W, H, 3 * W, mask.ctypes.data, W, int(r))
        rid = ctypes.c_uint64()
        _check(self.lib.inpaint_server_submit(self.s, ctypes.byref(im), ctypes.byref(rid)),
               "inpaint_server_submit")
        self.shapes[rid.value] = (H, W)
        return rid.value

    def poll(self, rid: int):
        H, W = self.shapes[rid]
        out = np.zeros((H, W, 3), np.uint8)
        info = _lib.RequestInfo()
        rc = _check(self.lib.inpaint_server_poll(self.s, ctypes.c_uint64(rid), out.ctypes.data, 3 * W,
                                                 ctypes.byref(info)), "inpaint_server_poll")
        if rc == _lib.STATUS["PENDING"]:
            return None
        del self.shapes[rid]
        return out, {f: getattr(info, f) for f, _ in _lib.RequestInfo._fields_}

    def wait_idle(self, timeout_s: float = 600.0):
        return _check(self.lib.inpaint_server_wait_idle(self.s, float(timeout_s)), "inpaint_server_wait_idle")

    def stats(self):
        st = _lib.ServerStats()
        _check(self.lib.inpaint_server_stats_get(self.s, ctypes.byref(st)), "inpaint_server_stats_get")
        return {f: getattr(st, f) for f, _ in _lib.ServerStats._fields_}

    def clock(self) -> float:
        return float(self.lib.inpaint_server_clock(self.s))
