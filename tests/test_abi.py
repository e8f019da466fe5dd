"""The C-ABI library builds for sm_103a and exports every declared entry point.

No kernel is launched here (no GPU on the build machine)."""
import ctypes
import os
import re

from paper_1403_4238_gb300 import _lib

HEADER_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared_functions():
    names = set()
    for f in os.listdir(HEADER_DIR):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"typedef[^;]*;", "", text, flags=re.S)
        for m in re.finditer(r"\b(inpaint_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = _lib.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert "inpaint_create" in names and "inpaint_run" in names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding covers the same entry points
    assert names <= set(_lib.SIGNATURES), sorted(names - set(_lib.SIGNATURES))


def test_status_strings_without_gpu():
    lib = _lib.load()
    for name, code in _lib.STATUS.items():
        assert lib.inpaint_status_str(code)
    opt = _lib.Options()
    lib.inpaint_options_default(ctypes.byref(opt))
    assert opt.form == 0 and opt.search_alpha < 0 and opt.search_variant == 0


def test_search_variant_options_checked_before_any_device_work():
    lib = _lib.load()
    ctx = ctypes.c_void_p()
    buf = (ctypes.c_uint8 * (3 * 30 * 30))()

    def create(r, **fields):
        opt = _lib.Options()
        lib.inpaint_options_default(ctypes.byref(opt))
        for k, v in fields.items():
            setattr(opt, k, v)
        return lib.inpaint_create(buf, 30, 30, 90, buf, 30, r, ctypes.byref(opt), ctypes.byref(ctx))

    assert create(2, search_variant=5) == -1
    # the partial-overlap variant: plain form, radius <= 8, graph loop only
    assert create(2, search_variant=1, form=1) == -6
    assert create(9, search_variant=1) == -6
    assert create(2, search_variant=1, loop_mode=1) == -6
    assert not ctx.value


def test_bad_arguments_rejected_before_any_device_work():
    lib = _lib.load()
    ctx = ctypes.c_void_p()
    buf = (ctypes.c_uint8 * 300)()
    # radius 0, radius 33, image smaller than a patch, null pointers
    assert lib.inpaint_create(buf, 10, 10, 30, buf, 10, 0, None, ctypes.byref(ctx)) == -1
    assert lib.inpaint_create(buf, 10, 10, 30, buf, 10, 33, None, ctypes.byref(ctx)) == -1
    assert lib.inpaint_create(buf, 4, 4, 12, buf, 4, 2, None, ctypes.byref(ctx)) == -1
    assert lib.inpaint_create(None, 10, 10, 30, buf, 10, 1, None, ctypes.byref(ctx)) == -1
    assert lib.inpaint_create(buf, 10, 10, 20, buf, 10, 1, None, ctypes.byref(ctx)) == -1
    assert not ctx.value
    # failure injection: null context or an out-of-range wait limit
    done = ctypes.c_int(7)
    assert lib.inpaint_run_withheld(None, 0, 0.05, 0, ctypes.byref(done)) == -1 and done.value == 0
    assert lib.inpaint_run_withheld(None, -1, 0.05, 0, None) == -1
    assert lib.inpaint_run_withheld(None, 0, 0.0, 0, None) == -1
    key = ctypes.c_uint64(5)
    assert lib.inpaint_search_rows(None, 0, 10, ctypes.byref(key)) == -1
    assert lib.inpaint_apply_key(None, 0, None) == -1


def test_one_shot_batch_rejects_bad_arguments_before_any_device_work():
    lib = _lib.load()
    n = 2
    buf = (ctypes.c_uint8 * (3 * 30 * 30))()
    ptrs = (ctypes.c_void_p * n)(ctypes.addressof(buf), ctypes.addressof(buf))
    nulls = (ctypes.c_void_p * n)(ctypes.addressof(buf), None)
    ints = (ctypes.c_int * n)(30, 30)
    radii = (ctypes.c_int * n)(2, 2)
    st = (ctypes.c_int * n)()
    assert lib.inpaint_batch_run(0, ptrs, ptrs, ints, ints, radii, None, ptrs, st) == -1
    assert lib.inpaint_batch_run(n, None, ptrs, ints, ints, radii, None, ptrs, st) == -1
    assert lib.inpaint_batch_run(n, ptrs, ptrs, ints, ints, radii, None, nulls, st) == -1
    assert b"index 1" in lib.inpaint_last_error()
