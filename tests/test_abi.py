"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/hjlo.h declares; argument errors are reported before any
device work (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(hjlo_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("hjlo_plan_create", "hjlo_step", "hjlo_run", "hjlo_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1210_4090_gb300 import hjlo
    L = hjlo.lib()
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing
    # the binding wraps exactly the declared set
    assert sorted(hjlo.exported_symbols()) == declared_symbols()
    assert L.hjlo_version() == 1


@pytest.mark.parametrize("field,value", [("ndim", 0), ("ndim", 4), ("h", 0.0), ("h", float("nan")),
                                         ("dtype", 7), ("algo", 9), ("reserved", 1)])
def test_invalid_descriptor_rejected_without_device_work(field, value):
    from paper_1210_4090_gb300 import hjlo
    d = hjlo.make_desc((8, 8), 0.125, 0.1, (0.1, 0.2), (2, 2))
    setattr(d, field, value)
    out = ctypes.c_void_p()
    st = hjlo.lib().hjlo_plan_create(ctypes.byref(d), None, ctypes.byref(out))
    assert st == 1 and not out.value          # HJLO_EINVAL
    assert hjlo.lib().hjlo_last_error()


def test_invalid_shapes_and_steps_rejected():
    from paper_1210_4090_gb300 import hjlo
    d = hjlo.make_desc((8, 0), 0.125, 0.1, (0.1, 0.2), (2, 2))
    out = ctypes.c_void_p()
    assert hjlo.lib().hjlo_plan_create(ctypes.byref(d), None, ctypes.byref(out)) == 1
    d = hjlo.make_desc((8, 8), (0.125, -1.0), 0.1, (0.1, 0.2), (2, 2))
    assert hjlo.lib().hjlo_plan_create(ctypes.byref(d), None, ctypes.byref(out)) == 1
    assert hjlo.lib().hjlo_plan_create(None, None, ctypes.byref(out)) == 1
    assert hjlo.lib().hjlo_plan_destroy(None) == 0
    assert hjlo.lib().hjlo_run(None, None, None, 1) == 1
    assert hjlo.lib().hjlo_step(None, None, None, None, None) == 1
