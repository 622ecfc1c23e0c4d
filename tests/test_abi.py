"""The C-ABI library loads, exports every entry point include/fot.h declares, and rejects
bad host-side arguments before touching a GPU.  CPU only (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fot.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fot_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_19072_gb300 import build
    if not os.path.exists(build.LIB) or any(
            os.path.getmtime(s) > os.path.getmtime(build.LIB) for s in build.sources()):
        build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("fot_create", "fot_solve", "fot_potentials", "fot_phase", "fot_destroy",
                 "fot_c_transform", "fot_u_update", "fot_v_update", "fot_marginal_error"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_mirrors_the_header():
    # the binding declares the same names (parse it as text: importing it needs the .so)
    src = open(os.path.join(ROOT, "paper_2512_19072_gb300", "binding.py")).read()
    for name in _declared():
        assert f'"{name}"' in src, name


def test_host_side_argument_errors(lib):
    lib.fot_create.restype = ctypes.c_int
    lib.fot_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.fot_create(ctypes.byref(h), 0, 16, 0, 0, None) == 1       # FOT_EINVAL
    assert lib.fot_create(ctypes.byref(h), 16, 5000, 0, 0, None) == 1
    assert lib.fot_create(ctypes.byref(h), 16, 16, 7, 0, None) == 1      # bad precision
    assert lib.fot_create(None, 16, 16, 0, 0, None) == 1
    lib.fot_status_string.restype = ctypes.c_char_p
    assert b"invalid" in lib.fot_status_string(1)
    lib.fot_solve.restype = ctypes.c_int
    assert lib.fot_solve(None, None, None, ctypes.c_double(0), None, 1, 0, 1) == 1
    lib.fot_launch_count.restype = ctypes.c_int64
    assert lib.fot_launch_count(None) == -1
    for name, nargs in (("fot_work_split", 1), ("fot_kernel_times", 2), ("fot_set_kernel_timing", 1)):
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        assert fn(None, *([None] * nargs)) == 1, name                    # FOT_EINVAL


def test_injected_allocation_failure(lib, monkeypatch):
    monkeypatch.setenv("FOT_FAULT_INJECT_ENOMEM", "1")
    lib.fot_create.restype = ctypes.c_int
    lib.fot_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.fot_create(ctypes.byref(h), 16, 16, 0, 0, None) == 2      # FOT_ENOMEM
    assert not h.value
