"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/*.h declares, and the binding names them all."""
import ctypes
import os
import re

import pytest

from paper_1802_05839_gb300 import wx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(wx\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(wx.LIB_PATH):
        from paper_1802_05839_gb300 import build
        build.build()
    return wx.lib()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("wx_create", "wx_set_params", "wx_load_fields", "wx_step", "wx_physics_columns",
              "wx_destroy", "wx_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in sorted(declared_functions()):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_bounds_checked_library_builds_and_exports_every_symbol():
    """The debug build with WX_BOUNDS_CHECK compiles (it is built beside
    libwx.so) and exports the same ABI."""
    from paper_1802_05839_gb300 import build
    if not os.path.exists(build.LIB_BOUNDS):
        build.build(bounds=True)
    L = ctypes.CDLL(build.LIB_BOUNDS)
    for n in sorted(declared_functions()):
        assert hasattr(L, n), f"{n} missing from the bounds-checked library"


def test_binding_covers_every_declared_symbol():
    bound = {n for n, _, _ in wx.SIGNATURES}
    missing = declared_functions() - bound
    assert not missing, missing


def test_create_fails_cleanly_without_gpu_or_with_bad_args(lib):
    p = ctypes.c_void_p()
    assert lib.wx_create(0, 4, 4, 0, ctypes.byref(p)) == -1
    assert b"sizes" in lib.wx_last_error(None)
    assert lib.wx_create(4, 4, 4, 7, ctypes.byref(p)) == -1
    assert lib.wx_create(4, 4, 300, 0, ctypes.byref(p)) == -8
    assert lib.wx_create(4, 4, 4, 0, None) == -1
    lib.wx_destroy(None)  # NULL-safe
    assert lib.wx_step(None, 1, None) == -1
    assert lib.wx_sync(None) == -1


def _build_c_example(tmp_path):
    """Compile and link the plain-C example against include/wx.h and
    libwx.so (C99, warnings as errors)."""
    import subprocess
    if not os.path.exists(wx.LIB_PATH):
        from paper_1802_05839_gb300 import build
        build.build()
    exe = str(tmp_path / "c_abi_example")
    libdir = os.path.dirname(wx.LIB_PATH)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-O1",
           os.path.join(ROOT, "tests", "c_abi_example.c"), "-I", os.path.join(ROOT, "include"),
           "-L", libdir, "-lwx", "-Wl,-rpath," + libdir, "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_header_is_plain_c_and_links(tmp_path):
    """include/wx.h compiles as strict C99 and every call the example makes
    resolves against the library (no C++ or CUDA types leak through)."""
    assert os.path.exists(_build_c_example(tmp_path))


@pytest.mark.gpu
def test_c_example_runs(tmp_path):
    import subprocess
    exe = _build_c_example(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "all checks passed" in r.stdout
