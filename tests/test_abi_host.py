"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/*.h declares, and the binding names them all."""
import ctypes
import os
import re

import numpy as np
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


def test_permutation_is_a_seeded_permutation(lib):
    """wx_permutation (host only): every index once, the same draw for the
    same (n, seed), another for another seed; the first draws checked
    against splitmix64 and the multiply-shift bound written out here in
    Python from their published definitions."""
    for n in (0, 1, 2, 17, 4096):
        p = wx.permutation(n, 7)
        assert p.dtype == np.int32 and np.array_equal(np.sort(p), np.arange(n, dtype=np.int32))
    a, b, c = wx.permutation(100_000, 1), wx.permutation(100_000, 1), wx.permutation(100_000, 2)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    # Fisher-Yates from the top, written out independently for n = 50
    M = 2 ** 64 - 1
    state, ref = 12345, list(range(50))
    for i in range(49, 0, -1):
        state = (state + 0x9E3779B97F4A7C15) & M
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        z ^= z >> 31
        r = (z * (i + 1)) >> 64
        ref[i], ref[r] = ref[r], ref[i]
    assert wx.permutation(50, 12345).tolist() == ref
    for bad in (-1, 2 ** 31):
        with pytest.raises(wx.WxError):
            wx.permutation(bad, 0)
