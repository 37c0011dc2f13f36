"""Thin ctypes binding of libwx.so (include/wx.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  Loading fails loudly when the library has not been
built (``python -m paper_1802_05839_gb300.build``); there is no fallback.
Functions keep the C names; ``Context`` wraps one ``wx_ctx*``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# WX_LIBRARY names another build of the same ABI to load instead (the
# bounds-checked libwx_bounds.so); it must exist as well
LIB_PATH = os.environ.get("WX_LIBRARY") or os.path.join(HERE, "libwx.so")

WX_F32, WX_F64, WX_MIXED = 0, 1, 2
WX_ADVECTION, WX_PHYSICS, WX_SUMS, WX_SURROGATE, WX_RK3 = 1, 2, 4, 8, 16
STATUS = {0: "WX_OK", -1: "WX_EINVAL", -2: "WX_ENOMEM", -3: "WX_ECUDA", -4: "WX_ECFL",
          -5: "WX_ENONFINITE", -6: "WX_ETIMEOUT", -7: "WX_ESTATE", -8: "WX_EUNSUPPORTED"}
DTYPES = {"f32": WX_F32, "f64": WX_F64, "mixed": WX_MIXED}

_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p


class wx_params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("h", ctypes.c_double), ("kappa_h", ctypes.c_double),
                ("S0", ctypes.c_double), ("q_ref", ctypes.c_double),
                ("dd_threshold", ctypes.c_double),
                ("dz", _D), ("kappa_lev", _D), ("alpha", _D), ("kappa_mult", _D),
                ("flags", ctypes.c_uint)]


class WxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None

# (name, restype, argtypes) of every entry point declared in include/wx.h
SIGNATURES = [
    ("wx_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(_VP)]),
    ("wx_set_params", ctypes.c_int, [_VP, ctypes.POINTER(wx_params)]),
    ("wx_load_fields", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int]),
    ("wx_step", ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    ("wx_sync", ctypes.c_int, [_VP]),
    ("wx_read_fields", ctypes.c_int, [_VP, _VP, _VP]),
    ("wx_read_fields_device", ctypes.c_int, [_VP, _VP, _VP, _VP]),
    ("wx_load_state_f32", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int]),
    ("wx_read_state_f32", ctypes.c_int, [_VP, _VP, _VP]),
    ("wx_load_state_f32_async", ctypes.c_int, [_VP, _VP, _VP, _VP]),
    ("wx_read_state_f32_async", ctypes.c_int, [_VP, _VP, _VP, _VP]),
    ("wx_get_sums", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("wx_physics_columns", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_long, _VP]),
    ("wx_info", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long)]),
    ("wx_last_launches", ctypes.c_long, [_VP]),
    ("wx_flagged_columns", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_long)]),
    ("wx_set_step_config", ctypes.c_int, [_VP] + [ctypes.c_int] * 5),
    ("wx_get_step_config", ctypes.c_int, [_VP] + [ctypes.POINTER(ctypes.c_int)] * 6),
    ("wx_sums_noalloc", ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, _VP, ctypes.c_double, _VP, _VP]),
    ("wx_sums_noalloc_error", ctypes.c_char_p, []),
    ("wx_tune", ctypes.c_int, [_VP, ctypes.c_char_p, ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_double)]),
    ("wx_ens_create", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(_VP)]),
    ("wx_ens_size", ctypes.c_int, [_VP]),
    ("wx_ens_member", _VP, [_VP, ctypes.c_int]),
    ("wx_ens_step", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP]),
    ("wx_ens_sync", ctypes.c_int, [_VP]),
    ("wx_ens_set_step_config", ctypes.c_int, [_VP] + [ctypes.c_int] * 5),
    ("wx_ens_get_step_config", ctypes.c_int, [_VP] + [ctypes.POINTER(ctypes.c_int)] * 5),
    ("wx_ens_tune", ctypes.c_int, [_VP, ctypes.c_char_p, ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_double)]),
    ("wx_ens_last_launches", ctypes.c_long, [_VP]),
    ("wx_ens_destroy", None, [_VP]),
    ("wx_ens_last_error", ctypes.c_char_p, [_VP]),
    ("wx_dom_halo_plan", ctypes.c_int, [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_int)] * 2 +
     [ctypes.c_int, _VP]),
    ("wx_dom_create", ctypes.c_int, [ctypes.c_int] * 6 + [ctypes.POINTER(ctypes.c_int)] * 2 +
     [ctypes.POINTER(_VP)]),
    ("wx_dom_set_params", ctypes.c_int, [_VP, ctypes.POINTER(wx_params)]),
    ("wx_dom_load_fields", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    ("wx_dom_step", ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    ("wx_dom_sync", ctypes.c_int, [_VP]),
    ("wx_dom_read_fields", ctypes.c_int, [_VP, _VP, _VP]),
    ("wx_dom_get_sums", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("wx_dom_size", ctypes.c_int, [_VP]),
    ("wx_dom_block", _VP, [_VP, ctypes.c_int]),
    ("wx_dom_last_launches", ctypes.c_long, [_VP]),
    ("wx_dom_destroy", None, [_VP]),
    ("wx_dom_last_error", ctypes.c_char_p, [_VP]),
    ("wx_gemm_bf16", ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP,
                                    _VP, _VP, _VP, _VP, _VP]),
    ("wx_mlp_last_error", ctypes.c_char_p, []),
    ("wx_mlp_create", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_VP)]),
    ("wx_mlp_destroy", None, [_VP]),
    ("wx_mlp_set_weights", ctypes.c_int, [_VP, _VP, _VP]),
    ("wx_mlp_get_weights", ctypes.c_int, [_VP, _VP, _VP]),
    ("wx_mlp_get_grads", ctypes.c_int, [_VP, _VP, _VP]),
    ("wx_mlp_set_norm", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    ("wx_mlp_get_norm", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    ("wx_mlp_set_levels", ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP]),
    ("wx_mlp_fit_norm", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_long, _VP]),
    ("wx_mlp_prepare", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_long, _VP, _VP, _VP]),
    ("wx_mlp_forward", ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP]),
    ("wx_mlp_gradients", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP]),
    ("wx_mlp_train_step", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_float, _VP, _VP]),
    ("wx_mlp_status", ctypes.c_int, [_VP]),
    ("wx_set_surrogate", ctypes.c_int, [_VP, _VP, ctypes.c_double]),
    ("wx_selftest_wait_timeout", ctypes.c_int, [ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_ulonglong)]),
    ("wx_pf_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(_VP)]),
    ("wx_pf_set_params", ctypes.c_int, [_VP] + [ctypes.c_double] * 5),
    ("wx_pf_set_launch", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("wx_pf_load", ctypes.c_int, [_VP, _VP, ctypes.c_int]),
    ("wx_pf_read", ctypes.c_int, [_VP, _VP]),
    ("wx_pf_step", ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    ("wx_pf_sync", ctypes.c_int, [_VP]),
    ("wx_pf_last_launches", ctypes.c_long, [_VP]),
    ("wx_pf_destroy", None, [_VP]),
    ("wx_pf_last_error", ctypes.c_char_p, [_VP]),
    ("wx_surrogate_fallbacks", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_long)]),
    ("wx_set_surrogate_policy", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    ("wx_read_columns_f32", ctypes.c_int, [_VP, _VP, _VP, _VP]),
    ("wx_mlp_denormalize", ctypes.c_int, [_VP, _VP, ctypes.c_long, _VP, _VP]),
    ("wx_convert", ctypes.c_int, [_VP, _VP, ctypes.c_long, ctypes.c_int, _VP]),
    ("wx_gather_rows", ctypes.c_int, [_VP, ctypes.c_long, ctypes.c_long, _VP, ctypes.c_long, _VP, _VP]),
    ("wx_permutation", ctypes.c_int, [ctypes.c_long, ctypes.c_ulonglong, _VP]),
    ("wx_destroy", None, [_VP]),
    ("wx_last_error", ctypes.c_char_p, [_VP]),
]


def lib():
    """Load libwx.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1802_05839_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code, ctx=None):
    if code != 0:
        msg = lib().wx_last_error(ctx)
        raise WxError(code, msg.decode() if msg else "")


def _dptr(a):
    """Device pointer of a torch tensor, or host pointer of a numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


# Pointers cross the ABI without their sizes or types, so the binding checks
# every array it passes: a wrong dtype or a short buffer would otherwise be
# read or written out of bounds by the library.
def _is_cuda(a):
    return bool(getattr(a, "is_cuda", False))


def _host(a, dtype, n, what):
    """Host input: a C-contiguous numpy copy/view of `dtype` with n elements
    (a CPU torch tensor is taken by value)."""
    if _is_cuda(a):
        raise TypeError(f"{what}: expected a host array, got a CUDA tensor")
    if hasattr(a, "detach"):
        a = a.detach().numpy()
    a = np.ascontiguousarray(a, dtype)
    if a.size != n:
        raise ValueError(f"{what}: {a.size} elements, expected {n}")
    return a


def _out(a, dtype, n, what):
    """Host output written in place: a writable C-contiguous numpy array of
    `dtype` with n elements."""
    if not (isinstance(a, np.ndarray) and a.dtype == np.dtype(dtype) and a.flags.c_contiguous
            and a.flags.writeable):
        raise TypeError(f"{what}: expected a writable C-contiguous numpy {np.dtype(dtype).name} array")
    if a.size != n:
        raise ValueError(f"{what}: {a.size} elements, expected {n}")
    return a


def _dev(t, dtype, min_numel, what, optional=False, exact=False):
    """A CUDA tensor whose pointer crosses the ABI: dtype (a torch dtype name
    such as "float32"), contiguity and at least (exact: exactly) min_numel
    elements."""
    if t is None:
        if optional:
            return None
        raise TypeError(f"{what}: a CUDA tensor is required")
    if not hasattr(t, "data_ptr"):
        raise TypeError(f"{what}: expected a torch CUDA tensor, got {type(t).__name__}")
    if str(t.dtype) != "torch." + dtype:
        raise TypeError(f"{what}: dtype {t.dtype}, expected torch.{dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: not contiguous")
    if t.numel() < min_numel or (exact and t.numel() != min_numel):
        raise ValueError(f"{what}: {t.numel()} elements, need {'' if exact else 'at least '}{min_numel}")
    if not _is_cuda(t):
        raise TypeError(f"{what}: expected a CUDA tensor, got a {t.device} tensor")
    return t


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Context:
    """One wx_ctx*: resident fields of an nx x ny x nz grid."""

    def __init__(self, nx, ny, nz, dtype="f32"):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dtype = dtype
        p = _VP()
        _check(lib().wx_create(self.nx, self.ny, self.nz, DTYPES[dtype], ctypes.byref(p)))
        self.ptr = p
        self._keep = None

    def close(self):
        if getattr(self, "ptr", None):
            lib().wx_destroy(self.ptr)
            self.ptr = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- parameters ----------------------------------------------------
    def set_params(self, case, flags=None, dd_threshold=0.0):
        if flags is None:
            flags = (WX_ADVECTION if case.advection else 0) | (WX_PHYSICS if case.physics else 0)
        arr = lambda a: None if a is None else np.ascontiguousarray(a, np.float64).reshape(-1)
        keep = [arr(case.dz), arr(case.kappa_lev), arr(case.alpha), arr(case.kappa_mult)]
        ptr = lambda a: None if a is None else a.ctypes.data_as(_D)
        p = wx_params(case.dt, case.h, case.kappa_h, case.S0, case.q_ref, dd_threshold,
                      ptr(keep[0]), ptr(keep[1]), ptr(keep[2]), ptr(keep[3]), flags)
        self._keep = keep
        _check(lib().wx_set_params(self.ptr, ctypes.byref(p)), self.ptr)

    # -- state ---------------------------------------------------------
    def _n3(self):
        return self.nx * self.ny * self.nz

    def load_fields(self, T, q, U, V):
        """numpy FP64 (host) or torch FP64 CUDA tensors (device): T, q
        [nz][ny][nx], U, V [ny][nx]."""
        n3, n2 = self._n3(), self.nx * self.ny
        dev = _is_cuda(T)
        if dev:
            T, q = _dev(T, "float64", n3, "T", exact=True), _dev(q, "float64", n3, "q", exact=True)
            U, V = _dev(U, "float64", n2, "U", exact=True), _dev(V, "float64", n2, "V", exact=True)
        else:
            T, q = _host(T, np.float64, n3, "T"), _host(q, np.float64, n3, "q")
            U, V = _host(U, np.float64, n2, "U"), _host(V, np.float64, n2, "V")
        _check(lib().wx_load_fields(self.ptr, _dptr(T), _dptr(q), _dptr(U), _dptr(V), int(dev)),
               self.ptr)

    def read_fields(self, T=None, q=None):
        """FP64 host copies of T and q (into the given arrays, if any)."""
        n = (self.nz, self.ny, self.nx)
        T = np.empty(n) if T is None else _out(T, np.float64, self._n3(), "T")
        q = np.empty(n) if q is None else _out(q, np.float64, self._n3(), "q")
        _check(lib().wx_read_fields(self.ptr, _dptr(T), _dptr(q)), self.ptr)
        return T, q

    def load_state_f32(self, T, q):
        """T and q alone, FP32 (numpy host or torch CUDA); winds kept."""
        n3 = self._n3()
        dev = _is_cuda(T)
        if dev:
            T, q = _dev(T, "float32", n3, "T", exact=True), _dev(q, "float32", n3, "q", exact=True)
        else:
            T, q = _host(T, np.float32, n3, "T"), _host(q, np.float32, n3, "q")
        _check(lib().wx_load_state_f32(self.ptr, _dptr(T), _dptr(q), int(dev)), self.ptr)

    def read_state_f32(self, T=None, q=None):
        """FP32 host copies of T and q (into the given arrays, if any)."""
        n = (self.nz, self.ny, self.nx)
        T = np.empty(n, np.float32) if T is None else _out(T, np.float32, self._n3(), "T")
        q = np.empty(n, np.float32) if q is None else _out(q, np.float32, self._n3(), "q")
        _check(lib().wx_read_state_f32(self.ptr, _dptr(T), _dptr(q)), self.ptr)
        return T, q

    def load_state_f32_async(self, T, q, stream=None):
        """Enqueue the upload of pinned host FP32 T, q on `stream`."""
        n3 = self._n3()
        T, q = _host(T, np.float32, n3, "T"), _host(q, np.float32, n3, "q")
        _check(lib().wx_load_state_f32_async(self.ptr, _dptr(T), _dptr(q), _stream_ptr(stream)), self.ptr)

    def read_state_f32_async(self, T, q, stream=None):
        """Enqueue the download into pinned host FP32 arrays T, q on `stream`."""
        T, q = _out(T, np.float32, self._n3(), "T"), _out(q, np.float32, self._n3(), "q")
        _check(lib().wx_read_state_f32_async(self.ptr, _dptr(T), _dptr(q), _stream_ptr(stream)), self.ptr)

    def read_fields_into(self, T, q, stream=None):
        """Device FP64 outputs (torch tensors, either may be None), asynchronous
        on `stream`."""
        T = _dev(T, "float64", self._n3(), "T", optional=True)
        q = _dev(q, "float64", self._n3(), "q", optional=True)
        _check(lib().wx_read_fields_device(self.ptr, _dptr(T), _dptr(q), _stream_ptr(stream)),
               self.ptr)

    def read_columns_into(self, T, q, stream=None):
        """Device FP32 columns [nx*ny][nz] of T and q (torch tensors, either
        may be None), asynchronous on `stream`."""
        n = self._n3()
        T = _dev(T, "float32", n, "T", optional=True, exact=True)
        q = _dev(q, "float32", n, "q", optional=True, exact=True)
        _check(lib().wx_read_columns_f32(self.ptr, _dptr(T), _dptr(q), _stream_ptr(stream)), self.ptr)

    def step(self, n_steps=1, stream=None):
        _check(lib().wx_step(self.ptr, int(n_steps), _stream_ptr(stream)), self.ptr)

    def sync(self):
        _check(lib().wx_sync(self.ptr), self.ptr)

    def sums(self, max_steps=4096):
        m, e = np.empty(max_steps), np.empty(max_steps)
        n = ctypes.c_int(0)
        _check(lib().wx_get_sums(self.ptr, _dptr(m), _dptr(e), max_steps, ctypes.byref(n)), self.ptr)
        return m[:n.value], e[:n.value]

    def physics_columns(self, Ts, qs, kappa_mult, Tout, tend=None, stream=None):
        """Device arrays (torch tensors) of the context's storage type: Ts, qs
        [ncol][nz] in, kappa_mult [ncol] or None, Tout [ncol][nz] out, tend
        [ncol][2][nz] out or None."""
        st = "float64" if self.dtype == "f64" else "float32"
        ncol = int(Ts.shape[0]) if hasattr(Ts, "shape") else 0
        n = ncol * self.nz
        Ts, qs = _dev(Ts, st, n, "Ts"), _dev(qs, st, n, "qs")
        if Ts.numel() != n or qs.numel() != n:
            raise ValueError(f"Ts, qs: expected [{ncol}][{self.nz}]")
        kappa_mult = _dev(kappa_mult, st, ncol, "kappa_mult", optional=True, exact=True)
        Tout = _dev(Tout, st, n, "Tout")
        tend = _dev(tend, st, 2 * n, "tend", optional=True)
        _check(lib().wx_physics_columns(self.ptr, _dptr(Ts), _dptr(qs), _dptr(kappa_mult),
                                        _dptr(Tout), _dptr(tend), ncol, _stream_ptr(stream)),
               self.ptr)

    def info(self):
        v = [ctypes.c_int() for _ in range(4)]
        pitch, nbytes = ctypes.c_long(), ctypes.c_long()
        _check(lib().wx_info(self.ptr, *[ctypes.byref(x) for x in v], ctypes.byref(pitch),
                             ctypes.byref(nbytes)))
        return dict(nx=v[0].value, ny=v[1].value, nz=v[2].value, dtype=v[3].value,
                    pitch=pitch.value, device_bytes=nbytes.value)

    def set_step_config(self, ty, kb, stages, ctas_per_sm, prefetch=0):
        _check(lib().wx_set_step_config(self.ptr, ty, kb, stages, ctas_per_sm, prefetch), self.ptr)

    def step_config(self):
        v = [ctypes.c_int() for _ in range(6)]
        _check(lib().wx_get_step_config(self.ptr, *[ctypes.byref(x) for x in v]), self.ptr)
        return dict(zip(("ty", "kb", "stages", "ctas_per_sm", "prefetch", "smem_bytes"), (x.value for x in v)))

    def flagged_columns(self):
        n = ctypes.c_long()
        _check(lib().wx_flagged_columns(self.ptr, ctypes.byref(n)), self.ptr)
        return n.value

    def last_launches(self):
        return int(lib().wx_last_launches(self.ptr))

    def set_surrogate(self, mlp, fallback_tol=2e-2):
        """Attach an MLP (or detach with None) for steps with WX_SURROGATE."""
        _check(lib().wx_set_surrogate(self.ptr, mlp.ptr if mlp is not None else None,
                                      float(fallback_tol)), self.ptr)
        self._mlp = mlp

    def set_surrogate_policy(self, min_accept, probe_every=8, probe_rows=16):
        """Run the network only while its acceptance is >= min_accept (0: always)."""
        _check(lib().wx_set_surrogate_policy(self.ptr, float(min_accept), int(probe_every), int(probe_rows)),
               self.ptr)

    def surrogate_fallbacks(self):
        n = ctypes.c_long()
        _check(lib().wx_surrogate_fallbacks(self.ptr, ctypes.byref(n)), self.ptr)
        return n.value

    def tune(self, cache_path=None, force=False, stream=None):
        """Autotune the launch configuration (state restored); returns ms/step."""
        ms = ctypes.c_double()
        _check(lib().wx_tune(self.ptr, cache_path.encode() if cache_path else None, int(force),
                             _stream_ptr(stream), ctypes.byref(ms)), self.ptr)
        return ms.value


class _Member(Context):
    """A member context owned by an Ensemble (never destroyed on its own)."""

    def __init__(self, ptr, nx, ny, nz, dtype):
        self.ptr, self.nx, self.ny, self.nz, self.dtype = ptr, nx, ny, nz, dtype
        self._keep = None

    def close(self):
        self.ptr = None

    __del__ = close


def _echeck(code, e):
    if code != 0:
        msg = lib().wx_ens_last_error(e)
        raise WxError(code, msg.decode() if msg else "")


class Ensemble:
    """Up to 16 grids of uneven sizes stepped by one persistent launch per
    step (replayed from a CUDA graph)."""

    def __init__(self, sizes, dtype="f32"):
        m = len(sizes)
        arr = lambda k: (ctypes.c_int * m)(*[int(s[k]) for s in sizes])
        p = _VP()
        _echeck(lib().wx_ens_create(m, arr(0), arr(1), arr(2), DTYPES[dtype], ctypes.byref(p)), None)
        self.ptr = p
        self.members = [_Member(_VP(lib().wx_ens_member(p, i)), *sizes[i], dtype) for i in range(m)]

    def close(self):
        if getattr(self, "ptr", None):
            for mem in self.members:
                mem.ptr = None
            lib().wx_ens_destroy(self.ptr)
            self.ptr = None

    __del__ = close

    def step(self, n_steps=1, graph=True, stream=None):
        _echeck(lib().wx_ens_step(self.ptr, int(n_steps), int(graph), _stream_ptr(stream)), self.ptr)

    def sync(self):
        _echeck(lib().wx_ens_sync(self.ptr), self.ptr)

    def set_step_config(self, ty, kb, stages, ctas_per_sm, prefetch=0):
        _echeck(lib().wx_ens_set_step_config(self.ptr, ty, kb, stages, ctas_per_sm, prefetch), self.ptr)

    def step_config(self):
        v = [ctypes.c_int() for _ in range(5)]
        _echeck(lib().wx_ens_get_step_config(self.ptr, *[ctypes.byref(x) for x in v]), self.ptr)
        return dict(zip(("ty", "kb", "stages", "ctas_per_sm", "prefetch"), (x.value for x in v)))

    def tune(self, cache_path=None, force=False, stream=None):
        ms = ctypes.c_double()
        _echeck(lib().wx_ens_tune(self.ptr, cache_path.encode() if cache_path else None, int(force),
                                  _stream_ptr(stream), ctypes.byref(ms)), self.ptr)
        return ms.value

    def last_launches(self):
        return int(lib().wx_ens_last_launches(self.ptr))


def wx_sums_noalloc(T, q, dz, h, out, stream=None):
    """FP64 (mass_q, energy_T) sums of device fields T, q [nz][ny][nx] (torch
    float32 or float64 CUDA tensors) into the device tensor out[2], with no
    device allocation (see include/wx.h)."""
    import torch
    nz, ny, nx = T.shape
    dtype = WX_F32 if T.dtype == torch.float32 else WX_F64
    name = "float32" if dtype == WX_F32 else "float64"
    T, q = _dev(T, name, nx * ny * nz, "T", exact=True), _dev(q, name, nx * ny * nz, "q", exact=True)
    dz, out = _dev(dz, "float64", nz, "dz", exact=True), _dev(out, "float64", 2, "out")
    code = lib().wx_sums_noalloc(_dptr(T), _dptr(q), dtype, nx, ny, nz, _dptr(dz), float(h),
                                 _dptr(out), _stream_ptr(stream))
    if code != 0:
        raise WxError(code, lib().wx_sums_noalloc_error().decode())


def _mcheck(code):
    if code != 0:
        raise WxError(code, lib().wx_mlp_last_error().decode())


def wx_gemm_bf16(A, B, epilogue=0, bias=None, aux=None, out=None, out2=None, status=None, stream=None):
    """C = A . B^T (torch BF16 CUDA tensors A [M][K], B [N][K]) with an epilogue."""
    import torch
    M, K = A.shape
    N, KB = B.shape
    if KB != K:
        raise ValueError(f"A is [{M}][{K}] but B is [{N}][{KB}]")
    A, B = _dev(A, "bfloat16", M * K, "A", exact=True), _dev(B, "bfloat16", N * K, "B", exact=True)
    if out is None:
        out = torch.empty(M, N, device=A.device, dtype=torch.float32 if epilogue == 0 else torch.bfloat16)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=A.device)
    out = _dev(out, "float32" if epilogue == 0 else "bfloat16", M * N, "out")
    out2 = _dev(out2, "bfloat16", M * N, "out2", optional=True)
    bias = _dev(bias, "float32", N, "bias", optional=True)
    aux = _dev(aux, "bfloat16", M * N, "aux", optional=epilogue != 2)
    status = _dev(status, "int32", 1, "status")
    _mcheck(lib().wx_gemm_bf16(_dptr(A), _dptr(B), M, N, K, epilogue, _dptr(bias), _dptr(aux), _dptr(out),
                               _dptr(out2), _dptr(status), _stream_ptr(stream)))
    return out



# ------------------------------------------------------------------ MLP
MLP_SHAPES = [(512, 232), (512, 512), (512, 512), (116, 512)]  # (fan_out, fan_in)
MLP_IN, MLP_IN_PAD, MLP_OUT, MLP_OUT_PAD = 232, 256, 116, 128
MLP_X_WIDTH = 2 * MLP_IN_PAD  # [hi | lo] two-term BF16 input rows
MLP_NZ = 58                    # levels of the columns the network serves


def _f32arrays(arrs):
    arrs = [np.ascontiguousarray(a, np.float32) for a in arrs]
    ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    return arrs, ptrs


class MLP:
    """One wx_mlp*: the column-physics surrogate network (include/wx.h)."""

    def __init__(self, max_batch=4096):
        p = _VP()
        _mcheck(lib().wx_mlp_create(int(max_batch), ctypes.byref(p)))
        self.ptr = p
        self.max_batch = int(max_batch)

    def close(self):
        if getattr(self, "ptr", None):
            lib().wx_mlp_destroy(self.ptr)
            self.ptr = None

    __del__ = close

    def set_weights(self, Ws, bs):
        (Wk, Wp), (bk, bp) = _f32arrays(Ws), _f32arrays(bs)
        _mcheck(lib().wx_mlp_set_weights(self.ptr, Wp, bp))

    def _get(self, fn):
        Ws = [np.empty(s, np.float32) for s in MLP_SHAPES]
        bs = [np.empty(s[0], np.float32) for s in MLP_SHAPES]
        wp = (ctypes.c_void_p * 4)(*[a.ctypes.data for a in Ws])
        bp = (ctypes.c_void_p * 4)(*[a.ctypes.data for a in bs])
        _mcheck(fn(self.ptr, wp, bp))
        return Ws, bs

    def get_weights(self):
        return self._get(lib().wx_mlp_get_weights)

    def get_grads(self):
        return self._get(lib().wx_mlp_get_grads)

    def set_norm(self, mean_in, std_in, mean_out, std_out):
        a, _ = _f32arrays([mean_in, std_in, mean_out, std_out])
        _mcheck(lib().wx_mlp_set_norm(self.ptr, *[_dptr(x) for x in a]))

    def get_norm(self):
        a = [np.empty(MLP_IN, np.float32), np.empty(MLP_IN, np.float32),
             np.empty(MLP_OUT, np.float32), np.empty(MLP_OUT, np.float32)]
        _mcheck(lib().wx_mlp_get_norm(self.ptr, *[_dptr(x) for x in a]))
        return a

    def set_levels(self, kappa_lev, alpha_dz):
        a, _ = _f32arrays([kappa_lev, alpha_dz])
        _mcheck(lib().wx_mlp_set_levels(self.ptr, len(a[0]), _dptr(a[0]), _dptr(a[1])))

    @staticmethod
    def _columns(Ts, qs, kappa_mult, tend, tend_optional):
        ncol = int(Ts.shape[0]) if hasattr(Ts, "shape") else 0
        n = ncol * MLP_NZ
        Ts, qs = _dev(Ts, "float32", n, "Ts"), _dev(qs, "float32", n, "qs")
        if Ts.numel() != n or qs.numel() != n:
            raise ValueError(f"Ts, qs: expected [{ncol}][{MLP_NZ}]")
        kappa_mult = _dev(kappa_mult, "float32", ncol, "kappa_mult", optional=True, exact=True)
        tend = _dev(tend, "float32", 2 * n, "tend", optional=tend_optional)
        return ncol, Ts, qs, kappa_mult, tend

    def _rows(self, X, what="X"):
        M = int(X.shape[0]) if hasattr(X, "shape") else 0
        X = _dev(X, "bfloat16", M * MLP_X_WIDTH, what)
        if X.numel() != M * MLP_X_WIDTH:
            raise ValueError(f"{what}: expected [M][{MLP_X_WIDTH}]")
        return M, X

    def fit_norm(self, Ts, qs, kappa_mult, tend, stream=None):
        _, Ts, qs, kappa_mult, tend = self._columns(Ts, qs, kappa_mult, tend, False)
        _mcheck(lib().wx_mlp_fit_norm(self.ptr, _dptr(Ts), _dptr(qs), _dptr(kappa_mult), _dptr(tend),
                                      Ts.shape[0], _stream_ptr(stream)))

    def prepare(self, Ts, qs, kappa_mult, tend, X, Yt=None, stream=None):
        ncol, Ts, qs, kappa_mult, tend = self._columns(Ts, qs, kappa_mult, tend, Yt is None)
        rows = (ncol + 127) // 128 * 128
        X = _dev(X, "bfloat16", rows * MLP_X_WIDTH, "X")
        Yt = _dev(Yt, "float32", rows * MLP_OUT_PAD, "Yt", optional=True)
        _mcheck(lib().wx_mlp_prepare(self.ptr, _dptr(Ts), _dptr(qs), _dptr(kappa_mult), _dptr(tend),
                                     Ts.shape[0], _dptr(X), _dptr(Yt), _stream_ptr(stream)))

    def forward(self, X, Y, stream=None):
        M, X = self._rows(X)
        Y = _dev(Y, "float32", M * MLP_OUT_PAD, "Y")
        _mcheck(lib().wx_mlp_forward(self.ptr, _dptr(X), X.shape[0], _dptr(Y), _stream_ptr(stream)))

    def gradients(self, X, Yt, loss=None, stream=None):
        M, X = self._rows(X)
        Yt = _dev(Yt, "float32", M * MLP_OUT_PAD, "Yt")
        loss = _dev(loss, "float32", 1, "loss", optional=True)
        _mcheck(lib().wx_mlp_gradients(self.ptr, _dptr(X), _dptr(Yt), X.shape[0], _dptr(loss),
                                       _stream_ptr(stream)))

    def denormalize(self, Y, out, stream=None):
        """out [M][116] = Y[:, :116] * std_out + mean_out (device FP32)."""
        M = int(Y.shape[0])
        Y = _dev(Y, "float32", M * MLP_OUT_PAD, "Y", exact=True)
        out = _dev(out, "float32", M * MLP_OUT, "out", exact=True)
        _mcheck(lib().wx_mlp_denormalize(self.ptr, _dptr(Y), M, _dptr(out), _stream_ptr(stream)))

    def train_step(self, X, Yt, lr, loss=None, stream=None):
        M, X = self._rows(X)
        Yt = _dev(Yt, "float32", M * MLP_OUT_PAD, "Yt")
        loss = _dev(loss, "float32", 1, "loss", optional=True)
        _mcheck(lib().wx_mlp_train_step(self.ptr, _dptr(X), _dptr(Yt), X.shape[0], float(lr),
                                        _dptr(loss), _stream_ptr(stream)))

    def status(self):
        _mcheck(lib().wx_mlp_status(self.ptr))


# ------------------------------------------------ reduced application
class ReducedApp:
    """One wx_pf*: the paper's reduced weather application (include/wx.h)."""

    def __init__(self, nx, ny, nz, dtype="f64"):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        p = _VP()
        code = lib().wx_pf_create(self.nx, self.ny, self.nz, DTYPES[dtype], ctypes.byref(p))
        if code != 0:
            raise WxError(code, "wx_pf_create")
        self.ptr = p

    def _check(self, code):
        if code != 0:
            raise WxError(code, lib().wx_pf_last_error(self.ptr).decode())

    def close(self):
        if getattr(self, "ptr", None):
            lib().wx_pf_destroy(self.ptr)
            self.ptr = None

    __del__ = close

    def set_params(self, d=0.1, radiation=0.1, transfer=0.01, T_surf=330.0, T_pbl=200.0):
        self._check(lib().wx_pf_set_params(self.ptr, d, radiation, transfer, T_surf, T_pbl))

    def set_launch(self, layout="ijk", block=(32, 8)):
        self._check(lib().wx_pf_set_launch(self.ptr, {"ijk": 0, "kij": 1}[layout], int(block[0]), int(block[1])))

    def load(self, E):
        """The whole state [nz][ny+2][nx+2], FP64, host or CUDA tensor."""
        n = self.nz * (self.ny + 2) * (self.nx + 2)
        dev = _is_cuda(E)
        E = _dev(E, "float64", n, "E", exact=True) if dev else _host(E, np.float64, n, "E")
        self._keep = E
        self._check(lib().wx_pf_load(self.ptr, _dptr(E), int(dev)))

    def read(self):
        E = np.empty((self.nz, self.ny + 2, self.nx + 2))
        self._check(lib().wx_pf_read(self.ptr, _dptr(E)))
        return E

    def step(self, n_steps=1, stream=None):
        self._check(lib().wx_pf_step(self.ptr, int(n_steps), _stream_ptr(stream)))

    def sync(self):
        self._check(lib().wx_pf_sync(self.ptr))

    def last_launches(self):
        return int(lib().wx_pf_last_launches(self.ptr))


def wx_selftest_wait_timeout(limit_ns):
    """(status code, device ns waited) of the bounded-wait self test."""
    w = ctypes.c_ulonglong()
    code = lib().wx_selftest_wait_timeout(int(limit_ns), ctypes.byref(w))
    return code, w.value


# ---------------------------------------------------------------- decomposition
WX_HALO_WEST, WX_HALO_EAST, WX_HALO_SOUTH, WX_HALO_NORTH = 0, 1, 2, 3


class wx_halo_strip(ctypes.Structure):
    _fields_ = [("dir", ctypes.c_int), ("src", ctypes.c_int), ("src_line", ctypes.c_int),
                ("dst_line", ctypes.c_int), ("len", ctypes.c_int)]


def _splits(parts, given):
    if given is None:
        return None
    given = [int(x) for x in given]
    if len(given) != parts + 1:
        raise ValueError(f"split: {len(given)} boundaries, expected {parts + 1}")
    return (ctypes.c_int * (parts + 1))(*given)


def halo_plan(nx, ny, px, py, r, xsplit=None, ysplit=None):
    """The four ghost strips of block r (wx_dom_halo_plan) as dicts with the
    keys dir, src, src_line, dst_line, len.  Host-only: no GPU needed."""
    out = (wx_halo_strip * 4)()
    code = lib().wx_dom_halo_plan(int(nx), int(ny), int(px), int(py), _splits(px, xsplit),
                                  _splits(py, ysplit), int(r), ctypes.cast(out, _VP))
    if code != 0:
        raise WxError(code, "wx_dom_halo_plan: bad sizes or splits")
    return [{k: getattr(s, k) for k, _ in wx_halo_strip._fields_} for s in out]


def _dcheck(code, d):
    if code != 0:
        msg = lib().wx_dom_last_error(d)
        raise WxError(code, msg.decode() if msg else "")


class Decomposition:
    """One periodic nx x ny x nz grid split into px x py blocks stepped with
    a depth-1 halo exchange (wx_dom_*): host FP64 arrays of the whole grid
    in and out."""

    def __init__(self, nx, ny, nz, dtype="f32", px=2, py=1, xsplit=None, ysplit=None):
        self.nx, self.ny, self.nz, self.dtype, self.px, self.py = int(nx), int(ny), int(nz), dtype, px, py
        p = _VP()
        _dcheck(lib().wx_dom_create(self.nx, self.ny, self.nz, DTYPES[dtype], int(px), int(py),
                                    _splits(px, xsplit), _splits(py, ysplit), ctypes.byref(p)), None)
        self.ptr = p
        self._keep = None

    def close(self):
        if getattr(self, "ptr", None):
            lib().wx_dom_destroy(self.ptr)
            self.ptr = None

    __del__ = close

    def set_params(self, case, flags=None, dd_threshold=0.0):
        if flags is None:
            flags = (WX_ADVECTION if case.advection else 0) | (WX_PHYSICS if case.physics else 0)
        n2 = self.nx * self.ny
        arr = lambda a: None if a is None else np.ascontiguousarray(a, np.float64).reshape(-1)
        keep = [arr(case.dz), arr(case.kappa_lev), arr(case.alpha), arr(case.kappa_mult)]
        for a, n, what in zip(keep, (self.nz, self.nz, self.nz, n2), ("dz", "kappa_lev", "alpha", "kappa_mult")):
            if a is not None and a.size != n:
                raise ValueError(f"{what}: {a.size} elements, expected {n}")
        ptr = lambda a: None if a is None else a.ctypes.data_as(_D)
        p = wx_params(case.dt, case.h, case.kappa_h, case.S0, case.q_ref, dd_threshold,
                      ptr(keep[0]), ptr(keep[1]), ptr(keep[2]), ptr(keep[3]), flags)
        self._keep = keep
        _dcheck(lib().wx_dom_set_params(self.ptr, ctypes.byref(p)), self.ptr)

    def load_fields(self, T, q, U, V):
        n3, n2 = self.nx * self.ny * self.nz, self.nx * self.ny
        T, q = _host(T, np.float64, n3, "T"), _host(q, np.float64, n3, "q")
        U, V = _host(U, np.float64, n2, "U"), _host(V, np.float64, n2, "V")
        _dcheck(lib().wx_dom_load_fields(self.ptr, _dptr(T), _dptr(q), _dptr(U), _dptr(V)), self.ptr)

    def step(self, n_steps=1, stream=None):
        _dcheck(lib().wx_dom_step(self.ptr, int(n_steps), _stream_ptr(stream)), self.ptr)

    def sync(self):
        _dcheck(lib().wx_dom_sync(self.ptr), self.ptr)

    def read_fields(self):
        T, q = np.empty((self.nz, self.ny, self.nx)), np.empty((self.nz, self.ny, self.nx))
        _dcheck(lib().wx_dom_read_fields(self.ptr, _dptr(T), _dptr(q)), self.ptr)
        return T, q

    def sums(self, max_steps=4096):
        m, e = np.empty(max_steps), np.empty(max_steps)
        n = ctypes.c_int(0)
        _dcheck(lib().wx_dom_get_sums(self.ptr, _dptr(m), _dptr(e), max_steps, ctypes.byref(n)), self.ptr)
        return m[:n.value], e[:n.value]

    def size(self):
        return int(lib().wx_dom_size(self.ptr))

    def last_launches(self):
        return int(lib().wx_dom_last_launches(self.ptr))

    def block_step_config(self, r=0):
        """Launch configuration of block r (all blocks share it)."""
        b = _Member(_VP(lib().wx_dom_block(self.ptr, int(r))), 0, 0, 0, self.dtype)
        return b.step_config()


def wx_convert(src, dst, stream=None):
    """dst = src converted between FP32 and FP64 (device tensors of one size)."""
    n = src.numel()
    to64 = str(dst.dtype) == "torch.float64"
    src = _dev(src, "float32" if to64 else "float64", n, "src", exact=True)
    dst = _dev(dst, "float64" if to64 else "float32", n, "dst", exact=True)
    code = lib().wx_convert(_dptr(src), _dptr(dst), n, int(to64), _stream_ptr(stream))
    if code != 0:
        raise WxError(code, lib().wx_mlp_last_error().decode())


def permutation(n, seed):
    """A seeded permutation of 0..n-1 (numpy int32, host), drawn by the
    library (wx_permutation: Fisher-Yates with splitmix64)."""
    n = int(n)
    out = np.empty(n if 0 <= n < 2 ** 31 else 0, dtype=np.int32)
    code = lib().wx_permutation(n, int(seed) & (2 ** 64 - 1), out.ctypes.data_as(_VP) if out.size else None)
    if code != 0:
        raise WxError(code, "wx_permutation: n must be in [0, 2^31 - 1]")
    return out


def wx_gather_rows(src, idx, dst, stream=None):
    """dst[r] = src[idx[r]] for rows of a 2-D device tensor (row bytes a
    multiple of 16); idx a device int32 tensor (an index outside src's rows
    gives a zero row)."""
    n = int(idx.numel())
    rb = src.shape[1] * src.element_size()
    if dst.dtype != src.dtype or dst.shape[1] != src.shape[1] or dst.shape[0] < n:
        raise ValueError("wx_gather_rows: dst must hold n rows of src's type and width")
    idx = _dev(idx, "int32", n, "idx", exact=True)
    if not (src.is_contiguous() and dst.is_contiguous()) or not (src.is_cuda and dst.is_cuda):
        raise ValueError("wx_gather_rows: contiguous CUDA tensors required")
    code = lib().wx_gather_rows(_dptr(src), int(src.shape[0]), rb, _dptr(idx), n, _dptr(dst),
                                _stream_ptr(stream))
    if code != 0:
        raise WxError(code, lib().wx_mlp_last_error().decode())
