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
LIB_PATH = os.path.join(HERE, "libwx.so")

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
    def load_fields(self, T, q, U, V):
        """numpy FP64 (host) or torch FP64 CUDA tensors (device)."""
        dev = hasattr(T, "data_ptr")
        if not dev:
            T, q, U, V = (np.ascontiguousarray(a, np.float64) for a in (T, q, U, V))
        _check(lib().wx_load_fields(self.ptr, _dptr(T), _dptr(q), _dptr(U), _dptr(V), int(dev)),
               self.ptr)

    def read_fields(self, T=None, q=None):
        """FP64 host copies of T and q (into the given arrays, if any)."""
        n = (self.nz, self.ny, self.nx)
        T = np.empty(n) if T is None else T
        q = np.empty(n) if q is None else q
        _check(lib().wx_read_fields(self.ptr, _dptr(T), _dptr(q)), self.ptr)
        return T, q

    def load_state_f32(self, T, q):
        """T and q alone, FP32 (numpy host or torch CUDA); winds kept."""
        dev = hasattr(T, "data_ptr")
        if not dev:
            T, q = (np.ascontiguousarray(a, np.float32) for a in (T, q))
        _check(lib().wx_load_state_f32(self.ptr, _dptr(T), _dptr(q), int(dev)), self.ptr)

    def read_state_f32(self, T=None, q=None):
        """FP32 host copies of T and q (into the given arrays, if any)."""
        n = (self.nz, self.ny, self.nx)
        T = np.empty(n, np.float32) if T is None else T
        q = np.empty(n, np.float32) if q is None else q
        _check(lib().wx_read_state_f32(self.ptr, _dptr(T), _dptr(q)), self.ptr)
        return T, q

    def read_fields_into(self, T, q, stream=None):
        """Device FP64 outputs (torch tensors), asynchronous on `stream`."""
        _check(lib().wx_read_fields_device(self.ptr, _dptr(T), _dptr(q), _stream_ptr(stream)),
               self.ptr)

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
        """Device arrays (torch tensors) of the context's storage type."""
        ncol = Ts.shape[0]
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
    N = B.shape[0]
    if out is None:
        out = torch.empty(M, N, device=A.device, dtype=torch.float32 if epilogue == 0 else torch.bfloat16)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=A.device)
    _mcheck(lib().wx_gemm_bf16(_dptr(A), _dptr(B), M, N, K, epilogue, _dptr(bias), _dptr(aux), _dptr(out),
                               _dptr(out2), _dptr(status), _stream_ptr(stream)))
    return out



# ------------------------------------------------------------------ MLP
MLP_SHAPES = [(512, 232), (512, 512), (512, 512), (116, 512)]  # (fan_out, fan_in)
MLP_IN, MLP_IN_PAD, MLP_OUT, MLP_OUT_PAD = 232, 256, 116, 128
MLP_X_WIDTH = 2 * MLP_IN_PAD  # [hi | lo] two-term BF16 input rows


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

    def fit_norm(self, Ts, qs, kappa_mult, tend, stream=None):
        _mcheck(lib().wx_mlp_fit_norm(self.ptr, _dptr(Ts), _dptr(qs), _dptr(kappa_mult), _dptr(tend),
                                      Ts.shape[0], _stream_ptr(stream)))

    def prepare(self, Ts, qs, kappa_mult, tend, X, Yt=None, stream=None):
        _mcheck(lib().wx_mlp_prepare(self.ptr, _dptr(Ts), _dptr(qs), _dptr(kappa_mult), _dptr(tend),
                                     Ts.shape[0], _dptr(X), _dptr(Yt), _stream_ptr(stream)))

    def forward(self, X, Y, stream=None):
        _mcheck(lib().wx_mlp_forward(self.ptr, _dptr(X), X.shape[0], _dptr(Y), _stream_ptr(stream)))

    def gradients(self, X, Yt, loss=None, stream=None):
        _mcheck(lib().wx_mlp_gradients(self.ptr, _dptr(X), _dptr(Yt), X.shape[0], _dptr(loss),
                                       _stream_ptr(stream)))

    def train_step(self, X, Yt, lr, loss=None, stream=None):
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
        dev = hasattr(E, "data_ptr")
        if not dev:
            E = np.ascontiguousarray(E, np.float64)
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
