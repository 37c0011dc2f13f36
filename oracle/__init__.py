"""FP64 CPU oracle of the weather step (ctypes wrapper around wx_oracle.c).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers allowed.  Nothing here is
shared with the CUDA library: the C source has its own header, and this
wrapper only marshals numpy arrays.  ``build()`` compiles the C source with
gcc (``-ffp-contract=off`` so the arithmetic is exactly what the source
says); loading fails loudly when the library is missing.

The step it computes is documented in ``wx_oracle.h``: paper Eq. 1 (explicit
Euler heat diffusion, Sec. 3.1) with zero-flux vertical ends and periodic
horizontal boundaries as in the appendix diffusion listing, plus upwind
C-grid advection, a per-column implicit vertical-diffusion Thomas solve and
a top-down optical-depth scan giving radiative heating.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wx_oracle.c")
_LIB = os.path.join(_HERE, "libwxoracle.so")
# A test may point the wrapper at another build of the oracle (a copy with a
# planted mistake, to check that the pins catch it); it is loaded as is.
_LIB_OVERRIDE = os.environ.get("WX_ORACLE_LIB")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dt", ctypes.c_double), ("h", ctypes.c_double),
        ("kappa_h", ctypes.c_double), ("S0", ctypes.c_double),
        ("q_ref", ctypes.c_double),
        ("dz", _D), ("kappa_lev", _D), ("alpha", _D), ("kappa_mult", _D),
        ("advection", ctypes.c_int), ("physics", ctypes.c_int),
    ]


def build(openmp: bool = True, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle (``src``, default wx_oracle.c) into ``out``
    (default ``oracle/libwxoracle.so``); returns the library's path."""
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", src, "-o", out, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError as e:
        if openmp:  # toolchains without libgomp still get a serial oracle
            return build(openmp=False, src=src, out=out)
        raise RuntimeError("oracle build failed:\n" + e.stderr) from e
    return out


def lib():
    global _lib
    if _lib is None:
        path = _LIB_OVERRIDE or _LIB
        if not _LIB_OVERRIDE and (not os.path.exists(_LIB) or
                                  os.path.getmtime(_LIB) < os.path.getmtime(_SRC)):
            build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(_Params)
        L.wxo_dynamics.argtypes = [P, _D, _D, _D, _D, _D, _D]
        L.wxo_vdiff_coeffs.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D,
                                       ctypes.c_double, _D, _D, _D]
        L.wxo_thomas.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D]
        L.wxo_radiation.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double,
                                    ctypes.c_double, _D]
        L.wxo_physics_columns.argtypes = [ctypes.c_int, ctypes.c_long,
                                          ctypes.c_double, _D, _D, _D, _D,
                                          ctypes.c_double, ctypes.c_double,
                                          _D, _D, _D, _D]
        L.wxo_step.argtypes = [P, _D, _D, _D, _D, _D, _D]
        L.wxo_step_columns.argtypes = [P, _D, _D, _D, _D, ctypes.c_long,
                                       ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), _D, _D]
        L.wxo_run.argtypes = [P, ctypes.c_int, _D, _D, _D, _D, _D, _D]
        L.wxo_column_weighted_sum.argtypes = [P, _D]
        L.wxo_column_weighted_sum.restype = ctypes.c_double
        L.wxo_threads.restype = ctypes.c_int
        L.wxo_set_threads.argtypes = [ctypes.c_int]
        L.wxo_step_rk3.argtypes = [P, _D, _D, _D, _D, _D, _D]
        L.wxo_run_rk3.argtypes = [P, ctypes.c_int, _D, _D, _D, _D]
        PP = ctypes.POINTER(PFParams)
        L.wxo_pf_step.argtypes = [PP, _D, _D]
        L.wxo_pf_run.argtypes = [PP, ctypes.c_int, _D]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_D)


class _Bound:
    """Holds a _Params struct and keeps the arrays it points to alive."""

    def __init__(self, case, advection=None, physics=None):
        self.dz = _f64(case.dz)
        self.kappa_lev = _f64(case.kappa_lev)
        self.alpha = _f64(case.alpha)
        self.kappa_mult = None if case.kappa_mult is None else _f64(case.kappa_mult)
        adv = case.advection if advection is None else advection
        phys = case.physics if physics is None else physics
        self.s = _Params(case.nx, case.ny, case.nz, case.dt, case.h, case.kappa_h,
                         case.S0, case.q_ref, _ptr(self.dz), _ptr(self.kappa_lev),
                         _ptr(self.alpha), _ptr(self.kappa_mult), int(adv), int(phys))

    def ref(self):
        return ctypes.byref(self.s)


def set_threads(n: int) -> None:
    lib().wxo_set_threads(int(n))


def threads() -> int:
    return int(lib().wxo_threads())


def dynamics(case, T, q, U, V):
    """(T*, q*) of one step's dynamics."""
    b = _Bound(case)
    T, q, U, V = map(_f64, (T, q, U, V))
    Ts, qs = np.empty_like(T), np.empty_like(q)
    lib().wxo_dynamics(b.ref(), _ptr(T), _ptr(q), _ptr(U), _ptr(V), _ptr(Ts), _ptr(qs))
    return Ts, qs


def step(case, T, q, U, V):
    """One full step: returns (T^{n+1}, q^{n+1})."""
    b = _Bound(case)
    T, q, U, V = map(_f64, (T, q, U, V))
    Tn, qn = np.empty_like(T), np.empty_like(q)
    lib().wxo_step(b.ref(), _ptr(T), _ptr(q), _ptr(U), _ptr(V), _ptr(Tn), _ptr(qn))
    return Tn, qn


def step_columns(case, T, q, U, V, ci, cj):
    """The step's (T^{n+1}, q^{n+1}) at sampled columns (ci[c], cj[c]),
    each [ncol][nz]."""
    b = _Bound(case)
    T, q, U, V = map(_f64, (T, q, U, V))
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    cj = np.ascontiguousarray(cj, dtype=np.int32)
    n = ci.shape[0]
    Tn, qn = np.empty((n, case.nz)), np.empty((n, case.nz))
    IP = ctypes.POINTER(ctypes.c_int)
    lib().wxo_step_columns(b.ref(), _ptr(T), _ptr(q), _ptr(U), _ptr(V), n,
                           ci.ctypes.data_as(IP), cj.ctypes.data_as(IP), _ptr(Tn), _ptr(qn))
    return Tn, qn


def run(case, n_steps, T, q, U, V, sums=False):
    """n_steps steps; returns (T, q) or (T, q, mass_q[n], energy_T[n])."""
    b = _Bound(case)
    T, q = _f64(T).copy(), _f64(q).copy()
    U, V = _f64(U), _f64(V)
    m = np.zeros(max(n_steps, 1)) if sums else None
    e = np.zeros(max(n_steps, 1)) if sums else None
    lib().wxo_run(b.ref(), int(n_steps), _ptr(T), _ptr(q), _ptr(U), _ptr(V), _ptr(m), _ptr(e))
    if sums:
        return T, q, m[:n_steps], e[:n_steps]
    return T, q


def step_rk3(case, T, q, U, V):
    """One step with RK3 dynamics (wxo_step_rk3)."""
    b = _Bound(case)
    T, q, U, V = map(_f64, (T, q, U, V))
    Tn, qn = np.empty_like(T), np.empty_like(q)
    lib().wxo_step_rk3(b.ref(), _ptr(T), _ptr(q), _ptr(U), _ptr(V), _ptr(Tn), _ptr(qn))
    return Tn, qn


def run_rk3(case, n_steps, T, q, U, V):
    b = _Bound(case)
    T, q = _f64(T).copy(), _f64(q).copy()
    U, V = _f64(U), _f64(V)
    lib().wxo_run_rk3(b.ref(), int(n_steps), _ptr(T), _ptr(q), _ptr(U), _ptr(V))
    return T, q


def weighted_sum(case, phi):
    """h^2 * sum(phi * dz_k) in fixed order k, j, i."""
    b = _Bound(case)
    phi = _f64(phi)
    return float(lib().wxo_column_weighted_sum(b.ref(), _ptr(phi)))


def vdiff_coeffs(nz, dt, dz, kappa_lev, kappa_mult=1.0):
    """(a, b, c) of the implicit vertical-diffusion system of one column."""
    dz, kl = _f64(dz), _f64(kappa_lev)
    a, bb, c = np.empty(nz), np.empty(nz), np.empty(nz)
    lib().wxo_vdiff_coeffs(int(nz), float(dt), _ptr(dz), _ptr(kl), float(kappa_mult),
                           _ptr(a), _ptr(bb), _ptr(c))
    return a, bb, c


def thomas(a, b, c, r):
    a, b, c, r = map(_f64, (a, b, c, r))
    x = np.empty_like(r)
    lib().wxo_thomas(int(r.shape[0]), _ptr(a), _ptr(b), _ptr(c), _ptr(r), _ptr(x))
    return x


def radiation(qs, alpha, dz, S0, q_ref):
    qs, alpha, dz = map(_f64, (qs, alpha, dz))
    H = np.empty_like(qs)
    lib().wxo_radiation(int(qs.shape[0]), _ptr(qs), _ptr(alpha), _ptr(dz), float(S0),
                        float(q_ref), _ptr(H))
    return H


def physics_columns(nz, dt, dz, kappa_lev, kappa_mult, alpha, S0, q_ref, Ts, qs,
                    with_tend=False):
    """Column physics of [ncol][nz] columns; returns Tout (and tend [ncol][2][nz])."""
    Ts, qs = _f64(Ts).reshape(-1, nz), _f64(qs).reshape(-1, nz)
    ncol = Ts.shape[0]
    km = None if kappa_mult is None else _f64(kappa_mult).reshape(ncol)
    Tout = np.empty_like(Ts)
    tend = np.empty((ncol, 2, nz)) if with_tend else None
    lib().wxo_physics_columns(int(nz), int(ncol), float(dt), _ptr(_f64(dz)),
                              _ptr(_f64(kappa_lev)), _ptr(km), _ptr(_f64(alpha)),
                              float(S0), float(q_ref), _ptr(Ts), _ptr(qs),
                              _ptr(Tout), _ptr(tend))
    return (Tout, tend) if with_tend else Tout


# ------------------------------------------------------------------
# The paper's reduced weather application (wxo_pf_* in wx_oracle.h)
class PFParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("d", ctypes.c_double), ("radiation", ctypes.c_double),
                ("transfer", ctypes.c_double), ("T_surf", ctypes.c_double),
                ("T_pbl", ctypes.c_double)]


def pf_params(nx, ny, nz, d=0.1, radiation=0.1, transfer=0.01, T_surf=330.0, T_pbl=200.0):
    return PFParams(int(nx), int(ny), int(nz), float(d), float(radiation), float(transfer),
                    float(T_surf), float(T_pbl))


def pf_step(p, E):
    """One step of the reduced application; E is [nz][ny+2][nx+2]."""
    E = _f64(E)
    En = np.empty_like(E)
    lib().wxo_pf_step(ctypes.byref(p), _ptr(E), _ptr(En))
    return En


def pf_run(p, n_steps, E):
    E = _f64(E).copy()
    lib().wxo_pf_run(ctypes.byref(p), int(n_steps), _ptr(E))
    return E
