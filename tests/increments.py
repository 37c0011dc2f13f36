"""Element-wise increment checks for the FP32 paths (helpers, no tests here).

A per-step bound on the field itself, max|T_g - T_o| / max|T_o| <= 1e-5, is
330 ulp of T ~ 286 K: as large as the whole physics increment of a step at
the paper's configuration (T^{n+1} - T* ~ 2e-3 K ~ 65 ulp), so a physics
error of tens of percent would pass it.  These checks compare the GPU's
increments with the oracle's, element by element:

  physics increment  dP = T^{n+1} - T*   (T* = the oracle's dynamics of the
                                          same input state)
  step increment     dS = T^{n+1} - T^n

    max|dP_g - dP_o| / max|dP_o| <= N_ULP ulp(max|T|) / max|dP_o|

and the same for dS (both numerators are max|T_g - T_o| since T* and T^n
are shared).  N_ULP = 8 is the rounding budget of one FP32 step on a well
conditioned column: about 3.7 ulp for the dynamics (seven rounded
multiply-adds of values ~T and the FP32 rounding of the stencil
coefficients), 3 ulp for the physics (elimination, heating fold and back
substitution, each error damped by |c/m|, |e| << 1), and half an ulp for
storing the result.  `assert_increments` also requires the bar to resolve
the physics (N_ULP ulp / max|dP_o| <= RESOLVE), so a test whose physics
increment is too small to see cannot pass silently.
"""
import numpy as np

N_ULP = 8.0
RESOLVE = 0.25


def ulp32(x):
    return float(np.spacing(np.float32(abs(float(x)))))


def increment_report(T_in, Tstar, Tg, To, mask=None):
    """Errors of the GPU result Tg against the oracle's To for the step from
    T_in (dynamics result Tstar); arrays of one shape, `mask` selects cells."""
    sel = (lambda a: a[mask]) if mask is not None else (lambda a: a.ravel())
    err = float(np.max(np.abs(sel(Tg) - sel(To))))
    ulp = ulp32(np.max(np.abs(To)))
    dP = float(np.max(np.abs(sel(To) - sel(Tstar))))
    dS = float(np.max(np.abs(sel(To) - sel(T_in))))
    return {"err": err, "ulp": ulp, "err_ulp": err / ulp, "dP": dP, "dS": dS,
            "rel_phys": err / dP if dP > 0 else np.inf, "rel_step": err / dS if dS > 0 else np.inf,
            "bar_phys": N_ULP * ulp / dP if dP > 0 else np.inf,
            "bar_step": N_ULP * ulp / dS if dS > 0 else np.inf}


def assert_increments(T_in, Tstar, Tg, To, mask=None, what="", n_ulp=N_ULP, resolve=RESOLVE):
    r = increment_report(T_in, Tstar, Tg, To, mask)
    bar_p = n_ulp * r["ulp"] / r["dP"]
    bar_s = n_ulp * r["ulp"] / r["dS"]
    msg = (f"{what}: err {r['err']:.3e} K = {r['err_ulp']:.2f} ulp; physics increment {r['dP']:.3e} K "
           f"(rel {r['rel_phys']:.3e}, bar {bar_p:.3e}); step increment {r['dS']:.3e} K "
           f"(rel {r['rel_step']:.3e}, bar {bar_s:.3e})")
    assert bar_p <= resolve, "the bar cannot resolve the physics increment: " + msg
    assert r["rel_phys"] <= bar_p, msg
    assert r["rel_step"] <= bar_s, msg
    return r


def strong_physics(case):
    """The same case with a physics increment hundreds of times the FP32
    resolution: a level-to-level zig-zag of +-5 K on T (second differences of
    ~20 K for the vertical diffusion), ten times the vertical diffusivity,
    and S0 = 100 for the heating.  The dynamics' stability does not depend
    on either change (the vertical diffusion is implicit)."""
    c = case.copy()
    k = np.arange(c.nz)
    c.T = c.T + 5.0 * ((-1.0) ** k)[:, None, None]
    c.kappa_lev = c.kappa_lev * 10.0
    c.S0 = 100.0
    return c
