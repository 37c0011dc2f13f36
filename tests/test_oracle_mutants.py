"""The pins catch plausible mistakes in the oracle.  Each case plants one
mistake in a copy of the C oracle (a dropped term, a wrong sign, index,
coefficient or time level), builds it beside the test, and runs the pin
files against it in a child process: at least one pin must fail.  The
unmodified source, built the same way, must pass them all."""
import os
import shutil
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_pins.py", "tests/test_rk3_oracle_pins.py", "tests/test_pf_oracle_pins.py"]

# name -> (text of the correct source, the planted mistake)
MUTANTS = {
    "D1 drops the south neighbour": ("(pe + pw + pn + ps - 4.0 * c)", "(pe + pw + pn - 4.0 * c)"),
    "D1 west neighbour two cells away": ("iw = (i - 1 + nx) % nx;", "iw = (i - 2 + nx) % nx;"),
    "D2 lower flux with the wrong sign": ("Fdn = (c - phi[IDX3(p, i, j, k - 1)]) / g;",
                                          "Fdn = (phi[IDX3(p, i, j, k - 1)] - c) / g;"),
    "D2 without the layer thickness": ("const double Dz = p->kappa_h / p->dz[k] * (Fup - Fdn);",
                                       "const double Dz = p->kappa_h * (Fup - Fdn);"),
    "D3 upwind picks the downwind cell": ("return (u >= 0.0) ? phiL : phiR;", "return (u >= 0.0) ? phiR : phiL;"),
    "D3 west face wind taken at the east face": ("const double Uw = U[IDX2(p, iw, j)];",
                                                 "const double Uw = U[IDX2(p, i, j)];"),
    "D3 south face wind taken at the north neighbour": ("const double Vs = V[IDX2(p, i, js)];",
                                                        "const double Vs = V[IDX2(p, i, jn)];"),
    "D3 flux divergence with the wrong sign": ("Adv = -(1.0 / p->h) * (fe - fw + fn - fs);",
                                               "Adv = (1.0 / p->h) * (fe - fw + fn - fs);"),
    "P1 interface diffusivity from one level": (
        "const double kap = kappa_mult * 0.5 * (kappa_lev[k - 1] + kappa_lev[k]);",
        "const double kap = kappa_mult * kappa_lev[k];"),
    "P1 diagonal with the wrong signs": ("b[k] = 1.0 - a[k] - c[k];", "b[k] = 1.0 + a[k] + c[k];"),
    "P1 elimination divides by b instead of the pivot": ("dp[k] = (r[k] - a[k] * dp[k - 1]) / m;",
                                                         "dp[k] = (r[k] - a[k] * dp[k - 1]) / b[k];"),
    "P1 back substitution with the wrong sign": ("x[k] = dp[k] - cp[k] * x[k + 1];",
                                                 "x[k] = dp[k] + cp[k] * x[k + 1];"),
    "P2 optical depth without the thickness": ("dtau[k] = alpha[k] * dz[k] * qs[k] / q_ref;",
                                               "dtau[k] = alpha[k] * qs[k] / q_ref;"),
    "P2 beam scanned from the bottom": ("for (int k = nz - 1; k >= 0; --k) {\n        const double tau_bot",
                                        "for (int k = 0; k < nz; ++k) {\n        const double tau_bot"),
    "P2 heating added without dt": ("Tout[k] = x[k] + dt * H[k];", "Tout[k] = x[k] + H[k];"),
    "step: physics on the old T": ("    wxo_dynamics(p, T, q, U, V, Ts, qn);\n    physics_all(p, Ts, qn, Tn);",
                                   "    wxo_dynamics(p, T, q, U, V, Ts, qn);\n    physics_all(p, T, qn, Tn);"),
    "step: radiation from the old q": ("    wxo_dynamics(p, T, q, U, V, Ts, qn);\n    physics_all(p, Ts, qn, Tn);",
                                       "    wxo_dynamics(p, T, q, U, V, Ts, qn);\n    physics_all(p, Ts, q, Tn);"),
    "RK3 second stage at dt/3": ("rk3_stage(p, T, q, T1, q1, U, V, p->dt / 2.0, T2, q2);",
                                 "rk3_stage(p, T, q, T1, q1, U, V, p->dt / 3.0, T2, q2);"),
    "RK3 last stage from the first": ("rk3_stage(p, T, q, T2, q2, U, V, p->dt, T3, qn);",
                                      "rk3_stage(p, T, q, T1, q1, U, V, p->dt, T3, qn);"),
    "reduced app: interior keeps 1 - 5d": ("PF_AT(p, E, i, j, k) * (1.0 - 6 * d)", "PF_AT(p, E, i, j, k) * (1.0 - 5 * d)"),
    "reduced app: ghost row reads its inner neighbour's twin": (
        "d * (PF_AT(p, E, i, 1, k) + PF_AT(p, E, i, ny + 1, k))",
        "d * (PF_AT(p, E, i, 1, k) + PF_AT(p, E, i, ny, k))"),
    "reduced app: surface well at the top temperature": ("p->transfer * (x - p->T_surf)",
                                                         "p->transfer * (x - p->T_pbl)"),
}


def _run_pins(tmp_path, source):
    tmp_path.mkdir(parents=True, exist_ok=True)
    src = tmp_path / "wx_oracle.c"
    src.write_text(source)
    shutil.copy(os.path.join(os.path.dirname(oracle._SRC), "wx_oracle.h"), tmp_path)
    lib = oracle.build(openmp=False, src=str(src), out=str(tmp_path / "libwxoracle_copy.so"))
    env = dict(os.environ, WX_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes_every_pin(tmp_path):
    r = _run_pins(tmp_path, open(oracle._SRC).read())
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    good, bad = MUTANTS[name]
    source = open(oracle._SRC).read()
    assert source.count(good) == 1, "the planted text must name one place in the oracle"
    r = _run_pins(tmp_path, source.replace(good, bad))
    assert r.returncode == 1, f"no pin caught '{name}':\n" + r.stdout[-3000:]
