"""The pins catch plausible mistakes in the oracle.  Each case plants one
mistake in a copy of the C oracle (a dropped term, a wrong sign, index,
coefficient or time level) or of the MLP oracle, builds or loads it beside
the test, and runs the pin files against it in a child process: at least
one pin must fail.  The unmodified sources, handled the same way, must pass
them all."""
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


# --------------------------------------------------------------- MLP oracle
MLP_MUTANTS = {
    "bf16 rounds ties away from zero": ("r = ((u + 0x7FFF + lsb) & 0xFFFF0000)", "r = ((u + 0x8000) & 0xFFFF0000)"),
    "input expansion without its low term": ("return hi, bf16(f - hi)", "return hi, 0.0 * hi"),
    "GELU argument not scaled by 1/sqrt(2)": ("return 0.5 * z * (1.0 + erf(z * SQRT_HALF))",
                                             "return 0.5 * z * (1.0 + erf(z))"),
    "GELU derivative without z phi(z)": (
        "return 0.5 * (1.0 + erf(z * SQRT_HALF)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)",
        "return 0.5 * (1.0 + erf(z * SQRT_HALF))"),
    "forward without biases": ("z = h @ rnd(Ws[l]).T + np.asarray(bs[l], dtype=np.float64)",
                               "z = h @ rnd(Ws[l]).T"),
    "MSE gradient without its factor 2": ("return 2.0 * (Y - Yt) / Y.size", "return (Y - Yt) / Y.size"),
    "bias gradient averaged over the batch": ("db[l] = g.sum(axis=0)", "db[l] = g.mean(axis=0)"),
    "Adam without bias correction of m": ("mhat = m / (1.0 - b1 ** t)", "mhat = m"),
    "cosine schedule without its offset": ("return 0.5 * lr0 * (1.0 + np.cos(np.pi * min(step, total) / total))",
                                           "return lr0 * np.cos(np.pi * min(step, total) / total)"),
    "features ignore kappa_mult": ("kv = km[:, None] * np.asarray(kappa_lev, dtype=np.float64)[None, :]",
                                   "kv = np.ones_like(km)[:, None] * np.asarray(kappa_lev, dtype=np.float64)[None, :]"),
    "normalisation std without the mean": ("sd = np.sqrt(np.maximum((F * F).mean(axis=0) - mean * mean, 0.0))",
                                           "sd = np.sqrt(np.maximum((F * F).mean(axis=0), 0.0))"),
    "rho_vd relative to |A T*| instead of |A T* - T*|": ("den = np.linalg.norm(AT - Ts[c])",
                                                          "den = np.linalg.norm(AT)"),
    "rho_H from the thickest layer's optical depth only": ("absorbed = S0 * (1.0 - np.exp(-tau.sum(axis=1)))",
                                                           "absorbed = S0 * (1.0 - np.exp(-tau.max(axis=1)))"),
}

_MLP_RUNNER = """
import importlib.util, sys
import oracle, pytest
spec = importlib.util.spec_from_file_location("oracle.mlp", sys.argv[1])
mod = importlib.util.module_from_spec(spec)
sys.modules["oracle.mlp"] = mod
spec.loader.exec_module(mod)
oracle.mlp = mod
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "tests/test_mlp_oracle_pins.py"]))
"""


def _run_mlp_pins(tmp_path, source):
    path = tmp_path / "mlp.py"
    path.write_text(source)
    return subprocess.run([sys.executable, "-c", _MLP_RUNNER, str(path)], cwd=ROOT, capture_output=True,
                          text=True, timeout=600)


def _mlp_source():
    return open(os.path.join(os.path.dirname(oracle._SRC), "mlp.py")).read()


def test_unmodified_mlp_copy_passes_every_pin(tmp_path):
    r = _run_mlp_pins(tmp_path, _mlp_source())
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name", sorted(MLP_MUTANTS))
def test_planted_mlp_mistake_fails_a_pin(name, tmp_path):
    good, bad = MLP_MUTANTS[name]
    source = _mlp_source()
    assert source.count(good) == 1, "the planted text must name one place in the oracle"
    r = _run_mlp_pins(tmp_path, source.replace(good, bad))
    assert r.returncode == 1, f"no pin caught '{name}':\n" + r.stdout[-3000:] + r.stderr[-2000:]
