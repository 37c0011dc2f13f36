"""Pins of the FP64 oracle against facts fixed by the paper and by the
mathematics of the scheme (closed forms, invariants, special cases).

Each test is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign, a wrong upwind side or index, a transposed operand) fails.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1802_05839_gb300 import inputs


def bare_case(nx, ny, nz, *, dt=0.1, h=2.5, kappa_h=0.05, S0=0.0, q_ref=0.01,
              dz=None, kappa_lev=None, kappa_mult=None, advection=False, physics=False):
    z = np.zeros((nz, ny, nx))
    return inputs.Case(nx=nx, ny=ny, nz=nz, dt=dt, h=h, kappa_h=kappa_h, S0=S0,
                       q_ref=q_ref, dz=np.ones(nz) if dz is None else np.asarray(dz, float),
                       kappa_lev=np.full(nz, 0.02) if kappa_lev is None else np.asarray(kappa_lev, float),
                       alpha=inputs.absorber(nz), kappa_mult=kappa_mult, T=z, q=z.copy(),
                       U=np.zeros((ny, nx)), V=np.zeros((ny, nx)),
                       advection=advection, physics=physics)


# ---------------------------------------------------------------- dynamics

@pytest.mark.parametrize("m,n", [(1, 0), (2, 3), (5, 1)])
def test_p1_fourier_mode_horizontal_diffusion(m, n):
    """A single horizontal Fourier mode decays by the discrete Laplacian's
    symbol G = 1 - 4 d_h (sin^2(pi m/nx) + sin^2(pi n/ny)), d_h = kappa dt/h^2."""
    nx, ny, nz, N = 24, 20, 3, 7
    c = bare_case(nx, ny, nz, kappa_h=0.9, h=1.3)
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    phase = 2 * np.pi * (m * i / nx + n * j / ny)
    T0 = np.broadcast_to(5.0 + 2.0 * np.cos(phase), (nz, ny, nx)).copy()
    T, _ = oracle.run(c, N, T0, T0.copy(), c.U, c.V)
    dh = c.kappa_h * c.dt / c.h ** 2
    G = 1 - 4 * dh * (math.sin(math.pi * m / nx) ** 2 + math.sin(math.pi * n / ny) ** 2)
    expect = 5.0 + 2.0 * G ** N * np.cos(phase)
    assert np.max(np.abs(T - expect[None])) < 1e-13 * 7


@pytest.mark.parametrize("p", [1, 2, 5])
def test_vertical_cosine_mode_explicit_zero_flux(p):
    """With uniform dz the explicit vertical term has the cosine modes
    cos(pi p (k+1/2)/nz) as eigenvectors (mirror images at zero-flux ends),
    growth factor 1 - 4 d_z sin^2(pi p/(2 nz)), d_z = kappa dt/dz^2."""
    nx, ny, nz, N = 3, 2, 9, 5
    dz = 1.7
    c = bare_case(nx, ny, nz, kappa_h=0.8, dz=np.full(nz, dz))
    kk = np.arange(nz)
    mode = np.cos(np.pi * p * (kk + 0.5) / nz)
    T0 = np.broadcast_to((3.0 + mode)[:, None, None], (nz, ny, nx)).copy()
    T, _ = oracle.run(c, N, T0, T0.copy(), c.U, c.V)
    G = 1 - 4 * c.kappa_h * c.dt / dz ** 2 * math.sin(math.pi * p / (2 * nz)) ** 2
    expect = 3.0 + G ** N * mode
    assert np.max(np.abs(T - expect[:, None, None])) < 1e-13 * 4


def test_paper_listing_coefficients_uniform_grid():
    """With h = dz = 1 and no wind, one dynamics step is the paper's appendix
    diffusion listing: E(1-6d) + d*(six neighbours) inside and E(1-5d) + d*(five
    neighbours) at the bottom and top levels, d = kappa dt (periodic i, j)."""
    nx, ny, nz = 6, 5, 4
    c = bare_case(nx, ny, nz, h=1.0, kappa_h=0.3, dt=0.25)
    d = c.kappa_h * c.dt
    rng = np.random.default_rng(3)
    E = rng.uniform(200, 330, (nz, ny, nx))
    Ts, _ = oracle.dynamics(c, E, E, c.U, c.V)
    hsum = (np.roll(E, 1, 2) + np.roll(E, -1, 2) + np.roll(E, 1, 1) + np.roll(E, -1, 1))
    exp = np.empty_like(E)
    exp[1:-1] = E[1:-1] * (1 - 6 * d) + d * (hsum[1:-1] + E[:-2] + E[2:])
    exp[0] = E[0] * (1 - 5 * d) + d * (hsum[0] + E[1])
    exp[-1] = E[-1] * (1 - 5 * d) + d * (hsum[-1] + E[-2])
    assert np.max(np.abs(Ts - exp)) < 1e-12


@pytest.mark.parametrize("axis,sign", [("x", 1), ("x", -1), ("y", 1), ("y", -1)])
def test_p2_exact_shift_at_courant_one(axis, sign):
    """Uniform wind with Courant number 1 and no diffusion moves the field by
    exactly one cell downstream, per face and per direction (pins the upwind
    side and the sign of the flux divergence)."""
    nx, ny, nz = 7, 6, 2
    c = bare_case(nx, ny, nz, dt=0.25, h=2.0, kappa_h=0.0, advection=True)
    if axis == "x":
        c.U[:] = sign * 8.0
    else:
        c.V[:] = sign * 8.0
    rng = np.random.default_rng(1)
    T0 = rng.uniform(1, 2, (nz, ny, nx))
    T, _ = oracle.run(c, 3, T0, T0.copy(), c.U, c.V)
    ax = 2 if axis == "x" else 1
    assert np.max(np.abs(T - np.roll(T0, 3 * sign, axis=ax))) < 1e-14 * 2


@pytest.mark.parametrize("C", [0.3, 0.7])
def test_p2_upwind_symbol(C):
    """For Courant C < 1 a mode e^{i theta i} is multiplied per step by the
    first-order upwind symbol G = 1 - C (1 - e^{-i theta})."""
    nx, ny, nz, N, m = 16, 2, 1, 6, 3
    c = bare_case(nx, ny, nz, dt=0.1, h=1.0, kappa_h=0.0, advection=True)
    c.U[:] = C * c.h / c.dt
    theta = 2 * np.pi * m / nx
    i = np.arange(nx)
    T0 = np.broadcast_to(1.0 + np.cos(theta * i), (nz, ny, nx)).copy()
    T, _ = oracle.run(c, N, T0, T0.copy(), c.U, c.V)
    G = 1 - C * (1 - np.exp(-1j * theta))
    expect = 1.0 + np.real(G ** N * np.exp(1j * theta * i))
    assert np.max(np.abs(T[0, 0] - expect)) < 1e-13


def _generated(nx, ny, nz, seed=5, S0=0.0, near_singular=False, physics=True):
    c = inputs.paper_grid_case(nx, ny, nz, seed=seed, near_singular=near_singular)
    c.S0 = S0
    c.physics = physics
    return c


def test_p3_mass_conservation():
    """Periodic x/y, zero-flux z, flux-form advection and the dz-weighted
    conservative implicit solve keep sum(phi dz) constant (S0 = 0)."""
    c = _generated(23, 17, 9, near_singular=True)
    m0 = oracle.weighted_sum(c, c.q)
    e0 = oracle.weighted_sum(c, c.T)
    T, q, m, e = oracle.run(c, 10, c.T, c.q, c.U, c.V, sums=True)
    assert np.max(np.abs(m - m0)) / abs(m0) < 1e-12
    assert np.max(np.abs(e - e0)) / abs(e0) < 1e-12
    # the state itself did change
    assert np.max(np.abs(T - c.T)) > 1e-3


def test_p4_constant_fixed_point():
    """A constant field is a fixed point of the dynamics (discretely
    divergence-free winds) and of the implicit vertical diffusion."""
    c = _generated(19, 13, 7, near_singular=True)
    T0 = np.full((c.nz, c.ny, c.nx), 281.5)
    q0 = np.full((c.nz, c.ny, c.nx), 0.0125)
    T, q = oracle.run(c, 4, T0, q0, c.U, c.V)
    # rounding only: the near-singular columns (kappa_mult up to 1e5) make the
    # implicit solve's condition number ~1e3, so allow a few hundred ulps
    assert np.max(np.abs(T - 281.5)) / 281.5 < 1e-13
    assert np.max(np.abs(q - 0.0125)) < 1e-15


def test_p5_discrete_maximum_principle():
    """With the default constants every coefficient of the explicit update is
    non-negative and they sum to one: the new state is bounded by the old."""
    c = _generated(31, 29, 11, physics=False)
    T, q = c.T, c.q
    for _ in range(3):
        Tn, qn = oracle.step(c, T, q, c.U, c.V)
        assert Tn.min() >= T.min() - 1e-12 and Tn.max() <= T.max() + 1e-12
        assert qn.min() >= q.min() - 1e-15 and qn.max() <= q.max() + 1e-15
        T, q = Tn, qn


# ------------------------------------------------------- implicit vertical

@pytest.mark.parametrize("p", [0, 1, 3, 7])
def test_p6_thomas_vertical_cosine_mode(p):
    """Uniform dz and kappa_v: (I - dt L) has eigenvectors cos(pi p (k+1/2)/nz)
    with eigenvalue 1 + 4 r sin^2(pi p/(2 nz)), r = dt kappa_v/dz^2."""
    nz, dz, kv, dt = 8, 1.3, 0.7, 0.4
    a, b, c = oracle.vdiff_coeffs(nz, dt, np.full(nz, dz), np.full(nz, kv))
    k = np.arange(nz)
    rhs = np.cos(np.pi * p * (k + 0.5) / nz)
    x = oracle.thomas(a, b, c, rhs)
    r = dt * kv / dz ** 2
    assert np.max(np.abs(x - rhs / (1 + 4 * r * math.sin(math.pi * p / (2 * nz)) ** 2))) < 1e-13


def test_p7_thomas_vs_dense_solve():
    """Thomas against numpy's LU with partial pivoting on random diagonally
    dominant 8-level systems."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        n = 8
        a = rng.uniform(-1, 1, n); a[0] = 0
        c = rng.uniform(-1, 1, n); c[-1] = 0
        b = np.abs(a) + np.abs(c) + rng.uniform(0.1, 2, n)
        b *= rng.choice([-1, 1], n)
        r = rng.normal(size=n)
        A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        x = oracle.thomas(a, b, c, r)
        xr = np.linalg.solve(A, r)
        assert np.max(np.abs(x - xr)) / np.max(np.abs(xr)) < 1e-13


def test_vdiff_operator_is_conservative_and_consistent():
    """Rows of I - dt L sum to one (constants preserved) and dz_k c_k =
    dz_{k+1} a_{k+1} (the flux leaving level k enters level k+1), with zero
    flux through the ends; stretched dz and varying kappa."""
    nz = 12
    dz = 1.05 ** np.arange(nz)
    kl = 0.01 + 0.04 * np.linspace(0, 1, nz) ** 2
    a, b, c = oracle.vdiff_coeffs(nz, 0.1, dz, kl, 37.0)
    assert a[0] == 0 and c[-1] == 0
    assert np.all(a[1:] < 0) and np.all(c[:-1] < 0)
    assert np.max(np.abs(a + b + c - 1)) < 1e-15
    assert np.max(np.abs(dz[:-1] * c[:-1] - dz[1:] * a[1:])) < 1e-15


# ---------------------------------------------------------------- radiation

def test_p9_radiation_energy_budget():
    """The heating telescopes: sum_k H_k dz_k = S0 (1 - exp(-tau_total))."""
    rng = np.random.default_rng(9)
    nz = 58
    dz = 1.05 ** np.arange(nz)
    alpha = inputs.absorber(nz)
    for S0 in (1.0, 3.5):
        qs = rng.uniform(0, 0.02, nz)
        H = oracle.radiation(qs, alpha, dz, S0, 0.01)
        tau = np.sum(alpha * dz * qs / 0.01)
        assert abs(np.sum(H * dz) - S0 * (1 - math.exp(-tau))) < 1e-13


def test_radiation_beam_from_top():
    """Two absorbing layers k1 < k2: the upper one gets the full beam, the
    lower one the beam attenuated by the upper; clear layers get nothing."""
    nz, k1, k2 = 10, 2, 7
    dz = np.linspace(1, 2, nz)
    alpha = np.full(nz, 0.3)
    qs = np.zeros(nz); qs[k1] = 0.02; qs[k2] = 0.01
    S0, qref = 2.0, 0.01
    H = oracle.radiation(qs, alpha, dz, S0, qref)
    d1 = alpha[k1] * dz[k1] * qs[k1] / qref
    d2 = alpha[k2] * dz[k2] * qs[k2] / qref
    expect = np.zeros(nz)
    expect[k2] = S0 * (1 - math.exp(-d2)) / dz[k2]
    expect[k1] = S0 * math.exp(-d2) * (1 - math.exp(-d1)) / dz[k1]
    assert np.max(np.abs(H - expect)) < 1e-15


def test_p8_scan_matches_brute_force_sums():
    """Every level's optical depth from the top, summed afresh over the
    levels above it (O(nz^2)), gives the oracle's heating profile."""
    rng = np.random.default_rng(8)
    for nz in (1, 2, 17, 58):
        dz = 1.05 ** np.arange(nz)
        alpha = 0.01 * np.exp(-np.arange(nz) / 8.0)
        qs = rng.uniform(0.0, 0.02, nz)
        S0, qref = 1.0, 0.01
        dtau = [alpha[k] * dz[k] * qs[k] / qref for k in range(nz)]
        H = np.empty(nz)
        for k in range(nz):
            top = 0.0
            for kk in range(k + 1, nz):
                top += dtau[kk]
            H[k] = S0 * (math.exp(-top) - math.exp(-(top + dtau[k]))) / dz[k]
        got = oracle.radiation(qs, alpha, dz, S0, qref)
        assert np.max(np.abs(got - H)) <= 1e-15 * max(1.0, np.max(np.abs(H)))


def test_p10_optically_thin_limit():
    """As q -> 0 the heating tends to S0 dtau_k/dz_k = S0 alpha_k q_k/q_ref."""
    nz = 20
    dz = 1.05 ** np.arange(nz)
    alpha = inputs.absorber(nz)
    qs = np.linspace(1, 2, nz) * 1e-9
    H = oracle.radiation(qs, alpha, dz, 1.0, 0.01)
    thin = alpha * qs / 0.01
    assert np.max(np.abs(H / thin - 1)) < 1e-6


# ------------------------------------------------------------- full step

def test_step_energy_budget():
    """Full step with radiation: the dz-weighted heat content grows by exactly
    dt*S0*(1 - exp(-tau_total(q*))) per column (dynamics and the implicit
    solve conserve; the heating telescopes), summed over the grid."""
    c = _generated(17, 15, 10, S0=1.0, near_singular=True)
    e0 = oracle.weighted_sum(c, c.T)
    Tn, qn = oracle.step(c, c.T, c.q, c.U, c.V)
    tau = np.einsum("kji,k->ji", qn * (c.alpha * c.dz)[:, None, None] / c.q_ref, np.ones(c.nz))
    gain = c.h ** 2 * c.dt * c.S0 * np.sum(1 - np.exp(-tau))
    e1 = oracle.weighted_sum(c, Tn)
    assert abs((e1 - e0) - gain) / gain < 1e-9
    assert abs(gain) > 1e-3


def test_physics_columns_matches_step_composition():
    """physics_columns on the step's own T*, q* gives the step's T^{n+1}; the
    tendencies reproduce it as T* + dt (H + vdiff)."""
    c = _generated(9, 7, 12, S0=1.0, near_singular=True)
    Ts, qs = oracle.dynamics(c, c.T, c.q, c.U, c.V)
    Tn, qn = oracle.step(c, c.T, c.q, c.U, c.V)
    cols = lambda a: a.reshape(c.nz, -1).T.copy()
    Tout, tend = oracle.physics_columns(c.nz, c.dt, c.dz, c.kappa_lev,
                                        c.kappa_mult.reshape(-1), c.alpha, c.S0,
                                        c.q_ref, cols(Ts), cols(qs), with_tend=True)
    assert np.array_equal(Tout, cols(Tn))
    assert np.array_equal(cols(qs), cols(qn))
    recon = cols(Ts) + c.dt * (tend[:, 0] + tend[:, 1])
    assert np.max(np.abs(recon - Tout)) < 1e-12


def test_near_singular_columns_have_low_dominance():
    """The mixed-precision input recipe: about 5% of columns get kappa_mult in
    [1e4, 1e5]; their dominance ratio min_k |b|/(|a|+|c|) is below 1.1 and
    the others' is above it."""
    c = inputs.paper_grid_case(64, 48, 58, near_singular=True)
    km = c.kappa_mult.reshape(-1)
    frac = np.mean(km > 1)
    assert 0.03 < frac < 0.07
    ratios = []
    for s in (1.0, km[km > 1].min()):
        a, b, cc = oracle.vdiff_coeffs(c.nz, c.dt, c.dz, c.kappa_lev, s)
        ratios.append(np.min(np.abs(b) / (np.abs(a) + np.abs(cc))))
    assert ratios[0] > 1.1 and ratios[1] < 1.1


def test_step_columns_equals_full_step():
    """The sampled-column form of the step is the full step restricted to
    those columns (bitwise: same arithmetic, same order)."""
    c = _generated(13, 11, 9, S0=1.0, near_singular=True)
    Tn, qn = oracle.step(c, c.T, c.q, c.U, c.V)
    ci = np.array([0, 12, 5, 0, 12])
    cj = np.array([0, 10, 4, 10, 0])
    Ts, qs = oracle.step_columns(c, c.T, c.q, c.U, c.V, ci, cj)
    assert np.array_equal(Ts, Tn[:, cj, ci].T)
    assert np.array_equal(qs, qn[:, cj, ci].T)
