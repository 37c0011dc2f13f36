"""Pins of the oracle's three-stage Runge-Kutta dynamics (wxo_step_rk3,
Wicker and Skamarock 2002) to closed forms: applied to an eigenmode of the
linear dynamics operator with per-step Euler factor 1 + z, the three stages
multiply the mode by R(z) = 1 + z + z^2/2 + z^3/6 (the scheme's stability
polynomial); plus conservation and the fixed point."""
import math

import numpy as np
import pytest

import oracle
from paper_1802_05839_gb300 import inputs

from test_oracle_pins import bare_case, _generated


def R(z):
    return 1 + z + z * z / 2 + z ** 3 / 6


@pytest.mark.parametrize("m,n", [(1, 0), (2, 3), (5, 1)])
def test_fourier_mode_decays_by_the_rk3_polynomial(m, n):
    nx, ny, nz, N = 24, 20, 3, 5
    c = bare_case(nx, ny, nz, kappa_h=0.9, h=1.3)
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    phase = 2 * np.pi * (m * i / nx + n * j / ny)
    T0 = np.broadcast_to(5.0 + 2.0 * np.cos(phase), (nz, ny, nx)).copy()
    T, _ = oracle.run_rk3(c, N, T0, T0.copy(), c.U, c.V)
    z = -4 * c.kappa_h * c.dt / c.h ** 2 * (math.sin(math.pi * m / nx) ** 2 + math.sin(math.pi * n / ny) ** 2)
    expect = 5.0 + 2.0 * R(z) ** N * np.cos(phase)
    assert np.max(np.abs(T - expect[None])) < 1e-13 * 7
    # and it differs from forward Euler's (1 + z)^N by more than rounding
    assert abs(R(z) ** N - (1 + z) ** N) > 1e-6


@pytest.mark.parametrize("C", [0.3, 0.9, 1.2])
def test_upwind_mode_takes_the_rk3_polynomial_of_the_upwind_symbol(C):
    """A mode e^{i theta i} under uniform wind: per step R(-C (1 - e^{-i theta})),
    also at Courant 1.2 where forward Euler's upwind scheme is unstable."""
    nx, ny, nz, N, m = 16, 2, 1, 6, 3
    c = bare_case(nx, ny, nz, dt=0.1, h=1.0, kappa_h=0.0, advection=True)
    c.U[:] = C * c.h / c.dt
    theta = 2 * np.pi * m / nx
    i = np.arange(nx)
    T0 = np.broadcast_to(1.0 + np.cos(theta * i), (nz, ny, nx)).copy()
    T, _ = oracle.run_rk3(c, N, T0, T0.copy(), c.U, c.V)
    g = R(-C * (1 - np.exp(-1j * theta)))
    expect = 1.0 + np.real(g ** N * np.exp(1j * theta * i))
    assert np.max(np.abs(T[0, 0] - expect)) < 1e-13


def test_mass_is_conserved_and_a_constant_is_fixed():
    c = _generated(23, 17, 9, near_singular=True)
    T, q = oracle.run_rk3(c, 6, c.T, c.q, c.U, c.V)
    wq0 = oracle.weighted_sum(c, c.q)
    assert abs(oracle.weighted_sum(c, q) - wq0) <= 1e-12 * abs(wq0)
    wT0 = oracle.weighted_sum(c, c.T)   # S0 = 0: the physics conserves T too
    assert abs(oracle.weighted_sum(c, T) - wT0) <= 1e-12 * abs(wT0)
    k = np.full_like(c.T, 287.5)
    Tk, qk = oracle.run_rk3(c, 3, k, k.copy(), c.U, c.V)
    # up to rounding, amplified in T by the near-singular columns' implicit solve
    assert np.max(np.abs(Tk - 287.5)) < 1e-13 * 287.5 and np.max(np.abs(qk - 287.5)) < 1e-13 * 287.5


def test_physics_follows_the_third_stage():
    """step_rk3 = column physics applied to the third stage's state: with the
    physics on, it equals physics_columns of the RK3 dynamics alone."""
    c = _generated(11, 9, 12, S0=1.0, near_singular=True)
    Tn, qn = oracle.step_rk3(c, c.T, c.q, c.U, c.V)
    c.physics = False
    T3, q3 = oracle.step_rk3(c, c.T, c.q, c.U, c.V)
    assert np.array_equal(qn, q3)
    ncol = c.nx * c.ny
    cols = lambda a: np.ascontiguousarray(a.reshape(c.nz, ncol).T)
    Tp = oracle.physics_columns(c.nz, c.dt, c.dz, c.kappa_lev, c.kappa_mult.reshape(ncol), c.alpha,
                                c.S0, c.q_ref, cols(T3), cols(q3))
    assert np.max(np.abs(cols(Tn) - Tp)) == 0.0
