"""The FP32 increment checks (tests/increments.py) are sharp enough to catch
a wrong FP32 physics path that the per-field bound (max relative error
1e-5) lets through.  Run on the CPU: the "GPU result" is the oracle's step
rounded once to FP32 (what a perfect FP32 kernel would store), and each
planted mistake is made in that stand-in on the host, never in a kernel."""
import numpy as np
import pytest

import oracle
from increments import assert_increments, increment_report, strong_physics
from paper_1802_05839_gb300 import inputs


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def maxrel(g, o):
    return float(np.max(np.abs(g - o)) / np.max(np.abs(o)))


@pytest.fixture(scope="module")
def plain():
    c = inputs.round_to_f32(inputs.paper_grid_case(40, 30, 58, seed=4, near_singular=True))
    To, _ = oracle.step(c, c.T, c.q, c.U, c.V)
    Ts, _ = oracle.dynamics(c, c.T, c.q, c.U, c.V)
    return c, To, Ts


@pytest.fixture(scope="module")
def strong():
    c = inputs.round_to_f32(strong_physics(inputs.paper_grid_case(40, 30, 58, seed=4)))
    To, _ = oracle.step(c, c.T, c.q, c.U, c.V)
    Ts, _ = oracle.dynamics(c, c.T, c.q, c.U, c.V)
    return c, To, Ts


def test_a_correctly_rounded_result_passes(plain, strong):
    for c, To, Ts in (plain, strong):
        r = assert_increments(c.T, Ts, f32(To), To, what="rounded oracle")
        assert r["err_ulp"] <= 0.5


def _listed(c):
    return np.broadcast_to((c.kappa_mult != 1.0)[None], c.T.shape)


def test_weak_vertical_diffusion_on_ordinary_columns(plain):
    """A physics path that applies 70% of the implicit vertical diffusion
    (as a wrong FP32 elimination would) on the kappa_mult = 1 columns: under
    the old per-field bound, caught by the increment check."""
    c, To, Ts = plain
    ok = ~_listed(c)
    bad = np.where(ok, Ts + 0.7 * (To - Ts), To)
    Tg = f32(bad)
    assert maxrel(Tg, To) <= 1e-5                      # the field bound lets it through
    with pytest.raises(AssertionError):
        assert_increments(c.T, Ts, Tg, To, what="planted")


def test_wrong_side_solve_on_listed_columns(plain):
    """The side solve of the near-singular columns off by 0.1% of their
    physics increment: the increment check over the listed columns fails."""
    c, To, Ts = plain
    lst = _listed(c)
    Tg = f32(np.where(lst, Ts + 0.999 * (To - Ts), To))
    with pytest.raises(AssertionError):
        assert_increments(c.T, Ts, Tg, To, mask=lst, what="planted")


def test_dropped_heating_is_caught(plain):
    """A fallback that forgets the radiative heating (at the configuration's
    S0 = 1 it is at most ~2e-3 K per step): invisible to the field bound,
    caught by the increment check."""
    c, To, Ts = plain
    dark = c.copy()
    dark.S0 = 0.0
    Tnh, _ = oracle.step(dark, c.T, c.q, c.U, c.V)  # the same step without the heating
    assert np.max(np.abs(To - Tnh)) > 16 * increment_report(c.T, Ts, To, To)["ulp"]
    Tg = f32(Tnh)
    assert maxrel(Tg, To) <= 1e-5
    with pytest.raises(AssertionError):
        assert_increments(c.T, Ts, Tg, To, what="planted")


def test_physics_applied_to_the_old_state_is_caught(strong):
    """Physics on T^n instead of T* (the dynamics increment lost on the way
    into the column solve): caught through the step increment as well."""
    c, To, Ts = strong
    Tg = f32(To - (Ts - c.T))
    with pytest.raises(AssertionError):
        assert_increments(c.T, Ts, Tg, To, what="planted")


def test_a_bar_that_cannot_resolve_the_physics_is_refused(plain):
    """With no physics (T^{n+1} = T*) the bar would be vacuous: refused."""
    c, To, Ts = plain
    with pytest.raises(AssertionError, match="cannot resolve"):
        assert_increments(c.T, Ts, f32(Ts), Ts + 1e-9, what="no physics")
