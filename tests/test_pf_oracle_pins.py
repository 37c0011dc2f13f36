"""Pins of the oracle of the paper's reduced weather application
(wxo_pf_step / wxo_pf_run): closed forms that each region of the listings'
update must meet -- the interior 7-point rule, the one-sided rule at the
bottom and top levels, the two-neighbour rule of the ghost rows and ghost
columns (corners last), uniform radiation and the two Newtonian heat
wells."""
import numpy as np
import pytest

import oracle
from paper_1802_05839_gb300 import inputs

NX, NY, NZ = 9, 7, 6


def zeros():
    return np.zeros((NZ, NY + 2, NX + 2))


def test_uniform_field_gains_exactly_the_radiation():
    """Every diffusion row sums to one (1 - 6d + 6d, 1 - 5d + 5d, 1 - 2d +
    2d), so a uniform field only gains n * radiation."""
    p = oracle.pf_params(NX, NY, NZ, d=0.125, radiation=0.25, transfer=0.0)
    E = np.full((NZ, NY + 2, NX + 2), 250.0)
    out = oracle.pf_run(p, 8, E)
    assert np.array_equal(out, np.full_like(E, 252.0))


def test_heat_wells_relax_geometrically():
    """Without diffusion and radiation the bottom level relaxes to T_surf and
    the top level to T_pbl as T_w + (c - T_w)(1 - transfer)^n; the levels
    between are untouched."""
    tau, n, c = 0.01, 25, 250.0
    p = oracle.pf_params(NX, NY, NZ, d=0.0, radiation=0.0, transfer=tau)
    out = oracle.pf_run(p, n, np.full((NZ, NY + 2, NX + 2), c))
    g = (1 - tau) ** n
    np.testing.assert_allclose(out[0], 330.0 + (c - 330.0) * g, rtol=1e-14)
    np.testing.assert_allclose(out[-1], 200.0 + (c - 200.0) * g, rtol=1e-14)
    assert np.all(out[1:-1] == c)


def test_radiation_comes_before_the_heat_wells():
    """One step, no diffusion: level 0 = (c + r) - tau (c + r - T_surf)."""
    c, r, tau = 100.0, 0.1, 0.01
    p = oracle.pf_params(NX, NY, NZ, d=0.0, radiation=r, transfer=tau)
    out = oracle.pf_step(p, np.full((NZ, NY + 2, NX + 2), c))
    assert np.allclose(out[0], (c + r) - tau * (c + r - 330.0), rtol=0, atol=1e-13)
    assert np.allclose(out[2], c + r, rtol=0, atol=1e-13)


@pytest.mark.parametrize("k", [2, 0, NZ - 1])
def test_interior_delta_response(k):
    """A unit value at an interior cell away from the ghost ring spreads to
    its six (or, at the bottom and top, five) neighbours with weight d and
    keeps 1 - 6d (1 - 5d)."""
    d = 0.1
    p = oracle.pf_params(NX, NY, NZ, d=d, radiation=0.0, transfer=0.0)
    E = zeros()
    i, j = 4, 3
    E[k, j, i] = 1.0
    out = oracle.pf_step(p, E)
    want = zeros()
    nb = [(k, j, i - 1), (k, j, i + 1), (k, j - 1, i), (k, j + 1, i)]
    if k > 0:
        nb.append((k - 1, j, i))
    if k < NZ - 1:
        nb.append((k + 1, j, i))
    want[k, j, i] = 1.0 - len(nb) * d
    for c in nb:
        want[c] = d
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-15)


def test_ghost_ring_is_state_with_its_own_rule():
    """A unit value in the ghost column i = 0 (j interior): it keeps 1 - 2d,
    the far ghost column i = nx+1 and the interior cell i = 1 each read it
    with weight d; nothing else sees it (ghosts have no vertical or j
    neighbours)."""
    d = 0.1
    p = oracle.pf_params(NX, NY, NZ, d=d, radiation=0.0, transfer=0.0)
    E = zeros()
    k, j = 3, 2
    E[k, j, 0] = 1.0
    out = oracle.pf_step(p, E)
    want = zeros()
    want[k, j, 0] = 1 - 2 * d
    want[k, j, NX + 1] = d
    want[k, j, 1] = d
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-15)


def test_ghost_row_rule():
    """A unit value in the far ghost row j = ny+1 (i interior): it keeps
    1 - 2d, the near ghost row j = 0 (which reads rows 1 and ny+1) and the
    interior row j = ny (whose north neighbour it is) each read it with
    weight d; nothing else sees it."""
    d = 0.1
    p = oracle.pf_params(NX, NY, NZ, d=d, radiation=0.0, transfer=0.0)
    E = zeros()
    k, i = 3, 4
    E[k, NY + 1, i] = 1.0
    out = oracle.pf_step(p, E)
    want = zeros()
    want[k, NY + 1, i] = 1 - 2 * d
    want[k, 0, i] = d
    want[k, NY, i] = d
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-15)


def test_interior_edge_feeds_only_its_own_ghost_column():
    """A unit value at i = 1: the ghost column i = 0 reads it (d), the far
    ghost column i = nx+1 does not (it reads i = nx and i = 0)."""
    d = 0.1
    p = oracle.pf_params(NX, NY, NZ, d=d, radiation=0.0, transfer=0.0)
    E = zeros()
    k, j = 2, 3
    E[k, j, 1] = 1.0
    out = oracle.pf_step(p, E)
    assert out[k, j, 0] == pytest.approx(d, abs=1e-15)
    assert out[k, j, NX + 1] == 0.0
    assert out[k, j, 2] == pytest.approx(d, abs=1e-15)
    assert out[k, j, 1] == pytest.approx(1 - 6 * d, abs=1e-15)


def test_corner_columns_take_the_ghost_column_rule():
    """The corners are written by the ghost-row loop and then by the
    ghost-column loop: a unit value at (i, j) = (0, 0) keeps 1 - 2d, feeds
    (nx+1, 0) with d, and the ghost-row corner (0, ny+1), which the row rule
    would feed, ends at 0 because the column rule overwrote it."""
    d = 0.1
    p = oracle.pf_params(NX, NY, NZ, d=d, radiation=0.0, transfer=0.0)
    E = zeros()
    k = 1
    E[k, 0, 0] = 1.0
    out = oracle.pf_step(p, E)
    want = zeros()
    want[k, 0, 0] = 1 - 2 * d
    want[k, 0, NX + 1] = d
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-15)


def test_box_initial_state():
    E = inputs.paper_box_state(128, 128, 128)
    assert E.shape == (128, 130, 130)
    assert E.sum() == 300.0 * 64 ** 3
    assert E[32, 33, 33] == 300.0 and E[31, 33, 33] == 0.0 and E[32, 33, 97] == 0.0
    assert np.all(E[:, 0, :] == 0) and np.all(E[:, :, 0] == 0)
