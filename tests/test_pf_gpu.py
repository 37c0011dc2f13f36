"""The paper's reduced weather application on the GPU (wx_pf_*) against its
FP64 oracle: every step on ragged and degenerate grids, the paper's 128^3 box
workload over 100 steps, and the status paths.

Tolerances: FP64 1e-12 max relative error per step (the update is a convex
combination of at most seven values plus an affine physics term, so each
step adds a few ulps); 1e-11 after 100 steps.  FP32: 1e-5 per step and 1e-4
relative L2 after 100 steps (inputs rounded once to FP32)."""
import numpy as np
import pytest

import oracle
from paper_1802_05839_gb300 import inputs, wx

pytestmark = pytest.mark.gpu


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def state(nx, ny, nz, seed=1):
    """The paper's box state plus seeded noise (so that every cell differs)."""
    E = inputs.paper_box_state(nx, ny, nz)
    return E + 10.0 * inputs.uniform(seed, 300, E.size).reshape(E.shape)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("shape", [(9, 7, 6), (1, 1, 2), (33, 5, 3), (64, 48, 20), (2, 40, 2)])
def test_every_step_matches_oracle(dtype, tol, shape):
    nx, ny, nz = shape
    p = oracle.pf_params(nx, ny, nz)
    E = state(nx, ny, nz)
    if dtype == "f32":
        E = E.astype(np.float32).astype(np.float64)
    app = wx.ReducedApp(nx, ny, nz, dtype)
    app.set_params()
    app.load(E)
    ref = E
    for _ in range(10):
        app.step(1)
        app.sync()
        got = app.read()
        ref = oracle.pf_step(p, ref)
        assert relmax(got, ref) <= tol
        if dtype == "f32":
            ref = got  # per-step error: restart the oracle from the GPU state
    app.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_paper_box_workload_100_steps(dtype):
    n = 128
    E = inputs.paper_box_state(n, n, n)
    app = wx.ReducedApp(n, n, n, dtype)
    app.set_params()
    app.load(E)
    app.step(100)
    app.sync()
    got = app.read()
    ref = oracle.pf_run(oracle.pf_params(n, n, n), 100, E)
    if dtype == "f64":
        assert relmax(got, ref) <= 1e-11
    else:
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4
    assert app.last_launches() == 100
    app.close()


def test_uniform_field_gains_exactly_the_radiation():
    app = wx.ReducedApp(20, 12, 8, "f64")
    app.set_params(d=0.125, radiation=0.25, transfer=0.0)
    app.load(np.full((8, 14, 22), 250.0))
    app.step(8)
    app.sync()
    assert np.array_equal(app.read(), np.full((8, 14, 22), 252.0))
    app.close()


def test_status_paths():
    app = wx.ReducedApp(8, 8, 4, "f64")
    with pytest.raises(wx.WxError) as e:
        app.step(1)                     # nothing loaded
    assert e.value.code == -7
    with pytest.raises(wx.WxError) as e:
        app.set_params(d=0.2)           # 1 - 6d < 0
    assert e.value.code == -4
    E = np.zeros((4, 10, 10))
    E[2, 5, 5] = np.nan
    app.set_params()
    app.load(E)
    app.step(1)
    with pytest.raises(wx.WxError) as e:
        app.sync()
    assert e.value.code == -5
    app.close()


@pytest.mark.parametrize("layout,block", [("kij", (32, 8)), ("ijk", (128, 1)), ("ijk", (32, 16)),
                                          ("kij", (64, 2))])
def test_storage_orders_and_block_shapes_match_oracle(layout, block):
    nx, ny, nz = 37, 23, 11
    p = oracle.pf_params(nx, ny, nz)
    E = state(nx, ny, nz, seed=5)
    app = wx.ReducedApp(nx, ny, nz, "f64")
    app.set_params()
    app.set_launch(layout, block)
    app.load(E)
    app.step(5)
    app.sync()
    assert relmax(app.read(), oracle.pf_run(p, 5, E)) <= 1e-12
    app.close()


def test_switching_storage_order_mid_run_is_bitwise_neutral():
    """The update is the same arithmetic in either order, so 3 IJK steps, a
    switch to KIJ and 3 more equal 6 IJK steps bit for bit."""
    nx, ny, nz = 30, 20, 9
    E = state(nx, ny, nz, seed=6)
    a = wx.ReducedApp(nx, ny, nz, "f64")
    a.set_params()
    a.load(E)
    a.step(6)
    a.sync()
    b = wx.ReducedApp(nx, ny, nz, "f64")
    b.set_params()
    b.load(E)
    b.step(3)
    b.set_launch("kij", (32, 8))
    b.step(3)
    b.sync()
    assert np.array_equal(a.read(), b.read())
    with pytest.raises(wx.WxError):
        b.set_launch("ijk", (33, 1))
    a.close()
    b.close()
