"""The residual-checked surrogate step (wx_step with WX_SURROGATE) against the
FP64 oracles: the plain oracle's step where every column falls back, the MLP
oracle's prediction where every column is accepted, and bitwise agreement of
a two-step run with a run restarted from the saved state in between (the
surrogate path keeps the periodic ghost copies consistent)."""
import numpy as np
import pytest

import oracle
from increments import assert_increments, strong_physics
from oracle import mlp as omlp
from paper_1802_05839_gb300 import inputs, wx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NZ = 58


def case(nx=70, ny=50, seed=3, near_singular=False):
    return inputs.round_to_f32(inputs.paper_grid_case(nx, ny, NZ, seed=seed, near_singular=near_singular))


def random_net(c, seed=11, std_out=1.0):
    """A random network whose input normalisation fits the case's columns and
    whose outputs are O(std_out) in physical units."""
    m = wx.MLP(max_batch=512)
    Ws, bs = inputs.mlp_init(seed)
    m.set_weights(Ws, bs)
    n = c.nx * c.ny
    km = c.kappa_mult.reshape(n) if c.kappa_mult is not None else None
    F = omlp.raw_features(c.T.reshape(NZ, n).T, c.q.reshape(NZ, n).T, km, c.kappa_lev, c.alpha, c.dz)
    mean, sd = omlp.fit_norm(F)
    m.set_norm(mean, sd, np.zeros(116), np.full(116, std_out))
    return m


def ctx_for(c, net, tol, flags=wx.WX_ADVECTION | wx.WX_PHYSICS | wx.WX_SURROGATE):
    ctx = wx.Context(c.nx, c.ny, NZ, "f32")
    ctx.set_params(c, flags=flags)
    ctx.load_fields(c.T, c.q, c.U, c.V)
    if net is not None:
        ctx.set_surrogate(net, tol)
    return ctx


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("near_singular", [False, True])
def test_every_column_falling_back_gives_the_exact_step(near_singular):
    c = case(near_singular=near_singular)
    net = random_net(c)
    ctx = ctx_for(c, net, tol=0.0)
    ctx.step(3)
    ctx.sync()
    assert ctx.surrogate_fallbacks() == c.nx * c.ny
    T, q = ctx.read_fields()
    To, qo = oracle.run(c, 3, c.T, c.q, c.U, c.V)
    assert relmax(T, To) <= 1e-5 and relmax(q, qo) <= 1e-5
    ctx.close()
    # step by step from the GPU's own state: the exact path's increments,
    # on every column and on the near-singular ones alone
    ctx = ctx_for(c, net, tol=0.0)
    listed = None if c.kappa_mult is None else np.broadcast_to((c.kappa_mult != 1.0)[None], c.T.shape)
    Tp, qp = c.T, c.q
    for s in range(2):
        ctx.step(1)
        ctx.sync()
        Tg, qg = ctx.read_fields()
        To, _ = oracle.step(c, Tp, qp, c.U, c.V)
        Ts, _ = oracle.dynamics(c, Tp, qp, c.U, c.V)
        assert_increments(Tp, Ts, Tg, To, what=f"fallback step {s}")
        if listed is not None:
            assert_increments(Tp, Ts, Tg, To, mask=listed, what=f"fallback step {s}, listed")
        Tp, qp = Tg, qg
    ctx.close()
    net.close()


@pytest.mark.parametrize("near_singular", [False, True])
def test_fallback_strong_physics_increments(near_singular):
    """The exact path of the surrogate step (every column falls back) on a
    case with a physics increment of ~1 K: increments within 8 ulp of the
    oracle's, which resolves the FP32 solve and heating to a few 1e-3."""
    c = inputs.round_to_f32(strong_physics(inputs.paper_grid_case(70, 50, NZ, seed=3,
                                                                  near_singular=near_singular)))
    net = random_net(c)
    ctx = ctx_for(c, net, tol=0.0)
    ctx.step(1)
    ctx.sync()
    assert ctx.surrogate_fallbacks() == c.nx * c.ny
    Tg, qg = ctx.read_fields()
    To, qo = oracle.step(c, c.T, c.q, c.U, c.V)
    Ts, _ = oracle.dynamics(c, c.T, c.q, c.U, c.V)
    assert_increments(c.T, Ts, Tg, To, what="fallback", resolve=0.01)
    if near_singular:
        listed = np.broadcast_to((c.kappa_mult != 1.0)[None], c.T.shape)
        assert_increments(c.T, Ts, Tg, To, mask=listed, what="fallback, listed", resolve=0.01)
    assert relmax(qg, qo) <= 1e-5
    ctx.close()
    net.close()


def test_policy_steps_exactly_while_the_network_declines():
    """Acceptance policy (min_accept 0.5): every column falls back (tol 0),
    so after the two steps the decision lags, steps run the fused exact
    step (1 launch), plus a probe of the network on 8 rows every 4 steps
    (6 more launches); every step stays within the FP32 bars of the
    oracle's step from the same state."""
    c = case(seed=5)
    net = random_net(c)
    ctx = ctx_for(c, net, tol=0.0)
    ctx.set_surrogate_policy(0.5, probe_every=4, probe_rows=8)
    launches = []
    Tp, qp = c.T, c.q
    for s in range(9):
        ctx.step(1)
        ctx.sync()
        launches.append(ctx.last_launches())
        assert ctx.surrogate_fallbacks() == c.nx * c.ny
        Tg, qg = ctx.read_fields()
        To, qo = oracle.step(c, Tp, qp, c.U, c.V)
        assert relmax(Tg, To) <= 1e-5 and relmax(qg, qo) <= 1e-5
        Ts, _ = oracle.dynamics(c, Tp, qp, c.U, c.V)
        assert_increments(Tp, Ts, Tg, To, what=f"policy step {s}")
        Tp, qp = Tg, qg
    # steps 0, 1: network (7 launches); 2 onwards exact, probes at 6 and 10, ...
    assert launches == [7, 7, 1, 1, 1, 1, 7, 1, 1], launches
    ctx.close()
    net.close()


def _policy_run(c, net):
    ctx = ctx_for(c, net, tol=1e30)
    ctx.set_surrogate_policy(1.0, probe_every=1, probe_rows=8)
    launches = []
    for _ in range(6):
        ctx.step(1)
        launches.append(ctx.last_launches())
    ctx.sync()
    out = ctx.read_fields()
    ctx.close()
    return launches, out


def test_policy_probe_returns_to_the_network():
    """A band of rows with q = 0 fails the heating residual at any
    tolerance, so a whole-grid step accepts fewer than all columns and the
    policy (min_accept 1.0) turns to exact steps; the probe covers rows
    0..7, where every column is accepted, and turns it back.  The same
    sequence of steps takes the same decisions and gives the same state."""
    c = case(seed=6)
    c.q[:, c.ny // 2 - 6:c.ny // 2 + 6, :] = 0.0
    net = random_net(c, std_out=0.1)
    la, (Ta, qa) = _policy_run(c, net)
    lb, (Tb, qb) = _policy_run(c, net)
    # 0, 1 network; 2 exact (decided from step 0); 3, 4 exact + probe;
    # 5 network again (decided from the probe of step 3)
    assert la == [7, 7, 1, 7, 7, 7], la
    assert la == lb and np.array_equal(Ta, Tb) and np.array_equal(qa, qb)
    net.close()


def test_policy_arguments():
    c = case(nx=20, ny=16)
    net = random_net(c)
    ctx = ctx_for(c, net, tol=2e-2)
    for bad in ((-0.1, 8, 16), (1.5, 8, 16), (0.5, 0, 16), (0.5, 8, 0)):
        with pytest.raises(wx.WxError) as e:
            ctx.set_surrogate_policy(*bad)
        assert e.value.code == -1
    ctx.set_surrogate_policy(0.0)  # off: the network runs on every step
    ctx.step(2)
    ctx.sync()
    assert ctx.last_launches() == 14
    ctx.close()
    net.close()


def test_accepted_predictions_match_the_mlp_oracle():
    c = case(seed=4)
    net = random_net(c, seed=12)
    ctx = ctx_for(c, net, tol=1e30)
    ctx.step(1)
    ctx.sync()
    assert ctx.surrogate_fallbacks() == 0
    T, q = ctx.read_fields()
    # oracle: dynamics, then the BF16-emulating forward on the same features
    Ts, qs = oracle.dynamics(c, c.T, c.q, c.U, c.V)
    n = c.nx * c.ny
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    Tc, qc = Ts.reshape(NZ, n).T, qs.reshape(NZ, n).T
    F = omlp.raw_features(f32(Tc), f32(qc), None, f32(c.kappa_lev), 1.0,
                          f32(np.asarray(c.alpha) * np.asarray(c.dz)))
    mi, si, mo, so = net.get_norm()
    X = ((F.astype(np.float32) - mi) * (np.float32(1) / si)).astype(np.float64)  # FP32; split by forward
    Ws, bs = net.get_weights()
    Y, _ = omlp.forward([W.astype(np.float64) for W in Ws], [b.astype(np.float64) for b in bs], X)
    y = Y * so + mo
    inc = c.dt * (y[:, :NZ] + y[:, NZ:])          # dt (H + vdiff rate)
    To = (Tc + inc).T.reshape(NZ, c.ny, c.nx)
    dT, dTo = T - Ts, To - Ts
    assert np.linalg.norm(dT - dTo) / np.linalg.norm(dTo) <= 5e-3
    assert relmax(q, qs) <= 1e-5
    ctx.close()
    net.close()


@pytest.mark.parametrize("tol", [0.0, 1e30])
def test_two_steps_equal_a_restart_in_between_bitwise(tol):
    c = case(nx=45, ny=33, seed=6)
    net = random_net(c, seed=13, std_out=0.1)
    a = ctx_for(c, net, tol)
    a.step(2)
    a.sync()
    Ta, qa = a.read_fields()
    b = ctx_for(c, net, tol)
    b.step(1)
    b.sync()
    T1, q1 = b.read_fields()
    b.load_fields(T1, q1, c.U, c.V)   # ghost ring rebuilt from the interior
    b.step(1)
    b.sync()
    Tb, qb = b.read_fields()
    assert np.array_equal(Ta, Tb) and np.array_equal(qa, qb)
    a.close()
    b.close()
    net.close()


def test_surrogate_configuration_errors():
    c = case(nx=20, ny=16)
    net = random_net(c)
    ctx = wx.Context(20, 16, NZ, "f32")
    with pytest.raises(wx.WxError) as e:
        ctx.set_params(c, flags=wx.WX_PHYSICS | wx.WX_SURROGATE | wx.WX_SUMS)
    assert e.value.code == -8
    ctx.set_params(c, flags=wx.WX_PHYSICS | wx.WX_SURROGATE)
    ctx.load_fields(c.T, c.q, c.U, c.V)
    with pytest.raises(wx.WxError) as e:
        ctx.step(1)                      # no network attached
    assert e.value.code == -7
    ctx.set_surrogate(net, 2e-2)
    ctx.step(1)
    ctx.sync()
    ctx.set_surrogate(None)
    with pytest.raises(wx.WxError) as e:
        ctx.step(1)
    assert e.value.code == -7
    ctx.close()
    d = wx.Context(20, 16, NZ, "f64")
    with pytest.raises(wx.WxError) as e:
        d.set_surrogate(net, 2e-2)
    assert e.value.code == -8
    d.close()
    s = wx.Context(20, 16, 30, "f32")
    with pytest.raises(wx.WxError) as e:
        s.set_surrogate(net, 2e-2)
    assert e.value.code == -8
    s.close()
    net.close()
