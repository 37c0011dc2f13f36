"""Training the column-physics surrogate with the library's own kernels and
what the trained network gains.

Training data: 2M columns of eight seeded paper-grid-generator states that
share the served model configuration, with FP64 tendencies; validation on
a held-out state.  The target is a relative L2 tendency error of at most
2e-2 in physical units (heating and vertical-diffusion rate together); the
gain is measured against the two trivial predictors (the training mean and
the untrained network).  Columns outside the training distribution
(near-singular kappa_mult) must be caught by the residual check and
recomputed exactly, so the surrogate step stays within the FP32 step
tolerance of the FP64 oracle."""
import numpy as np
import pytest

import oracle
from increments import assert_increments
from paper_1802_05839_gb300 import inputs, surrogate as S, wx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def trained():
    Ts, qs, km, tend = S.dataset(range(1, 9), 512, 512)
    m = wx.MLP(4096)
    Ws, bs = inputs.mlp_init(2024)
    m.set_weights(Ws, bs)
    S.set_levels_from_case(m, inputs.paper_grid_case(8, 8, 58, seed=1, config_seed=S.CONFIG_SEED))
    m.fit_norm(Ts, qs, km, tend)
    X, Yt = S.rows(m, Ts, qs, km, tend)
    val = S.dataset([101], 256, 256)
    before = S.tendency_error(m, *val)
    hist = S.train(m, X, Yt, Ts.shape[0], epochs=32, batch=4096, lr0=2e-3, seed=0)
    del X, Yt
    yield m, hist, before, val, (Ts, qs, km, tend)
    m.close()


def test_training_reaches_the_tendency_target_and_gains(trained):
    m, hist, before, val, _ = trained
    after = S.tendency_error(m, *val)
    _, _, mo, _ = m.get_norm()
    Y = val[3].reshape(val[3].shape[0], -1).double()
    mean_err = float((Y - torch.from_numpy(mo).cuda().double()).norm() / Y.norm())
    print(f"val error: untrained {before[0]:.3e}, training-mean {mean_err:.3e}, trained {after} ; "
          f"loss {hist[0]:.3e} -> {hist[-1]:.3e}")
    assert hist[-1] < hist[0] / 20
    assert after[0] <= 2e-2 and after[1] <= 2e-2
    assert after[0] <= 0.1 * mean_err and after[0] <= 0.1 * before[0]


def test_surrogate_step_falls_back_outside_the_training_distribution(trained):
    m = trained[0]
    c = inputs.round_to_f32(inputs.paper_grid_case(96, 80, 58, seed=103, near_singular=True,
                                                   config_seed=S.CONFIG_SEED))
    n_singular = int(np.sum(c.kappa_mult != 1.0))
    ctx = wx.Context(c.nx, c.ny, 58, "f32")
    ctx.set_params(c, flags=wx.WX_ADVECTION | wx.WX_PHYSICS | wx.WX_SURROGATE)
    ctx.load_fields(c.T, c.q, c.U, c.V)
    ctx.set_surrogate(m, 2e-2)
    listed = np.broadcast_to((c.kappa_mult != 1.0)[None], c.T.shape)
    Tp, qp = c.T, c.q
    for s in range(2):
        ctx.step(1)
        ctx.sync()
        assert ctx.surrogate_fallbacks() >= n_singular
        Tg, qg = ctx.read_fields()
        # the near-singular columns take the exact path: their increments
        # within 8 ulp of the oracle's step from the same state
        To, _ = oracle.step(c, Tp, qp, c.U, c.V)
        Ts, _ = oracle.dynamics(c, Tp, qp, c.U, c.V)
        assert_increments(Tp, Ts, Tg, To, mask=listed, what=f"step {s}, near-singular columns")
        Tp, qp = Tg, qg
    T, q = ctx.read_fields()
    To, qo = oracle.run(c, 2, c.T, c.q, c.U, c.V)
    assert np.max(np.abs(T - To)) / np.max(np.abs(To)) <= 1e-5
    assert np.max(np.abs(q - qo)) / np.max(np.abs(qo)) <= 1e-5
    ctx.close()
