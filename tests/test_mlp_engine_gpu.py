"""The MLP engine (include/wx.h, wx_mlp_*) against the FP64 MLP oracle:
forward on BF16 operands, gradients of every layer, Adam, feature and
target preparation, and the normalisation fit.

Tolerances: the forward rounds weights and hidden activations to BF16 and
takes inputs as two-term BF16 expansions on both sides, and differs only in
FP32 against FP64 accumulation (relative L2 1e-3).  The backward keeps its
incoming gradient, the saved pre-activation and its outgoing gradient in
BF16: three roundings of at most 2^-9 relative per layer, compounded over
four layers, bound the worst case near 2.3e-2 (the first layer's weight
gradient also takes the leading term of the inputs alone, 2^-9 more); the
test asks 2e-2 in relative L2 per layer and a cosine above 0.999."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1802_05839_gb300 import inputs, wx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def weights(seed):
    Ws, bs = inputs.mlp_init(seed)
    bs = [inputs.normal(seed, 70 + l, len(b)) * 0.05 for l, b in enumerate(bs)]
    # the device keeps FP32 masters: the oracle starts from the same values
    return [W.astype(np.float32).astype(np.float64) for W in Ws], \
           [b.astype(np.float32).astype(np.float64) for b in bs]


def device_rows(X, width):
    M = X.shape[0]
    out = torch.zeros(M, width, dtype=torch.float32)
    out[:, :X.shape[1]] = torch.from_numpy(X)
    return out


def two_term_rows(X):
    """[M][512] BF16 rows [hi | lo] of FP32(X) [M][232], as the device builds
    them (round-to-nearest-even conversions)."""
    x = torch.from_numpy(np.asarray(X, np.float32))
    hi = x.to(torch.bfloat16)
    lo = (x - hi.float()).to(torch.bfloat16)
    out = torch.zeros(x.shape[0], 512, dtype=torch.bfloat16)
    out[:, :232] = hi
    out[:, 256:488] = lo
    return out.cuda()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def net():
    m = wx.MLP(max_batch=512)
    yield m
    m.close()


def test_forward_matches_oracle(net):
    Ws, bs = weights(11)
    net.set_weights(Ws, bs)
    M = 384
    X = inputs.normal(12, 1, M * 232).reshape(M, 232)
    Xd = two_term_rows(X)
    Y = torch.empty(M, 128, dtype=torch.float32, device="cuda")
    net.forward(Xd, Y)
    Yo, _ = omlp.forward(Ws, bs, X, bf16_path=True)
    Yg = Y[:, :116].cpu().numpy().astype(np.float64)
    assert rel_l2(Yg, Yo) <= 1e-3
    assert np.all(Y[:, 116:].cpu().numpy() == 0.0)  # zero padding rows of W4, b4


def test_forward_in_chunks_beyond_max_batch(net):
    Ws, bs = weights(13)
    net.set_weights(Ws, bs)
    M = 1280  # 2.5 x max_batch
    X = inputs.normal(14, 1, M * 232).reshape(M, 232)
    Xd = two_term_rows(X)
    Y = torch.empty(M, 128, dtype=torch.float32, device="cuda")
    net.forward(Xd, Y)
    Y2 = torch.empty(256, 128, dtype=torch.float32, device="cuda")
    net.forward(Xd[1024:].contiguous(), Y2)
    torch.cuda.synchronize()
    assert torch.equal(Y[1024:], Y2)
    Yo, _ = omlp.forward(Ws, bs, X, bf16_path=True)
    assert rel_l2(Y[:, :116].cpu().numpy().astype(np.float64), Yo) <= 1e-3


def test_gradients_match_oracle(net):
    Ws, bs = weights(21)
    net.set_weights(Ws, bs)
    M = 512
    X = inputs.normal(22, 1, M * 232).reshape(M, 232)
    Yt = inputs.normal(22, 2, M * 116).reshape(M, 116)
    Xd = two_term_rows(X)
    Ytd = device_rows(Yt.astype(np.float32), 128).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.gradients(Xd, Ytd, loss=loss)
    net.status()
    dWg, dbg = net.get_grads()
    # oracle: FP64 backward through the BF16 forward, targets as the device holds them
    Lo, dWo, dbo = omlp.loss_and_grads(Ws, bs, X, Yt.astype(np.float32).astype(np.float64))
    assert abs(loss.item() - Lo) <= 1e-3 * Lo
    for l in range(4):
        for g, o in ((dWg[l], dWo[l]), (dbg[l], dbo[l])):
            g = g.astype(np.float64)
            assert rel_l2(g, o) <= 2e-2, (l, rel_l2(g, o))
            cos = float(np.dot(g.ravel(), o.ravel()) / (np.linalg.norm(g) * np.linalg.norm(o)))
            assert cos >= 0.999, (l, cos)


def test_adam_steps_match_closed_form(net):
    Ws, bs = weights(31)
    net.set_weights(Ws, bs)
    M = 256
    X = inputs.normal(32, 1, M * 232).reshape(M, 232)
    Yt = inputs.normal(32, 2, M * 116).reshape(M, 116)
    Xd = two_term_rows(X)
    Ytd = device_rows(Yt.astype(np.float32), 128).cuda()
    p = [W.copy() for W in Ws] + [b.copy() for b in bs]
    mom = [np.zeros_like(a) for a in p]
    vel = [np.zeros_like(a) for a in p]
    lrs = [1e-3, 7e-4]
    for t, lr in enumerate(lrs, start=1):
        net.gradients(Xd, Ytd)          # the gradients the step is about to use
        dW, db = net.get_grads()
        g = [a.astype(np.float64) for a in dW + db]
        net.train_step(Xd, Ytd, lr)
        for i in range(8):
            p[i], mom[i], vel[i] = omlp.adam_step(p[i], g[i], mom[i], vel[i], t, lr)
        Wg, bg = net.get_weights()
        for i, a in enumerate(Wg + bg):
            np.testing.assert_allclose(a.astype(np.float64), p[i], rtol=0, atol=2e-6)


def columns(seed, ncol_side=16, near_singular=True):
    c = inputs.paper_grid_case(ncol_side, ncol_side, 58, seed=seed, near_singular=near_singular)
    c = inputs.round_to_f32(c)
    n = c.nx * c.ny
    Ts = np.ascontiguousarray(c.T.reshape(58, n).T)
    qs = np.ascontiguousarray(c.q.reshape(58, n).T)
    km = c.kappa_mult.reshape(n) if c.kappa_mult is not None else np.ones(n)
    _, tend = oracle.physics_columns(58, c.dt, c.dz, c.kappa_lev, km, c.alpha, c.S0, c.q_ref,
                                     Ts, qs, with_tend=True)
    return c, Ts, qs, km, tend


def test_fit_norm_and_prepare_match_oracle(net):
    c, Ts, qs, km, tend = columns(5)
    n = Ts.shape[0]
    kl32 = np.asarray(c.kappa_lev, np.float32)
    adz32 = np.asarray(np.asarray(c.alpha) * np.asarray(c.dz), np.float32)
    net.set_levels(kl32, adz32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    Tsd, qsd, kmd, td = dev(Ts), dev(qs), dev(km), dev(tend)
    net.fit_norm(Tsd, qsd, kmd, td)
    mi, si, mo, so = net.get_norm()
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    F = omlp.raw_features(f32(Ts), f32(qs), f32(km), kl32.astype(np.float64), 1.0, adz32.astype(np.float64))
    # alpha*dz enters as the product the device was given
    F[:, 174:] = adz32.astype(np.float64)[None, :]
    F[:, 116:174] = (np.float32(1) * (km.astype(np.float32)[:, None] * kl32[None, :])).astype(np.float64)
    mean, sd = omlp.fit_norm(F)
    assert np.allclose(mi, mean, rtol=1e-6, atol=1e-9)
    varying = np.ptp(F, axis=0) > 0
    assert np.allclose(si[varying], sd[varying], rtol=1e-4)
    Tm, Ts_ = omlp.fit_norm(omlp.raw_targets(f32(tend)))
    assert np.allclose(mo, Tm, rtol=1e-5, atol=1e-12)
    assert np.allclose(so, Ts_, rtol=1e-4)
    # prepare: BF16 rows and FP32 targets with the device's normalisation
    pad = (n + 127) // 128 * 128
    X = torch.empty(pad, 512, dtype=torch.bfloat16, device="cuda")
    Yt = torch.empty(pad, 128, dtype=torch.float32, device="cuda")
    net.prepare(Tsd, qsd, kmd, td, X, Yt)
    Xg = X.float().cpu().numpy().astype(np.float64)
    # the same FP32 normalisation on both sides, then the two-term expansion
    hi, lo = omlp.bf16_pair((F.astype(np.float32) - mi) * (np.float32(1) / si))
    assert np.array_equal(Xg[:n, :232], hi) and np.array_equal(Xg[:n, 256:488], lo)
    assert np.all(Xg[n:] == 0) and np.all(Xg[:, 232:256] == 0) and np.all(Xg[:, 488:] == 0)
    Yo = (f32(tend).reshape(n, -1) - mo) / so
    assert np.allclose(Yt[:n, :116].cpu().numpy(), Yo, rtol=1e-5, atol=1e-5)
    assert np.all(Yt[n:].cpu().numpy() == 0) and np.all(Yt[:, 116:].cpu().numpy() == 0)


def test_bad_arguments_are_rejected(net):
    X = torch.zeros(100, 512, dtype=torch.bfloat16, device="cuda")
    Y = torch.zeros(100, 128, dtype=torch.float32, device="cuda")
    with pytest.raises(wx.WxError) as e:
        net.forward(X, Y)
    assert e.value.code == -1
    X = torch.zeros(1024, 512, dtype=torch.bfloat16, device="cuda")
    Y = torch.zeros(1024, 128, dtype=torch.float32, device="cuda")
    with pytest.raises(wx.WxError):
        net.train_step(X, Y, 1e-3)  # above max_batch
    with pytest.raises(wx.WxError) as e:
        net.set_levels(np.zeros(40, np.float32), np.zeros(40, np.float32))
    assert e.value.code == -8
