"""The data-movement kernels the surrogate's training driver uses instead of
PyTorch arithmetic: the state read out as FP32 columns (wx_read_columns_f32),
FP32 <-> FP64 conversion (wx_convert), the minibatch row gather
(wx_gather_rows) and the network's denormalisation (wx_mlp_denormalize),
each against numpy on the same data."""
import numpy as np
import pytest

from paper_1802_05839_gb300 import inputs, wx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("shape", [(37, 29, 8), (1, 5, 3), (70, 33, 58)])
def test_columns_are_the_transposed_state(dtype, shape):
    c = inputs.paper_grid_case(*shape, seed=3)
    ctx = wx.Context(c.nx, c.ny, c.nz, dtype)
    ctx.set_params(c)
    ctx.load_fields(c.T, c.q, c.U, c.V)
    ctx.step(2)
    ctx.sync()
    T, q = ctx.read_fields()
    n = c.nx * c.ny
    Tc = torch.full((n, c.nz), float("nan"), device="cuda")
    qc = torch.full((n, c.nz), float("nan"), device="cuda")
    ctx.read_columns_into(Tc, qc)
    ctx.sync()
    ref = lambda a: a.reshape(c.nz, n).T.astype(np.float32)
    assert np.array_equal(Tc.cpu().numpy(), ref(T)) and np.array_equal(qc.cpu().numpy(), ref(q))
    ctx.read_columns_into(None, qc)  # either output may be omitted
    ctx.close()


def test_convert_round_trip_and_rounding():
    rng = np.random.default_rng(0)
    a = rng.standard_normal(100_003) * 300.0
    d = torch.from_numpy(a).cuda()
    f = torch.empty(a.size, dtype=torch.float32, device="cuda")
    wx.wx_convert(d, f)
    assert np.array_equal(f.cpu().numpy(), a.astype(np.float32))  # round to nearest
    back = torch.empty_like(d)
    wx.wx_convert(f, back)
    assert np.array_equal(back.cpu().numpy(), a.astype(np.float32).astype(np.float64))


def test_gather_rows_and_out_of_range_indices():
    rng = np.random.default_rng(1)
    X = torch.from_numpy(rng.standard_normal((1000, 64)).astype(np.float32)).cuda()
    idx = rng.permutation(1000)[:300].astype(np.int32)
    idx[7] = 5000  # outside the source: a zero row
    dst = torch.full((300, 64), float("nan"), device="cuda")
    wx.wx_gather_rows(X, torch.from_numpy(idx).cuda(), dst)
    ref = X.cpu().numpy()[np.clip(idx, 0, 999)]
    ref[7] = 0.0
    assert np.array_equal(dst.cpu().numpy(), ref)
    Xb = torch.from_numpy(rng.standard_normal((256, 512)).astype(np.float32)).to(torch.bfloat16).cuda()
    db = torch.empty(128, 512, dtype=torch.bfloat16, device="cuda")
    ib = rng.integers(0, 256, 128).astype(np.int32)
    wx.wx_gather_rows(Xb, torch.from_numpy(ib).cuda(), db)
    assert torch.equal(db.cpu(), Xb.cpu()[torch.from_numpy(ib).long()])


def test_denormalize_matches_numpy():
    m = wx.MLP(256)
    rng = np.random.default_rng(2)
    mi, si = rng.standard_normal(232).astype(np.float32), (rng.random(232) + 0.5).astype(np.float32)
    mo, so = rng.standard_normal(116).astype(np.float32), (rng.random(116) + 0.5).astype(np.float32)
    m.set_norm(mi, si, mo, so)
    Y = torch.from_numpy(rng.standard_normal((256, 128)).astype(np.float32)).cuda()
    out = torch.empty(256, 116, device="cuda")
    m.denormalize(Y, out)
    ref = Y.cpu().numpy()[:, :116].astype(np.float64) * so + mo
    assert np.max(np.abs(out.cpu().numpy() - ref) / (np.abs(ref) + 1e-6)) < 1e-6
    m.close()
