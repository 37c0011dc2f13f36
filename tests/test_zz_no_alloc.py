"""wx_sums_noalloc: the FP64 conservation sums for callers that cannot
allocate device memory (a plug-in whose host application owns every device
byte through its own pool, or a real-time loop that cannot accept
cudaMalloc's synchronisation and latency).  Its per-tile partials live in a
fixed array inside the library, so this checks it against the step's own
sums (wx_get_sums, the existing entry point) and against a numpy FP64 sum of
the same state on two calls in a row, which also shows that the shared array
carries nothing over from one call to the next.  The FP32 case keeps the
unrounded FP64 layer thicknesses, so a dz rounded to float would fail it.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test first; it also passes on its own in a fresh
process.
"""
import numpy as np
import pytest

from paper_1802_05839_gb300 import inputs, wx

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 sums tolerance of the step's own sums tests
EUNSUPPORTED = -8  # WX_EUNSUPPORTED


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_sums_match_step_sums_twice(dtype):
    torch = pytest.importorskip("torch")
    # FP64 inputs as generated: dz_k = 1.05^k is not a float, so the FP32
    # path must carry it beyond single precision to stay within TOL
    case = inputs.paper_grid_case(150, 90, 24, seed=21, near_singular=True)
    assert np.any(case.dz != case.dz.astype(np.float32).astype(np.float64))
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    ctx.set_params(case, flags=wx.WX_ADVECTION | wx.WX_PHYSICS | wx.WX_SUMS)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    dz = torch.from_numpy(case.dz.copy()).cuda()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    T64 = torch.empty(case.nz, case.ny, case.nx, dtype=torch.float64, device="cuda")
    q64 = torch.empty_like(T64)
    w = case.h ** 2 * case.dz[:, None, None]
    for steps in (3, 2):  # two calls in a row, on two different states
        ctx.step(steps)
        ctx.sync()
        m, e = ctx.sums()
        ctx.read_fields_into(T64, q64)
        torch.cuda.synchronize()
        Tf, qf = T64.to(tdt).contiguous(), q64.to(tdt).contiguous()
        wx.wx_sums_noalloc(Tf, qf, dz, case.h, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # the stored state (exact in FP64) times the FP64 dz, summed in numpy
        mo = float(np.sum(qf.double().cpu().numpy() * w))
        eo = float(np.sum(Tf.double().cpu().numpy() * w))
        assert abs(got[0] - mo) <= TOL * abs(mo), (got[0], mo)
        assert abs(got[1] - eo) <= TOL * abs(eo), (got[1], eo)
        assert abs(got[0] - m[-1]) <= TOL * abs(m[-1]), (got[0], m[-1])
        assert abs(got[1] - e[-1]) <= TOL * abs(e[-1]), (got[1], e[-1])
    ctx.close()


def _call(t, dz, out, nx, ny):
    return wx.lib().wx_sums_noalloc(wx._dptr(t), wx._dptr(t), wx.WX_F32, nx, ny, 1,
                                    wx._dptr(dz), 1.0, wx._dptr(out), None)


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    t = torch.zeros(4, device="cuda")
    dz = torch.ones(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    # 300 x 300 tiles of 32x4 columns > 65536: refused before any launch
    assert _call(t, dz, out, 32 * 300, 4 * 300) == EUNSUPPORTED
    assert b"65536" in wx.lib().wx_sums_noalloc_error()
    # one column, 65536 tile rows: within the tile count, beyond the row limit
    assert _call(t, dz, out, 1, 4 * 65536) == EUNSUPPORTED
    assert b"262140" in wx.lib().wx_sums_noalloc_error()
