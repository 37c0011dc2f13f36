"""wx_sums_noalloc: the FP64 conservation sums for callers that cannot
allocate device memory (graph capture, host-owned device memory, latency-
bound loops).  Its per-tile partials live in a fixed array inside the
library, so this checks it against the step's own sums (wx_get_sums, the
existing entry point) on two calls in a row, which also shows that the
shared array carries nothing over from one call to the next.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test first; it also passes on its own in a fresh
process.
"""
import numpy as np
import pytest

from paper_1802_05839_gb300 import inputs, wx

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 sums tolerance of the step's own sums tests


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_sums_match_step_sums_twice(dtype):
    torch = pytest.importorskip("torch")
    case = inputs.paper_grid_case(150, 90, 24, seed=21, near_singular=True)
    if dtype == "f32":
        case = inputs.round_to_f32(case)
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    ctx.set_params(case, flags=wx.WX_ADVECTION | wx.WX_PHYSICS | wx.WX_SUMS)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    dz = torch.from_numpy(case.dz.copy()).cuda()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    T64 = torch.empty(case.nz, case.ny, case.nx, dtype=torch.float64, device="cuda")
    q64 = torch.empty_like(T64)
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
        assert abs(got[0] - m[-1]) <= TOL * abs(m[-1]), (got[0], m[-1])
        assert abs(got[1] - e[-1]) <= TOL * abs(e[-1]), (got[1], e[-1])
    ctx.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    t = torch.zeros(4, device="cuda")
    dz = torch.ones(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(wx.WxError) as ei:
        # 300 x 300 tiles of 32x4 columns > 65536: refused before any launch
        code = wx.lib().wx_sums_noalloc(wx._dptr(t), wx._dptr(t), wx.WX_F32, 32 * 300, 4 * 300, 1,
                                        wx._dptr(dz), 1.0, wx._dptr(out), None)
        raise wx.WxError(code, wx.lib().wx_sums_noalloc_error().decode())
    assert ei.value.code == -8
    assert b"65536" in wx.lib().wx_sums_noalloc_error()
