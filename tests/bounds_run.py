"""Run by tests/test_bounds_gpu.py in a child process whose WX_LIBRARY points
at the bounds-checked libwx_bounds.so: every grid path on ragged and
degenerate shapes (edge tiles, one-column and one-row grids, listed
columns, blocks of a decomposition, ensemble members, RK3 stages, the
reduced application).  Every synchronisation must report no skipped
access, and the results must still match the oracle."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_1802_05839_gb300 import inputs, wx  # noqa: E402

assert os.path.basename(wx.LIB_PATH) == "libwx_bounds.so", wx.LIB_PATH
F = wx.WX_ADVECTION | wx.WX_PHYSICS


def maxrel(g, o):
    return float(np.max(np.abs(g - o)) / max(np.max(np.abs(o)), 1e-300))


def check(tag, got, ref, tol):
    for g, o in zip(got, ref):
        e = maxrel(g, o)
        assert e <= tol, (tag, e)
    print("ok", tag, flush=True)


for dtype, tol in (("f64", 3e-12), ("f32", 3e-5)):
    for shape in [(37, 29, 8), (33, 5, 3), (1, 1, 1), (1, 7, 5), (65, 1, 4), (96, 64, 58), (31, 33, 97)]:
        c = inputs.paper_grid_case(*shape, seed=11, near_singular=True)
        if dtype == "f32":
            c = inputs.round_to_f32(c)
        ctx = wx.Context(c.nx, c.ny, c.nz, dtype)
        ctx.set_params(c, flags=F | wx.WX_SUMS)
        ctx.load_fields(c.T, c.q, c.U, c.V)
        ctx.step(3)
        ctx.sync()  # raises WxError on a skipped out-of-bounds access
        check(f"step {dtype} {shape}", ctx.read_fields(), oracle.run(c, 3, c.T, c.q, c.U, c.V), tol)
        ctx.close()

c = inputs.round_to_f32(inputs.paper_grid_case(70, 33, 17, seed=5, near_singular=True))
ctx = wx.Context(c.nx, c.ny, c.nz, "mixed")
ctx.set_params(c, flags=F | wx.WX_SUMS)
ctx.load_fields(c.T, c.q, c.U, c.V)
ctx.step(3)
ctx.sync()
check("mixed", ctx.read_fields(), oracle.run(c, 3, c.T, c.q, c.U, c.V), 5e-5)
ctx.close()

d = wx.Decomposition(c.nx, c.ny, c.nz, "f32", 4, 2, [0, 1, 2, 35, 70], [0, 1, 33])
d.set_params(c)
d.load_fields(c.T, c.q, c.U, c.V)
d.step(3)
d.sync()
check("decomposition", d.read_fields(), oracle.run(c, 3, c.T, c.q, c.U, c.V), 5e-5)
d.close()

sizes = [(65, 17, 9), (3, 40, 12), (1, 1, 5)]
ens = wx.Ensemble(sizes, "f32")
cases = []
for m, (mem, s) in enumerate(zip(ens.members, sizes)):
    cc = inputs.round_to_f32(inputs.ensemble_member(m, *s))
    mem.set_params(cc)
    mem.load_fields(cc.T, cc.q, cc.U, cc.V)
    cases.append(cc)
ens.step(2, graph=True)
ens.sync()
for mem, cc in zip(ens.members, cases):
    check(f"ensemble member {cc.nx}x{cc.ny}x{cc.nz}", mem.read_fields(), oracle.run(cc, 2, cc.T, cc.q, cc.U, cc.V), 5e-5)
ens.close()

for dtype, tol in (("f32", 5e-5), ("f64", 3e-12)):
    cc = inputs.paper_grid_case(37, 29, 8, seed=4, near_singular=True)
    if dtype == "f32":
        cc = inputs.round_to_f32(cc)
    ctx = wx.Context(cc.nx, cc.ny, cc.nz, dtype)
    ctx.set_params(cc, flags=F | wx.WX_RK3)
    ctx.load_fields(cc.T, cc.q, cc.U, cc.V)
    ctx.step(2)
    ctx.sync()
    check(f"rk3 {dtype}", ctx.read_fields(), oracle.run_rk3(cc, 2, cc.T, cc.q, cc.U, cc.V), tol)
    ctx.close()

p = oracle.pf_params(13, 9, 6)
E = inputs.paper_box_state(13, 9, 6)
app = wx.ReducedApp(13, 9, 6, "f64")
app.set_params()
app.load(E)
app.step(3)
app.sync()
check("reduced application", [app.read()], [oracle.pf_run(p, 3, E)], 1e-12)
app.close()
print("BOUNDS_RUN_OK")
