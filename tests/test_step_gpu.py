"""GPU parity of the fused step (through the C ABI) against the FP64 oracle.

Tolerances (per step, max relative error normalised by the field's max-abs,
and relative L2 after many steps):
  FP64 path  <= 1e-12 per step
  FP32 path  <= 1e-5 per step, <= 1e-4 relative L2 after 100 steps
The FP32 runs compare against the oracle fed the same inputs rounded once to
FP32 (which is what the FP32 context stores on load).
"""
import numpy as np
import pytest

import oracle
from increments import assert_increments, strong_physics
from paper_1802_05839_gb300 import inputs, wx

pytestmark = pytest.mark.gpu


def maxrel(g, o):
    return float(np.max(np.abs(g - o)) / np.max(np.abs(o)))


def rel_l2(g, o):
    return float(np.linalg.norm((g - o).ravel()) / np.linalg.norm(o.ravel()))


def gpu_run(case, dtype, n, flags=None, per_step=False):
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    ctx.set_params(case, flags=flags)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    out = []
    if per_step:
        for _ in range(n):
            ctx.step(1)
            ctx.sync()
            out.append(ctx.read_fields())
    else:
        ctx.step(n)
        ctx.sync()
        out.append(ctx.read_fields())
    ctx.close()
    return out


def prepared(case, dtype):
    return inputs.round_to_f32(case) if dtype == "f32" else case


TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_small_case_ten_steps_per_step(dtype):
    """128x128x32, 10 steps, each step checked against the oracle advanced
    from the GPU's own previous state (per-step error, not accumulated)."""
    case = prepared(inputs.small_case(), dtype)
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    ctx.set_params(case)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    T, q = case.T, case.q
    for s in range(10):
        ctx.step(1)
        ctx.sync()
        Tg, qg = ctx.read_fields()
        To, qo = oracle.step(case, T, q, case.U, case.V)
        assert maxrel(Tg, To) <= TOL[dtype], (s, maxrel(Tg, To))
        assert maxrel(qg, qo) <= TOL[dtype], (s, maxrel(qg, qo))
        if dtype == "f32":  # the increments, element by element
            Ts, _ = oracle.dynamics(case, T, q, case.U, case.V)
            assert_increments(T, Ts, Tg, To, what=f"step {s}")
        T, q = Tg, qg
    ctx.close()


@pytest.mark.parametrize("shape", [(45, 38, 58), (70, 50, 58), (130, 30, 58), (7, 13, 58)])
def test_tmem_variant_row_ends_over_steps(shape):
    """The FP32 TMEM variant (twelve-row tiles) over several steps on rows
    whose length is not a multiple of the 32-byte sector, and on a row
    shorter than one sector: a ghost column lost or overwritten in step n
    shows from step n + 1 on, at the row ends, so every cell of three steps
    is checked (the increments too)."""
    case = prepared(inputs.paper_grid_case(*shape, seed=5), "f32")
    ctx = wx.Context(case.nx, case.ny, case.nz, "f32")
    ctx.set_params(case)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    assert ctx.step_config()["ty"] == 12
    T, q = case.T, case.q
    for s in range(3):
        ctx.step(1)
        ctx.sync()
        Tg, qg = ctx.read_fields()
        To, qo = oracle.step(case, T, q, case.U, case.V)
        assert maxrel(Tg, To) <= TOL["f32"] and maxrel(qg, qo) <= TOL["f32"], (s, maxrel(Tg, To), maxrel(qg, qo))
        Ts, _ = oracle.dynamics(case, T, q, case.U, case.V)
        assert_increments(T, Ts, Tg, To, what=f"{shape} step {s}")
        T, q = Tg, qg
    ctx.close()


@pytest.mark.parametrize("near_singular", [False, True])
def test_f32_strong_physics_increments(near_singular):
    """FP32 step on a case whose physics increment is ~1 K (a +-5 K level
    zig-zag, ten times the vertical diffusivity, S0 = 100): the increments
    T^{n+1} - T* and T^{n+1} - T^n within 8 ulp of max|T| of the oracle's,
    which resolves the physics to a few 1e-3 of its size; with near-singular
    columns this covers the FP32 side solve of the kappa_mult columns."""
    case = inputs.round_to_f32(strong_physics(
        inputs.paper_grid_case(96, 80, 58, seed=4, near_singular=near_singular)))
    ctx = wx.Context(case.nx, case.ny, case.nz, "f32")
    ctx.set_params(case)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    T, q = case.T, case.q
    for s in range(3):
        ctx.step(1)
        ctx.sync()
        Tg, qg = ctx.read_fields()
        To, qo = oracle.step(case, T, q, case.U, case.V)
        Ts, _ = oracle.dynamics(case, T, q, case.U, case.V)
        r = assert_increments(T, Ts, Tg, To, what=f"step {s}", resolve=0.01)
        print(f"step {s}: {r['err_ulp']:.2f} ulp, rel to the physics increment {r['rel_phys']:.2e}")
        assert maxrel(qg, qo) <= 1e-5
        T, q = Tg, qg
    ctx.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(37, 29, 8), (33, 5, 3), (1, 1, 1), (1, 7, 5), (65, 1, 4),
                                   (96, 64, 58), (31, 33, 97)])
def test_ragged_and_degenerate_shapes(dtype, shape):
    """Odd sizes (ragged last tile in x and y), single-column and single-row
    periodic grids, nz = 1, and deep columns."""
    nx, ny, nz = shape
    case = prepared(inputs.paper_grid_case(nx, ny, nz, seed=11, near_singular=True), dtype)
    (Tg, qg), = gpu_run(case, dtype, 3)
    To, qo = oracle.run(case, 3, case.T, case.q, case.U, case.V)
    tol = 3 * TOL[dtype]
    assert maxrel(Tg, To) <= tol, maxrel(Tg, To)
    assert maxrel(qg, qo) <= tol, maxrel(qg, qo)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("adv,phys", [(False, False), (True, False), (False, True)])
def test_flag_combinations(dtype, adv, phys):
    case = prepared(inputs.paper_grid_case(45, 38, 12, seed=2), dtype)
    case.advection, case.physics = adv, phys
    (Tg, qg), = gpu_run(case, dtype, 2)
    To, qo = oracle.run(case, 2, case.T, case.q, case.U, case.V)
    assert maxrel(Tg, To) <= 2 * TOL[dtype]
    assert maxrel(qg, qo) <= 2 * TOL[dtype]


def test_f32_hundred_steps_relative_l2():
    """FP32 path after 100 steps: relative L2 error <= 1e-4 per field."""
    case = inputs.round_to_f32(inputs.paper_grid_case(96, 80, 24, seed=4))
    (Tg, qg), = gpu_run(case, "f32", 100)
    To, qo = oracle.run(case, 100, case.T, case.q, case.U, case.V)
    assert rel_l2(Tg, To) <= 1e-4, rel_l2(Tg, To)
    assert rel_l2(qg, qo) <= 1e-4, rel_l2(qg, qo)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_sums_match_oracle(dtype):
    """FP64 mass/energy sums recorded after every step: FP64 path within
    1e-12 of the oracle's sums; the FP32 path's sums are those of its own
    FP32 state, so they are held to the FP32 field tolerance."""
    case = prepared(inputs.paper_grid_case(70, 50, 20, seed=8, near_singular=True), dtype)
    flags = wx.WX_ADVECTION | wx.WX_PHYSICS | wx.WX_SUMS
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    ctx.set_params(case, flags=flags)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    ctx.step(5)
    ctx.sync()
    m, e = ctx.sums()
    Tg, qg = ctx.read_fields()
    ctx.close()
    _, _, mo, eo = oracle.run(case, 5, case.T, case.q, case.U, case.V, sums=True)
    assert len(m) == 5
    tol = 1e-12 if dtype == "f64" else 1e-5
    assert np.max(np.abs(m - mo) / np.abs(mo)) <= tol
    assert np.max(np.abs(e - eo) / np.abs(eo)) <= tol
    # the recorded sums are the sums of the state the GPU holds (FP64 tally)
    w = case.h ** 2 * case.dz[:, None, None]
    assert abs(e[-1] - np.sum(Tg * w)) / abs(e[-1]) < 1e-12
    assert abs(m[-1] - np.sum(qg * w)) / abs(m[-1]) < 1e-12


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_paper_grid_full_size_sampled(dtype):
    """1581x1301x58 (the paper's grid), one step in the bench's launch
    configuration; checked at 4000 sampled columns (all edges and corners
    included) against the oracle's per-column step."""
    case = prepared(inputs.paper_grid_case(), dtype)
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    ctx.set_params(case)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    ctx.step(1)
    ctx.sync()
    Tg, qg = ctx.read_fields()
    ctx.close()
    rng = np.random.default_rng(0)
    ci = np.concatenate([rng.integers(0, case.nx, 3900), [0, case.nx - 1, 0, case.nx - 1] * 25])
    cj = np.concatenate([rng.integers(0, case.ny, 3900), [0, 0, case.ny - 1, case.ny - 1] * 25])
    To, qo = oracle.step_columns(case, case.T, case.q, case.U, case.V, ci, cj)
    Tgs, qgs = Tg[:, cj, ci].T, qg[:, cj, ci].T
    scaleT, scaleq = np.max(np.abs(case.T)), np.max(np.abs(case.q))
    assert np.max(np.abs(Tgs - To)) / scaleT <= TOL[dtype]
    assert np.max(np.abs(qgs - qo)) / scaleq <= TOL[dtype]
    if dtype == "f32":  # increments at the sampled columns (T* from the dynamics alone)
        dyn = case.copy()
        dyn.physics = False
        Ts, _ = oracle.step_columns(dyn, case.T, case.q, case.U, case.V, ci, cj)
        assert_increments(case.T[:, cj, ci].T, Ts, Tgs, To, what="paper grid, sampled columns")
    # whole-field properties at full size: finite, and q inside its old range
    assert np.isfinite(Tg).all() and np.isfinite(qg).all()
    assert qg.min() >= case.q.min() - 1e-7 and qg.max() <= case.q.max() + 1e-7


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_checkpoint_resume_is_bitwise(dtype):
    """read_fields -> load_fields -> step equals the uninterrupted run."""
    case = prepared(inputs.paper_grid_case(40, 36, 10, seed=6), dtype)
    (Ta, qa), = gpu_run(case, dtype, 6)
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    ctx.set_params(case)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    ctx.step(3)
    ctx.sync()
    T3, q3 = ctx.read_fields()
    ctx.close()
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    ctx.set_params(case)
    ctx.load_fields(T3, q3, case.U, case.V)
    ctx.step(3)
    ctx.sync()
    Tb, qb = ctx.read_fields()
    ctx.close()
    assert np.array_equal(Ta, Tb) and np.array_equal(qa, qb)


def test_deterministic_runs():
    case = inputs.paper_grid_case(200, 150, 30, seed=9)
    flags = wx.WX_ADVECTION | wx.WX_PHYSICS | wx.WX_SUMS
    outs = []
    for _ in range(2):
        ctx = wx.Context(case.nx, case.ny, case.nz, "f32")
        ctx.set_params(case, flags=flags)
        ctx.load_fields(case.T, case.q, case.U, case.V)
        ctx.step(4)
        ctx.sync()
        outs.append((*ctx.read_fields(), *ctx.sums()))
        ctx.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_device_pointer_load_and_read():
    torch = pytest.importorskip("torch")
    case = inputs.paper_grid_case(50, 40, 9, seed=3)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = wx.Context(case.nx, case.ny, case.nz, "f64")
    ctx.set_params(case)
    ctx.load_fields(dev(case.T), dev(case.q), dev(case.U), dev(case.V))
    s = torch.cuda.current_stream()
    ctx.step(2, stream=s)
    Td = torch.empty(case.nz, case.ny, case.nx, dtype=torch.float64, device="cuda")
    qd = torch.empty_like(Td)
    ctx.read_fields_into(Td, qd, stream=s)
    ctx.sync()
    torch.cuda.synchronize()
    To, qo = oracle.run(case, 2, case.T, case.q, case.U, case.V)
    assert maxrel(Td.cpu().numpy(), To) <= 1e-12
    assert maxrel(qd.cpu().numpy(), qo) <= 1e-12
    ctx.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_physics_columns(dtype):
    torch = pytest.importorskip("torch")
    case = prepared(inputs.paper_grid_case(30, 20, 58, seed=5, near_singular=True), dtype)
    rng = np.random.default_rng(1)
    ncol = 1000
    Ts = 280 + rng.normal(0, 2, (ncol, case.nz))
    qs = rng.uniform(0, 0.02, (ncol, case.nz))
    km = np.where(rng.random(ncol) < 0.1, 10 ** rng.uniform(4, 5, ncol), 1.0)
    if dtype == "f32":
        Ts, qs, km = (a.astype(np.float32).astype(np.float64) for a in (Ts, qs, km))
    tdt = torch.float64 if dtype == "f64" else torch.float32
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=tdt)
    Tout = torch.empty(ncol, case.nz, dtype=tdt, device="cuda")
    tend = torch.empty(ncol, 2, case.nz, dtype=tdt, device="cuda")
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    ctx.set_params(case)
    ctx.physics_columns(d(Ts), d(qs), d(km), Tout, tend)
    ctx.sync()
    To, tendo = oracle.physics_columns(case.nz, case.dt, case.dz, case.kappa_lev, km, case.alpha,
                                       case.S0, case.q_ref, Ts, qs, with_tend=True)
    g = Tout.double().cpu().numpy()
    assert maxrel(g, To) <= TOL[dtype]
    gt = tend.double().cpu().numpy()
    # tendencies: heating and vertical-diffusion rate, normalised per kind
    tol_t = 1e-10 if dtype == "f64" else 2e-2
    for kind in range(2):
        assert maxrel(gt[:, kind], tendo[:, kind]) <= tol_t
    ctx.close()


def test_nonfinite_input_is_reported():
    case = inputs.paper_grid_case(40, 30, 6, seed=1)
    T = case.T.copy()
    T[3, 7, 11] = np.nan
    ctx = wx.Context(case.nx, case.ny, case.nz, "f32")
    ctx.set_params(case)
    ctx.load_fields(T, case.q, case.U, case.V)
    ctx.step(1)
    with pytest.raises(wx.WxError) as ei:
        ctx.sync()
    assert ei.value.code == -5
    ctx.close()


def test_cfl_violation_is_refused():
    case = inputs.paper_grid_case(40, 30, 6, seed=1)
    ctx = wx.Context(case.nx, case.ny, case.nz, "f32")
    ctx.set_params(case)
    ctx.load_fields(case.T, case.q, 5 * case.U, 5 * case.V)
    with pytest.raises(wx.WxError) as ei:
        ctx.step(1)
    assert ei.value.code == -4
    with pytest.raises(wx.WxError) as ei:
        wx.Context(8, 8, 4, "f32").step(1)
    assert ei.value.code == -7
    ctx.close()


def test_bounded_wait_gives_up_and_context_survives():
    """A wait that nothing will end returns WX_ETIMEOUT after its limit (the
    failure-detection path every kernel's waits share), and the context can
    still step afterwards."""
    code, waited = wx.wx_selftest_wait_timeout(20_000_000)  # 20 ms
    assert code == -6
    assert 20_000_000 <= waited < 2_000_000_000
    case = inputs.round_to_f32(inputs.small_case(40, 30, 8))
    ctx = wx.Context(40, 30, 8, "f32")
    ctx.set_params(case)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    ctx.step(2)
    ctx.sync()
    T, _ = ctx.read_fields()
    To, _ = oracle.run(case, 2, case.T, case.q, case.U, case.V)
    assert np.max(np.abs(T - To)) / np.max(np.abs(To)) <= 1e-5
    ctx.close()
    assert wx.wx_selftest_wait_timeout(0)[0] == -1


@pytest.mark.parametrize("dtype,km", [("f64", False), ("f32", True), ("mixed", True)])
def test_deepest_columns(dtype, km):
    """nz = 256, the deepest column wx_create accepts (the launch
    configuration falls back to short tiles to fit the per-column state),
    with and without a per-column kappa_mult."""
    case = inputs.paper_grid_case(40, 9, 256, seed=12, near_singular=km)
    if dtype != "f64":
        case = inputs.round_to_f32(case)
    (Tg, qg), = gpu_run(case, dtype, 3)
    To, qo = oracle.run(case, 3, case.T, case.q, case.U, case.V)
    tol = 3 * TOL["f64" if dtype == "f64" else "f32"]
    assert maxrel(Tg, To) <= tol and maxrel(qg, qo) <= tol


def test_fp64_kappa_mult_depth_limit():
    """FP64 with a per-column kappa_mult eliminates per column on the fly and
    keeps two values per level of every column in shared memory: 174 levels
    run (checked against the oracle), 175 are refused at wx_set_params."""
    case = inputs.paper_grid_case(33, 6, 174, seed=13, near_singular=True)
    (Tg, qg), = gpu_run(case, "f64", 2)
    To, qo = oracle.run(case, 2, case.T, case.q, case.U, case.V)
    assert maxrel(Tg, To) <= 3e-12 and maxrel(qg, qo) <= 3e-12
    deep = inputs.paper_grid_case(8, 4, 175, seed=13, near_singular=True)
    ctx = wx.Context(8, 4, 175, "f64")
    with pytest.raises(wx.WxError) as e:
        ctx.set_params(deep)
    assert e.value.code == -8 and "174" in str(e.value)
    ctx.close()


def test_zero_work_is_a_no_op():
    """Empty requests: zero steps (single grid, ensemble with and without a
    graph, reduced application) and zero columns leave every state bit for
    bit and launch nothing; negative step counts are refused."""
    import torch
    case = inputs.round_to_f32(inputs.paper_grid_case(40, 24, 10, seed=14))
    ctx = wx.Context(case.nx, case.ny, case.nz, "f32")
    ctx.set_params(case)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    before = ctx.read_fields()
    ctx.step(0)
    ctx.sync()
    assert ctx.last_launches() == 0
    after = ctx.read_fields()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    e = torch.empty(0, dtype=torch.float32, device="cuda")
    ctx.physics_columns(e, e, None, e, None)
    ctx.sync()
    with pytest.raises(wx.WxError) as err:
        ctx.step(-1)
    assert err.value.code == -1
    ctx.close()
    ens = wx.Ensemble([(case.nx, case.ny, case.nz)], "f32")
    m = ens.members[0]
    m.set_params(case)
    m.load_fields(case.T, case.q, case.U, case.V)
    for graph in (False, True):
        ens.step(0, graph=graph)
        ens.sync()
        assert ens.last_launches() == 0
    out = m.read_fields()
    assert np.array_equal(out[0], before[0]) and np.array_equal(out[1], before[1])
    ens.close()
    app = wx.ReducedApp(9, 7, 4, "f64")
    app.set_params()
    E = np.arange(4 * 9 * 11, dtype=np.float64).reshape(4, 9, 11)
    app.load(E)
    app.step(0)
    app.sync()
    assert app.last_launches() == 0 and np.array_equal(app.read(), E)
    app.close()
