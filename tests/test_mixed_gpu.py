"""WX_MIXED: FP32 fields and stencil, FP64 conservation sums, and the FP64
Thomas elimination for columns whose diagonal dominance ratio
min_k |b_k|/(|a_k|+|c_k|) is below 1.1.  Errors are stated against the FP64
oracle run on the same FP32-rounded inputs."""
import numpy as np
import pytest

import oracle
from increments import assert_increments, strong_physics
from paper_1802_05839_gb300 import inputs, wx

pytestmark = pytest.mark.gpu


def maxrel(g, o):
    return float(np.max(np.abs(g - o)) / np.max(np.abs(o)))


def dominance_ratio(case, km):
    a, b, c = oracle.vdiff_coeffs(case.nz, case.dt, case.dz, case.kappa_lev, km)
    off = np.abs(a) + np.abs(c)
    return np.min(np.abs(b)[off > 0] / off[off > 0])


def run(case, dtype, n, sums=False):
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    flags = wx.WX_ADVECTION | wx.WX_PHYSICS | (wx.WX_SUMS if sums else 0)
    ctx.set_params(case, flags=flags)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    nflag = ctx.flagged_columns()
    ctx.step(n)
    ctx.sync()
    T, q = ctx.read_fields()
    m, e = ctx.sums() if sums else (None, None)
    ctx.close()
    return T, q, nflag, m, e


def test_flagged_columns_are_the_weakly_dominant_ones():
    case = inputs.round_to_f32(inputs.paper_grid_case(97, 61, 58, seed=3, near_singular=True))
    km = case.kappa_mult.reshape(-1)
    expect = int(np.sum([dominance_ratio(case, s) < 1.1 for s in km]))
    ctx = wx.Context(case.nx, case.ny, case.nz, "mixed")
    ctx.set_params(case)
    assert ctx.flagged_columns() == expect
    frac = expect / km.size
    assert 0.03 < frac < 0.07  # about 5% of columns, as the input recipe seeds
    ctx.close()


def per_step(case, dtype, n, flags=None):
    """n steps one at a time; each checked against the oracle step from the
    GPU's own previous state: field error <= 1e-5, and the increments (all
    columns, then the listed kappa_mult != 1 ones alone) within 8 ulp."""
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    ctx.set_params(case, flags=flags)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    listed = np.broadcast_to((case.kappa_mult != 1.0)[None], (case.nz, case.ny, case.nx))
    T, q = case.T, case.q
    for s in range(n):
        ctx.step(1)
        ctx.sync()
        Tg, qg = ctx.read_fields()
        To, qo = oracle.step(case, T, q, case.U, case.V)
        assert maxrel(Tg, To) <= 1e-5 and maxrel(qg, qo) <= 1e-5, (s, maxrel(Tg, To), maxrel(qg, qo))
        Ts, _ = oracle.dynamics(case, T, q, case.U, case.V)
        assert_increments(T, Ts, Tg, To, what=f"{dtype} step {s}")
        if listed.any():
            assert_increments(T, Ts, Tg, To, mask=listed, what=f"{dtype} step {s}, listed columns")
        T, q = Tg, qg
    ctx.close()


@pytest.mark.parametrize("shape", [(97, 61, 58), (70, 33, 17), (1, 5, 9)])
def test_mixed_matches_oracle(shape):
    nx, ny, nz = shape
    case = inputs.round_to_f32(inputs.paper_grid_case(nx, ny, nz, seed=5, near_singular=True))
    Tg, qg, nflag, _, _ = run(case, "mixed", 5)
    To, qo = oracle.run(case, 5, case.T, case.q, case.U, case.V)
    # five steps accumulated: five times the per-step bound
    assert maxrel(Tg, To) <= 5e-5 and maxrel(qg, qo) <= 5e-5
    per_step(case, "mixed", 3)


@pytest.mark.parametrize("dtype", ["mixed", "f32"])
def test_strong_physics_increments_with_kappa_mult(dtype):
    """Physics increments ~1 K on well-conditioned columns and several K on
    the near-singular ones (FP64 elimination under WX_MIXED, the FP32 side
    solve under WX_F32): both within 8 ulp of the oracle's."""
    case = inputs.round_to_f32(strong_physics(
        inputs.paper_grid_case(97, 61, 58, seed=3, near_singular=True)))
    per_step(case, dtype, 3)


def test_mixed_improves_flagged_columns_over_fp32():
    """On the near-singular columns the FP64 elimination is at least as close
    to the FP64 oracle as the all-FP32 path (stated per field)."""
    case = inputs.round_to_f32(inputs.paper_grid_case(128, 96, 58, seed=8, near_singular=True))
    To, qo = oracle.run(case, 10, case.T, case.q, case.U, case.V)
    Tm, qm, nflag, _, _ = run(case, "mixed", 10)
    Tf, qf, _, _, _ = run(case, "f32", 10)
    mask = (case.kappa_mult > 1)[None]
    err_m = np.max(np.abs(Tm - To)[np.broadcast_to(mask, To.shape)])
    err_f = np.max(np.abs(Tf - To)[np.broadcast_to(mask, To.shape)])
    print(f"flagged {nflag}: max |T err| mixed {err_m:.3e} K, fp32 {err_f:.3e} K")
    assert nflag > 0
    assert err_m <= err_f * 1.05 + 1e-6
    assert maxrel(qm, qo) <= 1e-4


def test_mixed_sums_each_step():
    case = inputs.round_to_f32(inputs.paper_grid_case(90, 70, 30, seed=2, near_singular=True))
    Tg, qg, nflag, m, e = run(case, "mixed", 6, sums=True)
    _, _, mo, eo = oracle.run(case, 6, case.T, case.q, case.U, case.V, sums=True)
    assert len(m) == 6
    assert np.max(np.abs(m - mo) / np.abs(mo)) <= 1e-5
    assert np.max(np.abs(e - eo) / np.abs(eo)) <= 1e-5
    w = case.h ** 2 * case.dz[:, None, None]
    assert abs(e[-1] - np.sum(Tg * w)) / abs(e[-1]) < 1e-12
    assert abs(m[-1] - np.sum(qg * w)) / abs(m[-1]) < 1e-12


def test_error_against_the_oracle_at_steps_1_100_500():
    """The mixed-precision configuration's error per field against the FP64
    oracle after 1, 100 and 500 steps (near-singular columns seeded), beside
    the all-FP32 path.  Bounds: relative L2 1e-5 / 1e-4 / 5e-4."""
    case = inputs.round_to_f32(inputs.paper_grid_case(192, 160, 58, seed=11, near_singular=True))
    marks = (1, 100, 500)
    got = {}
    for dtype in ("mixed", "f32"):
        ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
        ctx.set_params(case)
        ctx.load_fields(case.T, case.q, case.U, case.V)
        done, out = 0, []
        for m in marks:
            ctx.step(m - done)
            done = m
            ctx.sync()
            out.append(ctx.read_fields())
        ctx.close()
        got[dtype] = out
    T, q = case.T.copy(), case.q.copy()
    done = 0
    for idx, m in enumerate(marks):
        T, q = oracle.run(case, m - done, T, q, case.U, case.V)
        done = m
        for dtype in ("mixed", "f32"):
            Tg, qg = got[dtype][idx]
            eT = np.linalg.norm(Tg - T) / np.linalg.norm(T)
            eq = np.linalg.norm(qg - q) / np.linalg.norm(q)
            print(f"step {m:3d} {dtype:5s}: rel L2 T {eT:.3e} q {eq:.3e}; "
                  f"max rel T {maxrel(Tg, T):.3e} q {maxrel(qg, q):.3e}")
            if dtype == "mixed":
                bound = {1: 1e-5, 100: 1e-4, 500: 5e-4}[m]
                assert eT <= bound and eq <= bound


@pytest.mark.parametrize("shape", [(97, 61, 58), (70, 33, 17)])
def test_fp32_with_kappa_mult_matches_oracle(shape):
    """WX_F32 with a kappa_mult field: the table path plus the FP32 side
    solve of the kappa_mult != 1 columns, within the FP32 per-step bound
    (1e-5) and the increment bar, on all columns and the listed ones."""
    nx, ny, nz = shape
    case = inputs.round_to_f32(inputs.paper_grid_case(nx, ny, nz, seed=7, near_singular=True))
    ctx = wx.Context(nx, ny, nz, "f32")
    ctx.set_params(case)
    assert ctx.flagged_columns() == 0      # none in FP64
    ctx.close()
    per_step(case, "f32", 3)


def test_c3_full_size_sampled():
    """The mixed-precision workload at its full size (1581x1301x58,
    near-singular columns seeded, FP64 sums on), one step in the bench's
    launch configuration: 3000 sampled columns plus 1000 flagged ones and
    the corners against the oracle's per-column step (FP32 per-step bound),
    and the recorded sums against the FP64 sums of the GPU state."""
    case = inputs.round_to_f32(inputs.paper_grid_case(near_singular=True))
    ctx = wx.Context(case.nx, case.ny, case.nz, "mixed")
    ctx.set_params(case, flags=wx.WX_ADVECTION | wx.WX_PHYSICS | wx.WX_SUMS)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    assert ctx.flagged_columns() > 0
    ctx.step(1)
    ctx.sync()
    Tg, qg = ctx.read_fields()
    m, e = ctx.sums()
    ctx.close()
    rng = np.random.default_rng(1)
    flagged = np.flatnonzero(case.kappa_mult.reshape(-1) != 1.0)
    pick = rng.choice(flagged, 1000, replace=False)
    ci = np.concatenate([rng.integers(0, case.nx, 3000), pick % case.nx, [0, case.nx - 1, 0, case.nx - 1]])
    cj = np.concatenate([rng.integers(0, case.ny, 3000), pick // case.nx, [0, 0, case.ny - 1, case.ny - 1]])
    To, qo = oracle.step_columns(case, case.T, case.q, case.U, case.V, ci, cj)
    Tgs, qgs = Tg[:, cj, ci].T, qg[:, cj, ci].T
    assert np.max(np.abs(Tgs - To)) / np.max(np.abs(case.T)) <= 1e-5
    assert np.max(np.abs(qgs - qo)) / np.max(np.abs(case.q)) <= 1e-5
    dyn = case.copy()
    dyn.physics = False
    Ts, _ = oracle.step_columns(dyn, case.T, case.q, case.U, case.V, ci, cj)
    Tin = case.T[:, cj, ci].T
    assert_increments(Tin, Ts, Tgs, To, what="C3 sampled columns")
    assert_increments(Tin[3000:4000], Ts[3000:4000], Tgs[3000:4000], To[3000:4000],
                      what="C3 flagged columns")
    w = case.h ** 2 * case.dz[:, None, None]
    assert len(m) == 1
    assert abs(e[-1] - np.sum(Tg * w)) / abs(e[-1]) < 1e-12
    assert abs(m[-1] - np.sum(qg * w)) / abs(m[-1]) < 1e-12
