"""The horizontal (IJ) decomposition with a depth-1 halo exchange (the
paper's block decomposition of ASUCA, App. F, Sec. 5.4) on one GPU: every
block's interior equals the undecomposed step bit for bit (uneven splits,
one-column and one-row blocks, kappa_mult and mixed precision included),
the whole grid stays within the oracle's per-step bars, the combined FP64
sums match the undecomposed ones and the FP64 sums of the state, and the
refusals hold."""
import numpy as np
import pytest

import oracle
from increments import assert_increments
from paper_1802_05839_gb300 import inputs, wx

pytestmark = pytest.mark.gpu

FLAGS = wx.WX_ADVECTION | wx.WX_PHYSICS


def single(case, dtype, n, flags=FLAGS):
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    ctx.set_params(case, flags=flags)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    ctx.step(n)
    ctx.sync()
    out = ctx.read_fields() + (ctx.sums() if flags & wx.WX_SUMS else (None, None))
    ctx.close()
    return out


def decomposed(case, dtype, n, px, py, xs=None, ys=None, flags=FLAGS):
    d = wx.Decomposition(case.nx, case.ny, case.nz, dtype, px, py, xs, ys)
    d.set_params(case, flags=flags)
    d.load_fields(case.T, case.q, case.U, case.V)
    d.step(n)
    d.sync()
    launches = d.last_launches()  # the step kernel and the exchange kernel per step
    out = d.read_fields() + (d.sums() if flags & wx.WX_SUMS else (None, None))
    d.close()
    return out, launches


SPLITS = [  # px, py, xsplit, ysplit
    (2, 1, None, None),
    (2, 1, [0, 1, 45], None),             # a one-column block
    (2, 2, [0, 20, 45], [0, 1, 38]),      # a one-row block
    (1, 4, None, [0, 3, 4, 30, 38]),
    (4, 4, [0, 1, 2, 30, 45], [0, 10, 11, 12, 38]),
]


@pytest.mark.parametrize("dtype,nz", [("f32", 58), ("f64", 58), ("f32", 12)])
@pytest.mark.parametrize("px,py,xs,ys", SPLITS)
def test_blocks_equal_the_undecomposed_step_bitwise(dtype, nz, px, py, xs, ys):
    """FP32 at 58 levels (the TMEM variant), FP64, and FP32 with 12 levels
    (8-row tiles)."""
    case = inputs.paper_grid_case(45, 38, nz, seed=5)
    if dtype == "f32":
        case = inputs.round_to_f32(case)
    Ta, qa, _, _ = single(case, dtype, 10)
    (Tb, qb, _, _), launches = decomposed(case, dtype, 10, px, py, xs, ys)
    assert np.array_equal(Ta, Tb) and np.array_equal(qa, qb)
    assert launches == 10 * 2


@pytest.mark.parametrize("dtype", ["f32", "mixed"])
def test_kappa_mult_and_mixed_precision_blocks_bitwise(dtype):
    """Near-singular columns (side solve, FP64 elimination under WX_MIXED)
    split across blocks, some of which hold no listed column at all."""
    case = inputs.round_to_f32(inputs.paper_grid_case(70, 33, 17, seed=5, near_singular=True))
    Ta, qa, _, _ = single(case, dtype, 10)
    (Tb, qb, _, _), _ = decomposed(case, dtype, 10, 4, 2, [0, 1, 2, 35, 70], [0, 1, 33])
    assert np.array_equal(Ta, Tb) and np.array_equal(qa, qb)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_every_step_within_the_oracle_bars(dtype, tol):
    case = inputs.paper_grid_case(37, 29, 8, seed=3, near_singular=True)
    if dtype == "f32":
        case = inputs.round_to_f32(case)
    d = wx.Decomposition(case.nx, case.ny, case.nz, dtype, 3, 2, [0, 1, 20, 37], None)
    d.set_params(case)
    d.load_fields(case.T, case.q, case.U, case.V)
    T, q = case.T, case.q
    for s in range(4):
        d.step(1)
        d.sync()
        Tg, qg = d.read_fields()
        To, qo = oracle.step(case, T, q, case.U, case.V)
        assert np.max(np.abs(Tg - To)) / np.max(np.abs(To)) <= tol
        assert np.max(np.abs(qg - qo)) / np.max(np.abs(qo)) <= tol
        if dtype == "f32":
            Ts, _ = oracle.dynamics(case, T, q, case.U, case.V)
            assert_increments(T, Ts, Tg, To, what=f"decomposed step {s}")
        T, q = Tg, qg
    d.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_combined_sums(dtype):
    """The 2-double reduction of the blocks' sums equals the undecomposed
    run's sums and the FP64 sums of the gathered state (1e-12)."""
    case = inputs.paper_grid_case(60, 44, 58, seed=8)
    if dtype == "f32":
        case = inputs.round_to_f32(case)
    flags = FLAGS | wx.WX_SUMS
    _, _, ma, ea = single(case, dtype, 5, flags)
    (Tb, qb, mb, eb), launches = decomposed(case, dtype, 5, 2, 2, [0, 7, 60], [0, 30, 44], flags)
    assert len(mb) == 5 and launches == 5 * (2 + 4)  # + one sums kernel per block
    assert np.max(np.abs(mb - ma) / np.abs(ma)) <= 1e-12
    assert np.max(np.abs(eb - ea) / np.abs(ea)) <= 1e-12
    w = case.h ** 2 * case.dz[:, None, None]
    assert abs(eb[-1] - np.sum(Tb * w)) / abs(eb[-1]) <= 1e-12
    assert abs(mb[-1] - np.sum(qb * w)) / abs(mb[-1]) <= 1e-12


def test_single_block_is_the_plain_context():
    """px = py = 1: the exchange replaces the step's own periodic copies."""
    case = inputs.round_to_f32(inputs.small_case(40, 30, 8, seed=2))
    Ta, qa, _, _ = single(case, "f32", 5)
    (Tb, qb, _, _), _ = decomposed(case, "f32", 5, 1, 1)
    assert np.array_equal(Ta, Tb) and np.array_equal(qa, qb)


def test_refusals():
    case = inputs.round_to_f32(inputs.paper_grid_case(20, 16, 58, seed=1))
    with pytest.raises(wx.WxError) as e:
        wx.Decomposition(20, 16, 58, "f32", 5, 4)          # 20 blocks > 16
    assert e.value.code == -8
    with pytest.raises(wx.WxError) as e:
        wx.Decomposition(20, 16, 58, "f32", 2, 1, [0, 20, 20])
    assert e.value.code == -1
    d = wx.Decomposition(20, 16, 58, "f32", 2, 2)
    for flags in (FLAGS | wx.WX_RK3, FLAGS | wx.WX_SURROGATE):
        with pytest.raises(wx.WxError) as e:
            d.set_params(case, flags=flags)
        assert e.value.code == -8
    with pytest.raises(wx.WxError) as e:
        d.step(1)                                          # nothing loaded yet
    assert e.value.code == -7
    d.set_params(case)
    d.load_fields(case.T, case.q, case.U, case.V)
    d.step(0)
    d.sync()
    T, q = d.read_fields()
    assert np.array_equal(T, case.T) and np.array_equal(q, case.q)
    d.close()
