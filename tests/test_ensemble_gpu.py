"""Batched ensemble of uneven grids (one persistent launch per step over the
combined member x tile work list, replayed from a CUDA graph) and the
launch-configuration autotuner.

Every column's arithmetic is the same whatever the tile shape and batch, so
each member must equal, bit for bit, the same grid stepped on its own; and
each member is checked against the FP64 oracle at the FP32 tolerance."""
import os

import numpy as np
import pytest

import oracle
from increments import assert_increments
from paper_1802_05839_gb300 import inputs, wx

pytestmark = pytest.mark.gpu

SIZES = [(70, 50, 20), (45, 33, 17), (96, 64, 30), (33, 71, 9)]


def members(sizes, seed0=100):
    cases = []
    for m, (nx, ny, nz) in enumerate(sizes):
        c = inputs.round_to_f32(inputs.ensemble_member(m, nx, ny, nz, seed=seed0 + m))
        cases.append(c)
    return cases


def single(case, n):
    ctx = wx.Context(case.nx, case.ny, case.nz, "f32")
    ctx.set_params(case)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    ctx.step(n)
    ctx.sync()
    out = ctx.read_fields()
    ctx.close()
    return out


@pytest.mark.parametrize("graph", [False, True])
def test_ensemble_equals_single_runs_and_oracle(graph):
    cases = members(SIZES)
    ens = wx.Ensemble([(c.nx, c.ny, c.nz) for c in cases], "f32")
    for mem, c in zip(ens.members, cases):
        mem.set_params(c)
        mem.load_fields(c.T, c.q, c.U, c.V)
    ens.step(3, graph=graph)   # odd: buffer parity flips
    ens.step(2, graph=graph)
    ens.sync()
    for mem, c in zip(ens.members, cases):
        Tg, qg = mem.read_fields()
        Ts, qs = single(c, 5)
        assert np.array_equal(Tg, Ts) and np.array_equal(qg, qs)
        To, qo = oracle.run(c, 5, c.T, c.q, c.U, c.V)
        assert np.max(np.abs(Tg - To)) / np.max(np.abs(To)) <= 1e-5
        assert np.max(np.abs(qg - qo)) / np.max(np.abs(qo)) <= 1e-5
    ens.close()


def test_graph_replay_matches_plain_launches():
    cases = members(SIZES[:3], seed0=7)
    outs = []
    for graph in (False, True):
        ens = wx.Ensemble([(c.nx, c.ny, c.nz) for c in cases], "f32")
        for mem, c in zip(ens.members, cases):
            mem.set_params(c)
            mem.load_fields(c.T, c.q, c.U, c.V)
        for _ in range(3):  # the same captured graph is replayed three times
            ens.step(4, graph=graph)
        ens.sync()
        outs.append([m.read_fields() for m in ens.members])
        ens.close()
    for (Ta, qa), (Tb, qb) in zip(*outs):
        assert np.array_equal(Ta, Tb) and np.array_equal(qa, qb)


def test_ensemble_sums_under_graph_replay():
    cases = members(SIZES[:2], seed0=3)
    ens = wx.Ensemble([(c.nx, c.ny, c.nz) for c in cases], "f32")
    for mem, c in zip(ens.members, cases):
        mem.set_params(c, flags=wx.WX_ADVECTION | wx.WX_PHYSICS | wx.WX_SUMS)
        mem.load_fields(c.T, c.q, c.U, c.V)
    ens.step(2, graph=True)
    ens.step(2, graph=True)
    ens.sync()
    for mem, c in zip(ens.members, cases):
        m, e = mem.sums()
        _, _, mo, eo = oracle.run(c, 4, c.T, c.q, c.U, c.V, sums=True)
        assert len(m) == 4
        assert np.max(np.abs(e - eo) / np.abs(eo)) <= 1e-5
        assert np.max(np.abs(m - mo) / np.abs(mo)) <= 1e-5
    ens.close()


def test_near_singular_members_with_sums_under_graph_replay():
    """FP32 members with near-singular kappa_mult columns (the listing
    variant of the batch, then each member's side solve) and FP64 sums,
    replayed from a graph: each member equals its own context bit for bit,
    sums included, and its sums equal the FP64 sums of its state (1e-12).
    (Ensembles take WX_F32 or WX_F64 members.)"""
    dtype = "f32"
    sizes = [(70, 50, 58), (45, 33, 58), (33, 71, 40)]
    cases = []
    for m, (nx, ny, nz) in enumerate(sizes):
        c = inputs.round_to_f32(inputs.paper_grid_case(nx, ny, nz, seed=40 + m, near_singular=True))
        cases.append(c)
    flags = wx.WX_ADVECTION | wx.WX_PHYSICS | wx.WX_SUMS
    ens = wx.Ensemble([(c.nx, c.ny, c.nz) for c in cases], dtype)
    for mem, c in zip(ens.members, cases):
        mem.set_params(c, flags=flags)
        mem.load_fields(c.T, c.q, c.U, c.V)
    ens.step(3, graph=True)
    ens.step(2, graph=True)
    ens.sync()
    for mem, c in zip(ens.members, cases):
        Tg, qg = mem.read_fields()
        mg, eg = mem.sums()
        ctx = wx.Context(c.nx, c.ny, c.nz, dtype)
        ctx.set_params(c, flags=flags)
        ctx.load_fields(c.T, c.q, c.U, c.V)
        ctx.step(5)
        ctx.sync()
        Ts, qs = ctx.read_fields()
        ms, es = ctx.sums()
        ctx.close()
        assert np.array_equal(Tg, Ts) and np.array_equal(qg, qs)
        assert np.array_equal(mg, ms) and np.array_equal(eg, es)
        w = c.h ** 2 * c.dz[:, None, None]
        assert abs(eg[-1] - np.sum(Tg * w)) / abs(eg[-1]) <= 1e-12
        assert abs(mg[-1] - np.sum(qg * w)) / abs(mg[-1]) <= 1e-12
    ens.close()


def test_ensemble_rejects_mismatched_members():
    cases = members(SIZES[:2])
    ens = wx.Ensemble([(c.nx, c.ny, c.nz) for c in cases], "f32")
    ens.members[0].set_params(cases[0])
    ens.members[1].set_params(cases[1], flags=wx.WX_PHYSICS)  # no advection
    for mem, c in zip(ens.members, cases):
        mem.load_fields(c.T, c.q, c.U, c.V)
    with pytest.raises(wx.WxError) as ei:
        ens.step(1)
    assert ei.value.code == -1
    ens.close()


def test_autotuner_picks_a_config_restores_state_and_caches(tmp_path):
    case = inputs.round_to_f32(inputs.paper_grid_case(300, 200, 40, seed=9))
    ctx = wx.Context(case.nx, case.ny, case.nz, "f32")
    ctx.set_params(case)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    ctx.step(1)
    ctx.sync()
    before = ctx.read_fields()
    cache = str(tmp_path / "tune.txt")
    ms = ctx.tune(cache)
    assert ms > 0
    after = ctx.read_fields()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    cfg = ctx.step_config()
    assert os.path.exists(cache) and len(open(cache).read().splitlines()) == 1
    # a second context finds the entry without timing anything
    ctx2 = wx.Context(case.nx, case.ny, case.nz, "f32")
    ctx2.set_params(case)
    ctx2.load_fields(case.T, case.q, case.U, case.V)
    ctx2.tune(cache)
    assert {k: ctx2.step_config()[k] for k in ("ty", "kb", "stages")} == \
        {k: cfg[k] for k in ("ty", "kb", "stages")}
    assert len(open(cache).read().splitlines()) == 1
    # the tuned configuration still gives the same answer
    ctx.step(2)
    ctx.sync()
    ctx2.step(3)
    ctx2.sync()
    a, b = ctx.read_fields(), ctx2.read_fields()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    ctx.close()
    ctx2.close()


def test_c4_full_size_sampled():
    """The 16-member ensemble at its full sizes (256x256x40 ... 1024x768x58),
    autotuned and replayed from a graph as the bench runs it, one step:
    every member at 400 sampled columns plus its corners against the
    oracle's per-column step (FP32 per-step bound)."""
    sizes = inputs.ensemble_sizes()
    cases = [inputs.round_to_f32(inputs.ensemble_member(m, *s)) for m, s in enumerate(sizes)]
    ens = wx.Ensemble(sizes, "f32")
    for mem, c in zip(ens.members, cases):
        mem.set_params(c)
        mem.load_fields(c.T, c.q, c.U, c.V)
    ens.tune()
    ens.step(1, graph=True)
    ens.sync()
    rng = np.random.default_rng(2)
    for mem, c in zip(ens.members, cases):
        Tg, qg = mem.read_fields()
        ci = np.concatenate([rng.integers(0, c.nx, 400), [0, c.nx - 1, 0, c.nx - 1]])
        cj = np.concatenate([rng.integers(0, c.ny, 400), [0, 0, c.ny - 1, c.ny - 1]])
        To, qo = oracle.step_columns(c, c.T, c.q, c.U, c.V, ci, cj)
        assert np.max(np.abs(Tg[:, cj, ci].T - To)) / np.max(np.abs(c.T)) <= 1e-5
        assert np.max(np.abs(qg[:, cj, ci].T - qo)) / np.max(np.abs(c.q)) <= 1e-5
        dyn = c.copy()
        dyn.physics = False
        Ts, _ = oracle.step_columns(dyn, c.T, c.q, c.U, c.V, ci, cj)
        assert_increments(c.T[:, cj, ci].T, Ts, Tg[:, cj, ci].T, To, what=f"member {c.nx}x{c.ny}x{c.nz}")
    ens.close()
