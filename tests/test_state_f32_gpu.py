"""The FP32 state entry points (wx_load_state_f32 / wx_read_state_f32): they
move T and q in the context's storage precision, so they must round-trip
bit for bit, agree with the FP64 entry points on FP32-representable values,
and leave the step's result unchanged."""
import numpy as np
import pytest
import torch

from paper_1802_05839_gb300 import inputs, wx

pytestmark = pytest.mark.gpu


def f32(a):
    return np.ascontiguousarray(a, np.float32)


@pytest.mark.parametrize("dtype", ["f32", "mixed"])
@pytest.mark.parametrize("shape", [(37, 29, 8), (1, 1, 1), (130, 3, 17)])
def test_round_trip_is_bitwise(dtype, shape):
    nx, ny, nz = shape
    case = inputs.small_case(nx=nx, ny=ny, nz=nz, seed=7)
    ctx = wx.Context(nx, ny, nz, dtype)
    ctx.set_params(case)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    T, q = ctx.read_state_f32()
    assert np.array_equal(T, f32(case.T)) and np.array_equal(q, f32(case.q))
    T2 = f32(case.T) * np.float32(1.001)
    q2 = f32(case.q)[::-1].copy()
    ctx.load_state_f32(T2, q2)
    Tg, qg = ctx.read_state_f32()
    assert np.array_equal(Tg, T2) and np.array_equal(qg, q2)
    # the FP64 read sees the same values
    Td, qd = ctx.read_fields()
    assert np.array_equal(Td, T2.astype(np.float64)) and np.array_equal(qd, q2.astype(np.float64))
    ctx.close()


@pytest.mark.parametrize("dtype", ["f32", "mixed"])
@pytest.mark.parametrize("src", ["host", "device"])
def test_step_after_state_load_equals_step_after_fields_load(dtype, src):
    """Three steps from load_state_f32 equal three steps from load_fields of
    the same FP32 values, bit for bit (the ghost ring is rebuilt by the load)."""
    case = inputs.round_to_f32(inputs.small_case(nx=96, ny=40, nz=12, seed=9))
    a = wx.Context(case.nx, case.ny, case.nz, dtype)
    a.set_params(case)
    a.load_fields(case.T, case.q, case.U, case.V)
    a.step(3)
    a.sync()
    want = a.read_state_f32()
    b = wx.Context(case.nx, case.ny, case.nz, dtype)
    b.set_params(case)
    b.load_fields(np.zeros_like(case.T), np.zeros_like(case.q), case.U, case.V)
    b.step(2)          # a different state first: load_state_f32 must replace it
    b.sync()
    T, q = f32(case.T), f32(case.q)
    if src == "device":
        T, q = torch.from_numpy(T).cuda(), torch.from_numpy(q).cuda()
        torch.cuda.synchronize()
    b.load_state_f32(T, q)
    b.step(3)
    b.sync()
    got = b.read_state_f32()
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    a.close()
    b.close()


def test_status_paths():
    case = inputs.small_case(nx=16, ny=8, nz=4, seed=3)
    c64 = wx.Context(16, 8, 4, "f64")
    c64.set_params(case)
    c64.load_fields(case.T, case.q, case.U, case.V)
    with pytest.raises(wx.WxError) as e:
        c64.load_state_f32(f32(case.T), f32(case.q))
    assert e.value.code == -8
    with pytest.raises(wx.WxError) as e:
        c64.read_state_f32()
    assert e.value.code == -8
    c64.close()
    c32 = wx.Context(16, 8, 4, "f32")
    c32.set_params(case)
    with pytest.raises(wx.WxError) as e:
        c32.load_state_f32(f32(case.T), f32(case.q))   # no winds yet
    assert e.value.code == -7
    with pytest.raises(wx.WxError) as e:
        c32.read_state_f32()
    assert e.value.code == -7
    c32.close()


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("dtype", ["f64", "f32", "mixed"])
def test_pinned_host_arrays_give_the_same_state_as_pageable_ones(dtype):
    """Pinned (cudaHostAlloc) and pageable host arrays give the same state
    bit for bit through both the FP64 and the FP32 entry points."""
    case = inputs.small_case(nx=70, ny=33, nz=9, seed=11)
    if dtype != "f64":
        case = inputs.round_to_f32(case)
    res = []
    for pin in (False, True):
        conv = _pinned if pin else (lambda a: np.ascontiguousarray(a))
        ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
        ctx.set_params(case)
        ctx.load_fields(conv(case.T), conv(case.q), conv(case.U), conv(case.V))
        ctx.step(2)
        ctx.sync()
        shape = (case.nz, case.ny, case.nx)
        out = ctx.read_fields(conv(np.empty(shape)), conv(np.empty(shape)))
        if dtype != "f64":
            ctx.load_state_f32(conv(f32(out[0])), conv(f32(out[1])))
            ctx.step(1)
            ctx.sync()
            out = out + ctx.read_state_f32(conv(np.empty(shape, np.float32)), conv(np.empty(shape, np.float32)))
        res.append(out)
        ctx.close()
    for x, y in zip(*res):
        assert np.array_equal(x, y)


def test_binding_refuses_mistyped_or_short_arrays():
    """Wrong dtypes, short buffers and host/device mixes are refused by the
    binding before any pointer reaches the library; the context stays usable."""
    case = inputs.small_case(nx=16, ny=8, nz=4, seed=3)
    ctx = wx.Context(16, 8, 4, "f32")
    ctx.set_params(case)
    n = 16 * 8 * 4
    d32 = torch.zeros(n, dtype=torch.float32, device="cuda")
    d64 = torch.zeros(n, dtype=torch.float64, device="cuda")
    U = torch.from_numpy(np.ascontiguousarray(case.U)).cuda()
    with pytest.raises(TypeError):
        ctx.load_fields(d32, d32, U, U)                   # FP32 into the FP64 call
    with pytest.raises(TypeError):
        ctx.load_fields(d64, d64, case.U, case.V)         # device fields, host winds
    with pytest.raises(ValueError):
        ctx.load_fields(case.T[:, :, :-1], case.q, case.U, case.V)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    with pytest.raises(ValueError):
        ctx.load_state_f32(d32[:-1], d32[:-1])
    with pytest.raises(TypeError):
        ctx.read_state_f32(np.empty(n, np.float64), np.empty(n, np.float64))
    with pytest.raises(ValueError):
        ctx.read_fields_into(d64[:-1], d64)
    T, q = ctx.read_state_f32()
    assert np.array_equal(T, f32(case.T))
    ctx.close()
    app = wx.ReducedApp(8, 6, 4, "f64")
    with pytest.raises(ValueError):
        app.load(np.zeros((4, 6, 8)))                     # missing the ghost ring
    app.close()


def test_async_transfers_match_the_synchronous_ones():
    """Enqueued upload, step and download on a stream give the bits of the
    synchronous calls; pageable host arrays are refused."""
    case = inputs.round_to_f32(inputs.small_case(nx=70, ny=33, nz=9, seed=15))
    T32, q32 = _pinned(f32(case.T) * np.float32(1.01)), _pinned(f32(case.q))
    shape = (case.nz, case.ny, case.nx)
    a = wx.Context(case.nx, case.ny, case.nz, "f32")
    a.set_params(case)
    a.load_fields(case.T, case.q, case.U, case.V)
    a.load_state_f32(T32, q32)
    a.step(2)
    a.sync()
    want = a.read_state_f32()
    a.close()
    b = wx.Context(case.nx, case.ny, case.nz, "f32")
    b.set_params(case)
    b.load_fields(case.T, case.q, case.U, case.V)
    s = torch.cuda.Stream()
    oT, oq = _pinned(np.zeros(shape, np.float32)), _pinned(np.zeros(shape, np.float32))
    b.load_state_f32_async(T32, q32, stream=s)
    b.step(2, stream=s)
    b.read_state_f32_async(oT, oq, stream=s)
    s.synchronize()
    assert np.array_equal(oT, want[0]) and np.array_equal(oq, want[1])
    with pytest.raises(wx.WxError) as e:
        b.load_state_f32_async(np.ascontiguousarray(T32.copy()), q32, stream=s)
    assert e.value.code == -1
    with pytest.raises(wx.WxError) as e:
        b.read_state_f32_async(np.zeros(shape, np.float32), oq, stream=s)
    assert e.value.code == -1
    b.close()


def test_two_contexts_pipelined_on_two_streams():
    """Independent states pushed through two contexts on two streams,
    alternating, all enqueued before one synchronize: every result equals
    the synchronous single-context step of its own input."""
    case = inputs.round_to_f32(inputs.small_case(nx=64, ny=40, nz=12, seed=16))
    shape = (case.nz, case.ny, case.nx)
    ins = [(_pinned(f32(case.T) + np.float32(i)), _pinned(f32(case.q) * np.float32(1 + 0.1 * i))) for i in range(6)]
    outs = [(_pinned(np.zeros(shape, np.float32)), _pinned(np.zeros(shape, np.float32))) for _ in range(6)]
    ctxs, streams = [], [torch.cuda.Stream(), torch.cuda.Stream()]
    for _ in range(2):
        c = wx.Context(case.nx, case.ny, case.nz, "f32")
        c.set_params(case)
        c.load_fields(case.T, case.q, case.U, case.V)
        ctxs.append(c)
    for it in range(6):
        c, s = ctxs[it % 2], streams[it % 2]
        c.load_state_f32_async(*ins[it], stream=s)
        c.step(1, stream=s)
        c.read_state_f32_async(*outs[it], stream=s)
    for s in streams:
        s.synchronize()
    ref = ctxs[0]
    for it in range(6):
        ref.load_state_f32(*ins[it])
        ref.step(1)
        ref.sync()
        T, q = ref.read_state_f32()
        assert np.array_equal(outs[it][0], T) and np.array_equal(outs[it][1], q)
    for c in ctxs:
        c.close()
