"""Bookkeeping of the horizontal (IJ) decomposition's depth-1 halo exchange
(the paper's block decomposition of ASUCA, App. F; the exchange is the
communication of its strong-scaling runs, Sec. 5.4), checked on the CPU with
no GPU: the library's plan (wx_dom_halo_plan) says which interior line of
which block fills each ghost strip.  Applied to numpy blocks of a global
periodic field, every ghost column and row must then hold the global
periodic neighbour values, and the corners must stay untouched (the
7-point stencil and the upwind fluxes never read them).  The same plan is
run as a real exchange between two gloo ranks that own alternate blocks."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _wx():
    sys.path.insert(0, ROOT)
    from paper_1802_05839_gb300 import wx
    return wx


def _split(n, parts, given):
    return list(given) if given is not None else [i * n // parts for i in range(parts + 1)]


def _blocks(G, px, py, xs, ys):
    """Block r = iy*px + ix of the global field G [nz][ny][nx] with a NaN
    ghost ring: [nz][ny_r+2][nx_r+2], interior at [1:-1, 1:-1]."""
    out = []
    for iy in range(py):
        for ix in range(px):
            sub = G[:, ys[iy]:ys[iy + 1], xs[ix]:xs[ix + 1]]
            b = np.full((G.shape[0], sub.shape[1] + 2, sub.shape[2] + 2), np.nan)
            b[:, 1:-1, 1:-1] = sub
            out.append(b)
    return out


def _line(b, s, src_side):
    """Interior line s['src_line'] of block b (src_side) or the view of ghost
    line s['dst_line'] (not src_side), over all levels."""
    col = s["dir"] in (0, 1)
    idx = (s["src_line"] if src_side else s["dst_line"]) + 1
    return b[:, 1:-1, idx] if col else b[:, idx, 1:-1]


def _expected_ghosts_ok(G, blocks, px, py, xs, ys):
    nx, ny = G.shape[2], G.shape[1]
    for iy in range(py):
        for ix in range(px):
            b = blocks[iy * px + ix]
            x0, x1, y0, y1 = xs[ix], xs[ix + 1], ys[iy], ys[iy + 1]
            cols = np.arange(x0, x1)
            rows = np.arange(y0, y1)
            assert np.array_equal(b[:, 1:-1, 0], G[:, y0:y1, (x0 - 1) % nx])
            assert np.array_equal(b[:, 1:-1, -1], G[:, y0:y1, x1 % nx])
            assert np.array_equal(b[:, 0, 1:-1], G[:, (y0 - 1) % ny][:, cols])
            assert np.array_equal(b[:, -1, 1:-1], G[:, y1 % ny][:, cols])
            assert np.isnan(b[:, [0, 0, -1, -1], [0, -1, 0, -1]]).all()  # corners untouched
            assert np.array_equal(b[:, 1:-1, 1:-1], G[:, rows][:, :, cols])


CASES = [  # nx, ny, px, py, xsplit, ysplit
    (13, 7, 1, 1, None, None),
    (13, 7, 2, 1, [0, 1, 13], None),        # a one-column block
    (13, 7, 2, 2, [0, 5, 13], [0, 1, 7]),   # a one-row block
    (13, 7, 3, 2, None, None),
    (9, 11, 4, 4, [0, 1, 2, 3, 9], [0, 4, 5, 10, 11]),
    (16, 16, 1, 4, None, None),
]


@pytest.mark.parametrize("nx,ny,px,py,xsplit,ysplit", CASES)
def test_plan_fills_every_ghost_strip_from_its_periodic_neighbour(nx, ny, px, py, xsplit, ysplit):
    wx = _wx()
    xs, ys = _split(nx, px, xsplit), _split(ny, py, ysplit)
    G = np.random.default_rng(0).standard_normal((3, ny, nx))
    blocks = _blocks(G, px, py, xs, ys)
    for r in range(px * py):
        for s in wx.halo_plan(nx, ny, px, py, r, xsplit, ysplit):
            dst = _line(blocks[r], s, False)
            src = _line(blocks[s["src"]], s, True)
            assert dst.shape == src.shape == (3, s["len"])
            dst[...] = src
    _expected_ghosts_ok(G, blocks, px, py, xs, ys)


def test_plan_names_directions_in_order_and_neighbours():
    wx = _wx()
    plan = wx.halo_plan(13, 7, 2, 2, 0, [0, 5, 13], [0, 1, 7])
    assert [s["dir"] for s in plan] == [wx.WX_HALO_WEST, wx.WX_HALO_EAST, wx.WX_HALO_SOUTH, wx.WX_HALO_NORTH]
    # block 0 = columns [0,5) x rows [0,1): west and east both from block 1,
    # south and north both from block 2 (two blocks per direction, periodic)
    assert [s["src"] for s in plan] == [1, 1, 2, 2]
    assert [(s["src_line"], s["dst_line"], s["len"]) for s in plan] == [(7, -1, 1), (0, 5, 1), (5, -1, 5), (0, 1, 5)]


@pytest.mark.parametrize("args", [
    (13, 7, 2, 1, [0, 13, 13], None),   # empty block
    (13, 7, 2, 1, [0, 7, 12], None),    # does not end at nx
    (13, 7, 2, 1, [1, 7, 13], None),    # does not start at 0
    (13, 7, 14, 1, None, None),         # more blocks than columns
    (13, 7, 2, 1, None, None, 2),       # block index out of range
])
def test_plan_refuses_bad_splits(args):
    wx = _wx()
    nx, ny, px, py, xs, ys = args[:6]
    r = args[6] if len(args) > 6 else 0
    with pytest.raises(wx.WxError):
        wx.halo_plan(nx, ny, px, py, r, xs, ys)


# ------------------------------------------------------------ two gloo ranks
def _rank(rank, world, port, q, nx, ny, px, py, xsplit, ysplit):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wx = _wx()
        xs, ys = _split(nx, px, xsplit), _split(ny, py, ysplit)
        G = np.random.default_rng(1).standard_normal((4, ny, nx))  # every rank knows the truth
        blocks = _blocks(G, px, py, xs, ys)
        mine = [r for r in range(px * py) if r % world == rank]
        plans = {r: wx.halo_plan(nx, ny, px, py, r, xsplit, ysplit) for r in range(px * py)}
        for r in range(px * py):  # other ranks' blocks: unknown here
            if r not in mine:
                blocks[r][:] = np.nan
        reqs, recv = [], []
        # send every strip another rank needs from my blocks, receive mine
        for r in range(px * py):
            for s in plans[r]:
                tag = 4 * r + s["dir"]
                owner_dst, owner_src = r % world, s["src"] % world
                if owner_src == rank and owner_dst != rank:
                    buf = torch.from_numpy(np.ascontiguousarray(_line(blocks[s["src"]], s, True)))
                    reqs.append(dist.isend(buf, dst=owner_dst, tag=tag))
                elif owner_dst == rank and owner_src != rank:
                    buf = torch.empty((G.shape[0], s["len"]), dtype=torch.float64)
                    reqs.append(dist.irecv(buf, src=owner_src, tag=tag))
                    recv.append((r, s, buf))
                elif owner_dst == rank:  # both blocks here
                    _line(blocks[r], s, False)[...] = _line(blocks[s["src"]], s, True)
        for rq in reqs:
            rq.wait()
        for r, s, buf in recv:
            _line(blocks[r], s, False)[...] = buf.numpy()
        # check only my blocks
        ok = True
        for r in mine:
            ix, iy = r % px, r // px
            b = blocks[r]
            x0, x1, y0, y1 = xs[ix], xs[ix + 1], ys[iy], ys[iy + 1]
            ok = ok and np.array_equal(b[:, 1:-1, 0], G[:, y0:y1, (x0 - 1) % nx])
            ok = ok and np.array_equal(b[:, 1:-1, -1], G[:, y0:y1, x1 % nx])
            ok = ok and np.array_equal(b[:, 0, 1:-1], G[:, (y0 - 1) % ny, x0:x1])
            ok = ok and np.array_equal(b[:, -1, 1:-1], G[:, y1 % ny, x0:x1])
            ok = ok and bool(np.isnan(b[:, [0, 0, -1, -1], [0, -1, 0, -1]]).all())
        q.put((rank, ok, len(mine), len(recv)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("nx,ny,px,py,xsplit,ysplit", [(13, 7, 2, 2, [0, 5, 13], [0, 1, 7]),
                                                      (12, 9, 3, 1, [0, 1, 2, 12], None)])
def test_two_gloo_ranks_exchange_strips_by_the_plan(nx, ny, px, py, xsplit, ysplit):
    world, port = 2, 29631 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q, nx, ny, px, py, xsplit, ysplit))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    assert all(ok for _, ok, _, _ in got)
    assert all(n > 0 for _, _, _, n in got)  # strips really crossed between the ranks
