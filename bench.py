"""Benchmark of the fused weather step on GB300.

Default workload: the paper's grid 1581 x 1301 x 58 (Sec. 5.4), FP32 fields,
dynamics + column physics, seeded synthetic state (the paper's JMA inputs are
not public).  One step = one pass of the whole hot path over the grid.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0.  `value` is whole-job cell-steps/s timed with
CUDA events on the launching stream (inputs resident in HBM; the two 955 MB
field buffers exceed the 129 MB L2, so no flush is needed); `e2e` is the same
metric through the C ABI with host buffers (load + step + read back every
step); `roofline` relates the step kernel's algorithmic bytes to the measured
HBM copy bandwidth; `cpu_baseline` times the FP64 CPU oracle on a bounded
sample of the same workload on this host's cores.  `variants` holds the
other measured configurations of the same hot path: the FP64 step, the
mixed-precision step with FP64 sums, the 16-member ensemble replayed from a
CUDA graph, the residual-checked MLP-surrogate step (network trained in this
run by the library's kernels) against the plain step, and the paper's own
reduced weather application on its three grids beside the paper's timings.

  python bench.py --only f64|mixed|ensemble|surrogate|reduced_app|ablation|rk3|decomposed [--nx --ny]   one variant
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CELL_BYTES = {"f32": 16, "f64": 32, "mixed": 16}  # read + write of (T, q) per cell
COL_BYTES = {"f32": 8, "f64": 16, "mixed": 12}     # U, V (+ kappa_mult) per column


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_case(dtype, nx=1581, ny=1301, nz=58):
    from paper_1802_05839_gb300 import inputs
    case = inputs.paper_grid_case(nx, ny, nz, near_singular=(dtype == "mixed"))
    return inputs.round_to_f32(case) if dtype in ("f32", "mixed") else case


def traffic_record(dtype):
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, or None when the kernel source changed since the capture."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    src = os.path.join(ROOT, "paper_1802_05839_gb300", "csrc", "wx_step.cu")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(dtype)
    if not rec:
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return rec["traffic_bytes_per_launch"] if rec.get("wx_step_cu_sha256") == sha else None


def cpu_baseline(case, budget_s=12.0):
    """The FP64 oracle's step on a bounded sample of columns (every 10th in
    raster order) of the same workload, repeated until ~budget_s of CPU work."""
    import oracle
    cols = np.arange(0, case.nx * case.ny, 10)
    ci, cj = (cols % case.nx).astype(np.int32), (cols // case.nx).astype(np.int32)
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.step_columns(case, case.T, case.q, case.U, case.V, ci, cj)
        done += 1
        el = time.perf_counter() - t0
        if el > budget_s:
            break
    return {"value": done * len(cols) * case.nz / el, "unit": "cell-steps/s",
            "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{done} x oracle step on {len(cols)} of {case.nx * case.ny} columns "
                      f"(every 10th) of the {case.nx}x{case.ny}x{case.nz} FP64 workload, "
                      f"{el:.1f} s"}


def run_reference(args):
    """--impl reference: the FP64 CPU oracle, as it stands, on this host's
    cores; each step a bounded sample (every 50th column) of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    case = make_case("f64")
    cols = np.arange(0, case.nx * case.ny, 50)
    ci, cj = (cols % case.nx).astype(np.int32), (cols // case.nx).astype(np.int32)
    for _ in range(args.warmup):
        oracle.step_columns(case, case.T, case.q, case.U, case.V, ci, cj)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.step_columns(case, case.T, case.q, case.U, case.V, ci, cj)
        times.append(time.perf_counter() - t0)
    per = sum(times) / len(times)
    value = len(cols) * case.nz / per
    sample = (f"oracle step on {len(cols)} of {case.nx * case.ny} columns (every 50th) of the "
              f"{case.nx}x{case.ny}x{case.nz} workload per step")
    print(json.dumps({
        "impl": "reference", "metric": args.metric, "value": value, "unit": "cell-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"paper grid {case.nx}x{case.ny}x{case.nz}, dynamics + physics",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": oracle.threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def e2e_measure(case, dtype, iters=5, n_ctx=3):
    """Load (H2D from pinned host) + one step + read back (D2H) per step;
    the median over `iters` steps (host-side copies on a shared host vary
    from one iteration to the next), the mean beside it.

    FP32-storage contexts move the state (T, q) in FP32, the prescribed
    winds (constant in time) loaded once beforehand.  The reported figure is
    pipelined: n_ctx contexts on n_ctx streams take steps in turn through the
    enqueued calls (wx_load_state_f32_async / wx_read_state_f32_async), so
    downloads overlap uploads; the synchronous one-context figure is kept
    under `sync_single_context`, and the FP64 calls (wx_load_fields with the
    winds, wx_read_fields) under `fp64_api`."""
    import torch
    from paper_1802_05839_gb300 import wx
    pin = lambda a, t=np.float64: torch.from_numpy(np.ascontiguousarray(a, t)).pin_memory().numpy()
    T, q, U, V = pin(case.T), pin(case.q), pin(case.U), pin(case.V)
    To = torch.empty(T.shape, dtype=torch.float64).pin_memory().numpy()
    qo = torch.empty(T.shape, dtype=torch.float64).pin_memory().numpy()
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    ctx.set_params(case)
    ctx.load_fields(T, q, U, V)
    ctx.step(1)
    ctx.sync()
    ctx.read_fields()
    lib = wx.lib()

    def timed(one_step):
        times = []
        for _ in range(iters):
            t0 = time.perf_counter()
            one_step()
            times.append(time.perf_counter() - t0)
        return statistics.median(times), statistics.mean(times)

    def step64():
        ctx.load_fields(T, q, U, V)
        ctx.step(1)
        ctx.sync()
        wx._check(lib.wx_read_fields(ctx.ptr, wx._dptr(To), wx._dptr(qo)), ctx.ptr)

    el64, mean64 = timed(step64)
    rec64 = {"value": case.cells / el64, "unit": "cell-steps/s",
             "h2d_bytes_per_step": int(T.nbytes + q.nbytes + U.nbytes + V.nbytes),
             "d2h_bytes_per_step": int(To.nbytes + qo.nbytes), "ms_per_step": el64 * 1e3,
             "ms_per_step_mean": mean64 * 1e3, "iterations": iters,
             "path": "wx_load_fields(host) + wx_step(1) + wx_read_fields(host), median step"}
    if dtype == "f64":
        ctx.close()
        return rec64
    T32, q32 = pin(case.T, np.float32), pin(case.q, np.float32)
    To32 = torch.empty(T.shape, dtype=torch.float32).pin_memory().numpy()
    qo32 = torch.empty(T.shape, dtype=torch.float32).pin_memory().numpy()

    def step32():
        wx._check(lib.wx_load_state_f32(ctx.ptr, wx._dptr(T32), wx._dptr(q32), 0), ctx.ptr)
        ctx.step(1)
        ctx.sync()
        wx._check(lib.wx_read_state_f32(ctx.ptr, wx._dptr(To32), wx._dptr(qo32)), ctx.ptr)

    el, mean = timed(step32)
    rec_sync = {"value": case.cells / el, "unit": "cell-steps/s",
                "h2d_bytes_per_step": int(T32.nbytes + q32.nbytes),
                "d2h_bytes_per_step": int(To32.nbytes + qo32.nbytes), "ms_per_step": el * 1e3,
                "ms_per_step_mean": mean * 1e3, "iterations": iters,
                "path": "one context, synchronous: wx_load_state_f32(host T, q) + wx_step(1) + "
                        "wx_read_state_f32(host), median step"}

    # Pipelined: n_ctx contexts on n_ctx streams take steps in turn, every
    # transfer enqueued (pinned host arrays), so one context's download
    # overlaps another's upload on the link's two copy engines.
    ctxs, streams, outs = [ctx], [torch.cuda.Stream()], [(To32, qo32)]
    for _ in range(n_ctx - 1):
        cx = wx.Context(case.nx, case.ny, case.nz, dtype)
        cx.set_params(case)
        cx.load_fields(T, q, U, V)
        ctxs.append(cx)
        streams.append(torch.cuda.Stream())
        outs.append((torch.empty(T.shape, dtype=torch.float32).pin_memory().numpy(),
                     torch.empty(T.shape, dtype=torch.float32).pin_memory().numpy()))

    def pipelined(n):
        for it in range(n):
            c, st = ctxs[it % n_ctx], streams[it % n_ctx]
            c.load_state_f32_async(T32, q32, stream=st)
            c.step(1, stream=st)
            c.read_state_f32_async(*outs[it % n_ctx], stream=st)
        for st in streams:
            st.synchronize()

    pipelined(4)
    n_pipe, rounds = 4 * iters, []
    for _ in range(5):  # a shared host's copy engines vary from round to round: the median of 5
        t0 = time.perf_counter()
        pipelined(n_pipe)
        rounds.append((time.perf_counter() - t0) / n_pipe)
    el_p = statistics.median(rounds)
    for c in ctxs:
        c.close()
    return {"value": case.cells / el_p, "unit": "cell-steps/s",
            "h2d_bytes_per_step": int(T32.nbytes + q32.nbytes),
            "d2h_bytes_per_step": int(To32.nbytes + qo32.nbytes), "ms_per_step": el_p * 1e3,
            "iterations": n_pipe, "ms_per_step_rounds": [r * 1e3 for r in rounds],
            "path": f"{n_ctx} contexts on {n_ctx} streams take steps in turn: wx_load_state_f32_async(pinned "
                    f"host T, q) + wx_step(1) + wx_read_state_f32_async(pinned host) each step, all "
                    f"enqueued; median of 5 rounds of {n_pipe} steps, each timed from the first call to "
                    f"the last stream synchronize; "
                    f"winds (constant in time) loaded once per context by wx_load_fields before timing",
            "sync_single_context": rec_sync, "fp64_api": rec64}


# ---------------------------------------------------------------- replicas
# With N GPUs the bench runs N independent replicas of the workload (the
# step has no exchange between GPUs: one grid per GPU).  The job's time is
# the slowest rank's; the job's throughput counts every rank's cells.
def max_over_ranks(ms, device="cuda"):
    """The largest of every rank's `ms` (all ranks receive it)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, cells_per_rank, ms_per_step):
    """Whole-job cell-steps/s of `world` replicas, each stepping
    `cells_per_rank` cells, timed by the slowest rank."""
    return world * cells_per_rank / (ms_per_step * 1e-3)


def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def _time_steps(step, n, stream, warmup=3):
    """Mean ms per call of step() over n calls after `warmup`, CUDA events on
    `stream` with a synchronize on both sides."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    torch.cuda.nvtx.range_push("timed")   # ncu --nvtx --nvtx-include timed/
    e0.record(stream)
    for _ in range(n):
        step()
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def variant_plain(dtype, steps, nx=1581, ny=1301, nz=58):
    """FP64 (C2) or mixed precision with FP64 sums (C3) at the paper grid."""
    import torch
    from paper_1802_05839_gb300 import wx
    case = make_case(dtype, nx, ny, nz)
    ctx = wx.Context(nx, ny, nz, dtype)
    flags = wx.WX_ADVECTION | wx.WX_PHYSICS | (wx.WX_SUMS if dtype == "mixed" else 0)
    ctx.set_params(case, flags=flags)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    st = torch.cuda.Stream()
    ms = _time_steps(lambda: ctx.step(1, stream=st), steps, st)
    ctx.sync()
    out = {"ms_per_step": ms, "value": case.cells / (ms * 1e-3), "unit": "cell-steps/s", "steps": steps,
           "workload": f"paper grid {nx}x{ny}x{nz} ({dtype})", "gpu_launches_per_step": ctx.last_launches()}
    peak, kind = peaks()
    alg = case.cells * CELL_BYTES[dtype] + nx * ny * COL_BYTES[dtype]
    out["hbm_frac"] = alg / (ms * 1e-3) / 1e9 / peak
    if dtype == "mixed":
        out["flagged_fp64_columns"] = ctx.flagged_columns()
        out["sums_recorded"] = len(ctx.sums()[0])
    if dtype == "f64":
        out["bound"] = ("fp64 pipe (one exp2 and about 25 explicit FP64 operations per cell, "
                        "reciprocals from the level tables; GB300 FP64 rate)")
    ctx.close()
    return out


def variant_decomposed(steps, nx=1581, ny=1301, nz=58, layouts=((2, 2), (4, 4)), plain_ms=None):
    """The paper grid split into px x py blocks (simulated ranks on one GPU):
    per step one step-kernel launch over all blocks, then one halo exchange
    launch that copies every block's edge lines into its neighbours' ghost
    lines; the algorithmic bytes add those halo strips (read + written) to
    the step's."""
    import torch
    from paper_1802_05839_gb300 import wx
    case = make_case("f32", nx, ny, nz)
    peak, _ = peaks()
    out = {"workload": f"paper grid {nx}x{ny}x{nz} (f32) in px x py blocks, depth-1 halo exchange"}
    for px, py in layouts:
        d = wx.Decomposition(nx, ny, nz, "f32", px, py)
        d.set_params(case)
        d.load_fields(case.T, case.q, case.U, case.V)
        st = torch.cuda.Stream()
        ms = _time_steps(lambda: d.step(1, stream=st), steps, st)
        d.sync()
        halo_cells = 2 * nz * 2 * (ny * px + nx * py)   # both fields, 4 strips per block
        alg = case.cells * CELL_BYTES["f32"] + nx * ny * COL_BYTES["f32"] + halo_cells * 2 * 4
        rec = {"ms_per_step": ms, "value": case.cells / (ms * 1e-3), "unit": "cell-steps/s",
               "steps": steps, "blocks": px * py, "gpu_launches_per_step": d.last_launches(),
               "halo_bytes_per_step": halo_cells * 2 * 4, "hbm_frac": alg / (ms * 1e-3) / 1e9 / peak}
        if plain_ms:
            rec["vs_plain_step"] = ms / plain_ms
        out[f"{px}x{py}"] = rec
        d.close()
    return out


def variant_ensemble(steps):
    """16 uneven members (C4), one persistent launch per step, graph-replayed."""
    import torch
    from paper_1802_05839_gb300 import inputs, wx
    sizes = inputs.ensemble_sizes()
    ens = wx.Ensemble(sizes, "f32")
    cells = 0
    for m, (mem, (nx, ny, nz)) in enumerate(zip(ens.members, sizes)):
        c = inputs.round_to_f32(inputs.ensemble_member(m, nx, ny, nz))
        mem.set_params(c)
        mem.load_fields(c.T, c.q, c.U, c.V)
        cells += nx * ny * nz
    st = torch.cuda.Stream()
    tuned_ms = ens.tune(stream=st)
    ens.step(steps, graph=True, stream=st)   # capture + warm-up replay
    ens.sync()
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    torch.cuda.nvtx.range_push("timed")   # ncu --nvtx --nvtx-include timed/
    e0.record(st)
    ens.step(steps, graph=True, stream=st)
    e1.record(st)
    torch.cuda.nvtx.range_pop()
    ens.sync()
    ms = e0.elapsed_time(e1) / steps
    peak, _ = peaks()
    alg = sum(nx * ny * nz * CELL_BYTES["f32"] + nx * ny * COL_BYTES["f32"] for nx, ny, nz in sizes)
    # the (member, tile) work list of one launch: tiles per member, the
    # persistent CTAs walking it and how full their last round is, counted
    # in tiles and in tile-levels (a tile's cost goes with its depth)
    cfg = ens.step_config()
    ty, ctas = cfg["ty"], torch.cuda.get_device_properties(0).multi_processor_count * cfg["ctas_per_sm"]
    tiles = [-(-nx // 64) * -(-ny // ty) for nx, ny, _ in sizes]
    levels = [t * nz for t, (_, _, nz) in zip(tiles, sizes)]
    rounds = -(-sum(tiles) // ctas)
    work = {"order": "members by size (cells) descending", "ctas": ctas,
            "tiles_per_member": tiles, "nz_per_member": [nz for _, _, nz in sizes], "tiles": sum(tiles),
            "rounds": rounds, "last_round_fill": (sum(tiles) - (rounds - 1) * ctas) / ctas, "tile_levels": sum(levels)}
    # utilisation in tile-levels: the work over CTAs x the busiest CTA's share
    order = sorted(range(len(sizes)), key=lambda m: -sizes[m][0] * sizes[m][1] * sizes[m][2])
    per_cta = [0] * ctas
    w = 0
    for m in order:
        for _ in range(tiles[m]):
            per_cta[w % ctas] += sizes[m][2]
            w += 1
    work["tile_level_utilisation"] = sum(levels) / (ctas * max(per_cta))
    out = {"ms_per_step": ms, "value": cells / (ms * 1e-3), "unit": "cell-steps/s (all members)",
           "steps": steps, "members": len(sizes), "cells": cells, "hbm_frac": alg / (ms * 1e-3) / 1e9 / peak,
           "graph": True, "tuned_config": cfg, "tune_ms": tuned_ms, "work_list": work,
           "gpu_launches_per_step": ens.last_launches() / steps}
    ens.close()
    return out


def variant_surrogate(steps, nx=1581, ny=1301, plain_ms=None, train_epochs=32):
    """C5: train the MLP on 2M columns with the library's kernels, then step
    the paper grid with the residual-checked surrogate."""
    import torch
    from paper_1802_05839_gb300 import inputs, surrogate as S, wx
    t0 = time.perf_counter()
    # train_epochs = 0: an untrained network (kernel timing and profiling only)
    Ts, qs, km, tend = S.dataset(range(1, 9), 512, 512) if train_epochs else S.dataset([1], 128, 128)
    net = wx.MLP(4096)
    Ws, bs = inputs.mlp_init(2024)
    net.set_weights(Ws, bs)
    S.set_levels_from_case(net, inputs.paper_grid_case(8, 8, 58, seed=1, config_seed=S.CONFIG_SEED))
    net.fit_norm(Ts, qs, km, tend)
    X, Yt = S.rows(net, Ts, qs, km, tend)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = S.train(net, X, Yt, Ts.shape[0], epochs=train_epochs, batch=4096, lr0=2e-3, seed=0) \
        if train_epochs else [float("nan")]
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    n_train = Ts.shape[0]
    del X, Yt, Ts, qs, km, tend
    val = S.dataset([101], 256, 256)
    err = S.tendency_error(net, *val)
    del val
    case = make_case("f32", nx, ny, 58)
    ctx = wx.Context(nx, ny, 58, "f32")
    ctx.set_params(case, flags=wx.WX_ADVECTION | wx.WX_PHYSICS | wx.WX_SURROGATE)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    ctx.set_surrogate(net, 2e-2)
    st = torch.cuda.Stream()
    ms = _time_steps(lambda: ctx.step(1, stream=st), steps, st)
    torch.cuda.nvtx.range_push("surrogate_step")
    ctx.step(1, stream=st)
    torch.cuda.nvtx.range_pop()
    ctx.sync()
    fb = ctx.surrogate_fallbacks()
    launches = ctx.last_launches()
    # the fallback fraction along a run from the initial state
    ctx.load_fields(case.T, case.q, case.U, case.V)
    fb_at, done = {}, 0
    for mark in (1, 50, 100):
        ctx.step(mark - done, stream=st)
        done = mark
        ctx.sync()
        fb_at[str(mark)] = ctx.surrogate_fallbacks() / (nx * ny)
    # the acceptance policy: exact fused steps while the network is declined,
    # a probe of 16 rows every 8 steps
    ctx.load_fields(case.T, case.q, case.U, case.V)
    ctx.set_surrogate_policy(0.5, probe_every=8, probe_rows=16)
    pol_ms = _time_steps(lambda: ctx.step(1, stream=st), steps, st)  # after its first decision
    ctx.sync()
    pol_launches = ctx.last_launches()
    ctx.close()
    # the network alone on every column of the grid (tensor-core roofline)
    rows = (nx * ny + 127) // 128 * 128
    Xf = torch.zeros(rows, wx.MLP_X_WIDTH, dtype=torch.bfloat16, device="cuda")
    Yf = torch.empty(rows, wx.MLP_OUT_PAD, dtype=torch.float32, device="cuda")
    big = wx.MLP(rows)
    big.set_weights(*net.get_weights())
    fwd_ms = _time_steps(lambda: big.forward(Xf, Yf, stream=st), 5, st)
    big.close()
    net.close()
    flop_col = 2 * (512 * 512 + 2 * 512 * 512 + 512 * 128)   # padded GEMM shapes actually run
    flop_alg = 2 * (232 * 512 + 2 * 512 * 512 + 512 * 116)   # the network's own
    tflops = nx * ny * flop_col / (fwd_ms * 1e-3) / 1e12
    tpk = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0
    out = {"ms_per_step": ms, "value": nx * ny * 58 / (ms * 1e-3), "unit": "cell-steps/s",
           "steps": steps, "workload": f"paper grid {nx}x{ny}x58, surrogate physics, fallback tol 2e-2",
           "fallback_columns_last_step": fb, "fallback_frac": fb / (nx * ny),
           "val_tendency_rel_l2": {"all": err[0], "heating": err[1], "vdiff": err[2]},
           "train": {"columns": n_train, "epochs": train_epochs, "batch": 4096, "loss_first": hist[0],
                     "loss_last": hist[-1], "seconds": t2 - t1, "setup_seconds": t1 - t0},
           "network_forward": {"ms": fwd_ms, "tflops": tflops, "peak_tflops": tpk, "frac": tflops / tpk,
                               "flop_per_column_run": flop_col, "flop_per_column_alg": flop_alg},
           "gpu_launches_per_step": launches,
           "fallback_frac_at": fb_at,
           "policy": {"min_accept": 0.5, "probe_every": 8, "probe_rows": 16, "ms_per_step": pol_ms,
                      "steps": steps, "gpu_launches_last_step": pol_launches,
                      "path": "wx_set_surrogate_policy: network steps while acceptance >= 0.5, else the fused "
                              "exact step with a 16-row network probe every 8 steps; timed after 3 warm-up "
                              "steps (the first two steps run the network before the first decision)"}}
    if plain_ms:
        out["vs_plain_step"] = ms / plain_ms
        out["policy"]["vs_plain_step"] = pol_ms / plain_ms
    return out


# The paper's own timings of its reduced weather application, 100 steps,
# FP64 (Sec. 5.1, block-size and performance tables): Tesla K20x with the
# Hybrid Fortran default 32 x 16 blocks, and a 6-core Xeon X5670.
PAPER_REDUCED_S = {(128, 128, 128): {"k20x_s": 0.10, "x5670_6core_s": 0.40},
                   (256, 256, 256): {"k20x_s": 0.55, "x5670_6core_s": 4.25},
                   (256, 256, 512): {"k20x_s": 2.16}}


def variant_reduced_app(steps=100):
    """The paper's reduced application (wx_pf_*) on its three grids, 100
    steps from the 300 K box state; device-resident time and the time with
    the state copied in and out (the paper's GPU times include the copies)."""
    import torch
    from paper_1802_05839_gb300 import inputs, wx
    out = {}
    for (nx, ny, nz), ref in PAPER_REDUCED_S.items():
        E = inputs.paper_box_state(nx, ny, nz)
        rec = {"paper": ref}
        for dtype in ("f64", "f32"):
            app = wx.ReducedApp(nx, ny, nz, dtype)
            app.set_params()
            app.load(E)
            st = torch.cuda.Stream()
            ms = _time_steps(lambda: app.step(steps, stream=st), 1, st) / steps
            app.sync()
            t0 = time.perf_counter()
            app.load(E)
            app.step(steps, stream=st)
            app.sync()
            app.read()
            e2e_s = time.perf_counter() - t0
            app.close()
            cells = nx * ny * nz
            r = {"ms_per_step": ms, "value": cells / (ms * 1e-3), "unit": "cell-steps/s",
                 "s_per_100_steps_device": ms * 0.1, "s_per_100_steps_with_copies": e2e_s,
                 "hbm_frac": cells * (16 if dtype == "f64" else 8) / (ms * 1e-3) / 1e9 / peaks()[0]}
            if dtype == "f64":
                r["vs_paper_k20x"] = ref["k20x_s"] / e2e_s
            rec[dtype] = r
        out[f"{nx}x{ny}x{nz}"] = rec
    return out


# The paper's storage-order (128^3, Sec. 5.1.1) and block-size (Sec. 5.1.4)
# tables, 100 steps, FP64.
PAPER_ORDER_S = {"ijk": {"k20x_openacc_s": 0.10, "x5670_1core_s": 1.73},
                 "kij": {"k20x_openacc_s": 0.77, "x5670_1core_s": 1.28}}
PAPER_BLOCK_S = {"128x1": {"128": 0.095, "256": 0.63, "256x512": 2.99},
                 "32x16": {"128": 0.10, "256": 0.55, "256x512": 2.16}}


def variant_ablation(steps=100):
    """The paper's storage-order and block-size experiments on GB300: the
    reduced application (box state, 100 steps, device-resident) in IJK and
    KIJ order at 128^3 and 256^3, and four block shapes in IJK order on the
    three grids; FP64 as in the paper (FP64-ALU-bound here) and FP32
    (memory-bound)."""
    import torch
    from paper_1802_05839_gb300 import inputs, wx
    st = torch.cuda.Stream()

    def run(nx, ny, nz, layout, block, dtype):
        app = wx.ReducedApp(nx, ny, nz, dtype)
        app.set_params()
        app.set_launch(layout, block)
        app.load(inputs.paper_box_state(nx, ny, nz))
        ms = _time_steps(lambda: app.step(steps, stream=st), 1, st)
        app.sync()
        app.close()
        return ms * 1e-3

    out = {"paper": {"storage_order_128": PAPER_ORDER_S, "block_k20x": PAPER_BLOCK_S}}
    for dtype in ("f64", "f32"):
        order = {}
        for n in (128, 256):
            r = {lay: run(n, n, n, lay, (32, 8), dtype) for lay in ("ijk", "kij")}
            r["kij_over_ijk"] = r["kij"] / r["ijk"]
            order[str(n)] = r
        blocks = {}
        for b in ((128, 1), (32, 16), (32, 8), (64, 4)):
            blocks[f"{b[0]}x{b[1]}"] = {g: run(*dims, "ijk", b, dtype) for g, dims in
                                        (("128", (128, 128, 128)), ("256", (256, 256, 256)),
                                         ("256x512", (256, 256, 512)))}
        out[dtype] = {"storage_order_s_per_100_steps": order, "block_shape_s_per_100_steps": blocks}
    return out


def variant_rk3(steps_f32=100, steps_f64=20, nx=1581, ny=1301, nz=58):
    """WX_RK3 at the paper grid.  FP32 (TMEM variant): three stage launches
    of the step kernel that write their stages themselves, the last fused
    with the column physics: 16 + 24 + 24 = 64 HBM bytes per cell-step
    (stage 1 reads and writes T, q; stages 2 and 3 also read phi^n).  FP64:
    three stage launches (dynamics only), the stage-2 combine and the
    stage-3 combine fused with the column physics: 3 x 16 + 32 + 32 = 112
    bytes in FP32 units, 224 in FP64."""
    import torch
    from paper_1802_05839_gb300 import wx
    out = {}
    for dtype, steps in (("f32", steps_f32), ("f64", steps_f64)):
        case = make_case(dtype, nx, ny, nz)
        ctx = wx.Context(nx, ny, nz, dtype)
        ctx.set_params(case, flags=wx.WX_ADVECTION | wx.WX_PHYSICS | wx.WX_RK3)
        ctx.load_fields(case.T, case.q, case.U, case.V)
        st = torch.cuda.Stream()
        ms = _time_steps(lambda: ctx.step(1, stream=st), steps, st)
        ctx.sync()
        launches = ctx.last_launches()
        ctx.close()
        b = (64 if launches == 3 else 112) if dtype == "f32" else 224
        out[dtype] = {"ms_per_step": ms, "value": case.cells / (ms * 1e-3), "unit": "cell-steps/s",
                      "steps": steps, "gpu_launches_per_step": launches, "bytes_per_cell_step": b,
                      "hbm_frac": case.cells * b / (ms * 1e-3) / 1e9 / peaks()[0]}
    return out


def variants_summary(v):
    """The variants' headline figures in a few hundred bytes; written as the
    line's last key, so that a reader keeping only the line's tail still
    sees them."""
    r = lambda x, n=4: None if x is None else float(f"{x:.{n}g}")
    s = {}
    for k in ("f64", "mixed", "ensemble", "rk3_f32", "decomposed_2x2", "decomposed_4x4"):
        if k.startswith("decomposed"):
            rec = (v.get("decomposed") or {}).get(k.split("_")[1])
        else:
            rec = v.get(k) if k != "rk3_f32" else (v.get("rk3") or {}).get("f32")
        if rec:
            s[k] = {"ms": r(rec.get("ms_per_step")), "hbm_frac": r(rec.get("hbm_frac"), 3)}
    sur = v.get("surrogate")
    if sur:
        s["surrogate"] = {"ms": r(sur.get("ms_per_step")), "vs_plain": r(sur.get("vs_plain_step"), 3),
                          "fallback_frac": r(sur.get("fallback_frac"), 3),
                          "tendency_rel_l2": r(sur.get("val_tendency_rel_l2", {}).get("all"), 3),
                          "gemm_bf16_frac": r(sur.get("network_forward", {}).get("frac"), 3)}
        if "fallback_frac_at" in sur:
            s["surrogate"]["fallback_frac_at"] = {k: r(x, 3) for k, x in sur["fallback_frac_at"].items()}
        if "policy" in sur:
            s["surrogate"]["policy_ms"] = r(sur["policy"].get("ms_per_step"))
            s["surrogate"]["policy_vs_plain"] = r(sur["policy"].get("vs_plain_step"), 3)
    return s


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1802_05839_gb300 import wx

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    dtype = args.dtype
    case = make_case(dtype, args.nx, args.ny, args.nz)
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    # the mixed-precision workload records FP64 mass/energy sums every step
    flags = wx.WX_ADVECTION | wx.WX_PHYSICS | (wx.WX_SUMS if dtype == "mixed" else 0)
    ctx.set_params(case, flags=flags)
    ctx.load_fields(case.T, case.q, case.U, case.V)
    stream = torch.cuda.Stream()

    # warm-up, then the timed region bracketed by barrier + synchronize
    for _ in range(args.warmup):
        ctx.step(1, stream=stream)
    ctx.sync()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")   # ncu --nvtx --nvtx-include timed/
    ev[0].record(stream)
    for s in range(args.steps):
        ctx.step(1, stream=stream)
        ev[s + 1].record(stream)
    torch.cuda.nvtx.range_pop()
    stream.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ctx.sync()
    per = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    if world > 1:
        total_ms = max_over_ranks(total_ms)
        dist.barrier()
    launches = ctx.last_launches() * args.steps  # one wx_step(1) per timed step
    step_cfg = ctx.step_config()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return

    ms = total_ms / args.steps
    value = job_throughput(world, case.cells, ms)
    peak, peak_kind = peaks()
    alg_bytes = case.cells * CELL_BYTES[dtype] + case.nx * case.ny * COL_BYTES[dtype]
    kern_ms = statistics.mean(per)
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    out = {
        "metric": args.metric, "value": value, "unit": "cell-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "f64": "f64", "mixed": "f32+f64"}[dtype], "data": "synthetic",
        "config": {"workload": f"paper grid {case.nx}x{case.ny}x{case.nz} ({dtype}), "
                               "dynamics + column physics per step",
                   "step_config": step_cfg,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (2 x field buffers of "
                         f"{case.cells * CELL_BYTES[dtype] // 2 / 1e6:.0f} MB), no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic_record(dtype),
                     "kernel": "step_kernel", "alg_bytes_per_launch": alg_bytes,
                     "kernel_ms": kern_ms, "peak_source": peak_kind},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.skip_e2e:
        out["e2e"] = e2e_measure(case, dtype, n_ctx=args.e2e_contexts)
    if not args.skip_cpu:
        out["cpu_baseline"] = cpu_baseline(case if dtype == "f64" else make_case("f64"))
    if not args.no_variants and dtype == "f32" and (case.nx, case.ny, case.nz) == (1581, 1301, 58):
        out["variants"] = {
            "f64": variant_plain("f64", 100),
            "mixed": variant_plain("mixed", 500),
            "ensemble": variant_ensemble(200),
            "surrogate": variant_surrogate(100, plain_ms=ms, train_epochs=args.epochs),
            "reduced_app": variant_reduced_app(100),
            "ablation": variant_ablation(100),
            "rk3": variant_rk3(),
            "decomposed": variant_decomposed(100, plain_ms=ms),
        }
        out["variants_summary"] = variants_summary(out["variants"])
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64", "mixed"])
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--e2e-contexts", type=int, default=3,
                    help="contexts (and streams) the pipelined end-to-end measurement rotates through")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--nx", type=int, default=1581, help="grid override (profiling captures only)")
    ap.add_argument("--ny", type=int, default=1301, help="grid override (profiling captures only)")
    ap.add_argument("--nz", type=int, default=58, help="grid override (profiling captures only)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--epochs", type=int, default=64, help="surrogate training epochs")
    ap.add_argument("--only", choices=["f64", "mixed", "ensemble", "surrogate", "reduced_app", "ablation", "rk3",
                                       "decomposed"],
                    help="run one variant alone and print its record (profiling captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.metric = "cell-steps/s at 1581x1301x58 (FP32 vs FP64), % HBM peak; surrogate vs plain"
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        if args.only in ("f64", "mixed"):
            rec = variant_plain(args.only, args.steps, args.nx, args.ny, args.nz)
        elif args.only == "ensemble":
            rec = variant_ensemble(args.steps)
        elif args.only == "reduced_app":
            rec = variant_reduced_app(args.steps)
        elif args.only == "ablation":
            rec = variant_ablation(args.steps)
        elif args.only == "decomposed":
            rec = variant_decomposed(args.steps, args.nx, args.ny, args.nz)
        elif args.only == "rk3":
            rec = variant_rk3(args.steps, max(3, args.steps // 5), args.nx, args.ny, args.nz)
        else:
            rec = variant_surrogate(args.steps, args.nx, args.ny, train_epochs=args.epochs)
        print(json.dumps({"variant": args.only, **rec}))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
