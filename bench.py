"""Benchmark of the fused weather step on GB300.

Default workload: the paper's grid 1581 x 1301 x 58 (Sec. 5.5), FP32 fields,
dynamics + column physics, seeded synthetic state (the paper's JMA inputs are
not public).  One step = one pass of the whole hot path over the grid.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0.  `value` is whole-job cell-steps/s timed with
CUDA events on the launching stream (inputs resident in HBM; the two 955 MB
field buffers exceed the 129 MB L2, so no flush is needed); `e2e` is the same
metric through the C ABI with host buffers (load + step + read back every
step); `roofline` relates the step kernel's algorithmic bytes to the measured
HBM copy bandwidth; `cpu_baseline` times the FP64 CPU oracle on a bounded
sample of the same workload on this host's cores.
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


def e2e_measure(case, dtype, iters=3):
    """Load (H2D from pinned host) + one step + read back (D2H) per step."""
    import torch
    from paper_1802_05839_gb300 import wx
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    T, q, U, V = pin(case.T), pin(case.q), pin(case.U), pin(case.V)
    To = torch.empty(T.shape, dtype=torch.float64).pin_memory().numpy()
    qo = torch.empty(T.shape, dtype=torch.float64).pin_memory().numpy()
    ctx = wx.Context(case.nx, case.ny, case.nz, dtype)
    ctx.set_params(case)
    ctx.load_fields(T, q, U, V)
    ctx.step(1)
    ctx.sync()
    ctx.read_fields()
    t0 = time.perf_counter()
    for _ in range(iters):
        ctx.load_fields(T, q, U, V)
        ctx.step(1)
        ctx.sync()
        lib = wx.lib()
        wx._check(lib.wx_read_fields(ctx.ptr, wx._dptr(To), wx._dptr(qo)), ctx.ptr)
    el = (time.perf_counter() - t0) / iters
    ctx.close()
    h2d = T.nbytes + q.nbytes + U.nbytes + V.nbytes
    return {"value": case.cells / el, "unit": "cell-steps/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(To.nbytes + qo.nbytes), "ms_per_step": el * 1e3,
            "path": "wx_load_fields(host) + wx_step(1) + wx_read_fields(host)"}


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
    ev[0].record(stream)
    for s in range(args.steps):
        ctx.step(1, stream=stream)
        ev[s + 1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ctx.sync()
    per = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        total_ms = float(t.item())
    launches = ctx.last_launches() * args.steps  # one wx_step(1) per timed step
    step_cfg = ctx.step_config()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return

    ms = total_ms / args.steps
    value = world * case.cells / (ms * 1e-3)
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
        out["e2e"] = e2e_measure(case, dtype)
    if not args.skip_cpu:
        out["cpu_baseline"] = cpu_baseline(case if dtype == "f64" else make_case("f64"))
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64", "mixed"])
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--nx", type=int, default=1581, help="grid override (profiling captures only)")
    ap.add_argument("--ny", type=int, default=1301, help="grid override (profiling captures only)")
    ap.add_argument("--nz", type=int, default=58, help="grid override (profiling captures only)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.metric = "cell-steps/s at 1581x1301x58 (FP32 vs FP64), % HBM peak"
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
