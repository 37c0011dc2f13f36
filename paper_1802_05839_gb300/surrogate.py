"""Training driver of the column-physics MLP surrogate.

Data: columns (T*, q*, kappa_mult) of seeded synthetic states after the
dynamics of one step, with their exact column-physics tendencies from the
library's column kernel (wx_physics_columns).  Training: minibatches of the
normalised rows through wx_mlp_train_step (forward, backward and Adam in the
library's kernels), cosine-decayed learning rate.  PyTorch only holds device
memory and reorders rows between calls.
"""
from __future__ import annotations

import numpy as np

from . import inputs, wx

NZ = 58


def _torch():
    import torch
    return torch


def state_columns(ctx, nx, ny, nz=NZ):
    """The context's current fields as device FP32 columns [nx*ny][nz]."""
    torch = _torch()
    T = torch.empty(nz, ny, nx, dtype=torch.float64, device="cuda")
    q = torch.empty_like(T)
    ctx.read_fields_into(T, q)
    ctx.sync()
    to_cols = lambda a: a.reshape(nz, -1).t().contiguous().float()
    return to_cols(T), to_cols(q)


def case_columns(case, adv_steps):
    """(T*, q*, kappa_mult or None, tend) of every column of `case` after
    `adv_steps` full FP32 steps and the dynamics of one more (device FP32
    tensors; the tendencies computed in FP64 from the FP32 inputs)."""
    torch = _torch()
    nx, ny, nz = case.nx, case.ny, case.nz
    ctx = wx.Context(nx, ny, nz, "f32")
    try:
        ctx.set_params(case)
        ctx.load_fields(case.T, case.q, case.U, case.V)
        if adv_steps:
            ctx.step(adv_steps)
        ctx.set_params(case, flags=wx.WX_ADVECTION)
        ctx.step(1)
        Ts, qs = state_columns(ctx, nx, ny, nz)
    finally:
        ctx.close()
    km = None
    if case.kappa_mult is not None:
        km = torch.from_numpy(np.ascontiguousarray(case.kappa_mult, np.float32).reshape(-1)).cuda()
    # Targets from the FP64 column kernel: T** - T* is ~1e-4 K, a few FP32
    # ulps of T ~ 280 K, so FP32 targets would be mostly rounding noise.
    c64 = wx.Context(nx, ny, nz, "f64")
    try:
        c64.set_params(case)
        Tout = torch.empty(Ts.shape, dtype=torch.float64, device="cuda")
        tend = torch.empty(Ts.shape[0], 2, nz, dtype=torch.float64, device="cuda")
        c64.physics_columns(Ts.double(), qs.double(), km.double() if km is not None else None, Tout, tend)
        c64.sync()
    finally:
        c64.close()
    return Ts, qs, km, tend.float()


CONFIG_SEED = 12345  # the model configuration (kappa_lev profile) served


def dataset(seeds, nx=256, ny=256, near_singular=False, max_adv=50, config_seed=CONFIG_SEED):
    """Concatenated columns of the paper-grid generator's states for each
    seed (one shared model configuration), advanced (7 seed) mod
    (max_adv + 1) steps first."""
    torch = _torch()
    parts = []
    for s in seeds:
        case = inputs.round_to_f32(inputs.paper_grid_case(nx, ny, NZ, seed=s, near_singular=near_singular,
                                                          config_seed=config_seed))
        parts.append(case_columns(case, (7 * s) % (max_adv + 1)))
    Ts = torch.cat([p[0] for p in parts])
    qs = torch.cat([p[1] for p in parts])
    km = None
    if near_singular:
        km = torch.cat([p[2] if p[2] is not None else torch.ones(p[0].shape[0], device="cuda") for p in parts])
    tend = torch.cat([p[3] for p in parts])
    return Ts, qs, km, tend


def rows(mlp, Ts, qs, km, tend=None):
    """Normalised BF16 input rows [ceil128(n)][512] (and FP32 targets)."""
    torch = _torch()
    n = Ts.shape[0]
    pad = (n + 127) // 128 * 128
    X = torch.empty(pad, wx.MLP_X_WIDTH, dtype=torch.bfloat16, device="cuda")
    Yt = torch.empty(pad, wx.MLP_OUT_PAD, dtype=torch.float32, device="cuda") if tend is not None else None
    mlp.prepare(Ts, qs, km, tend, X, Yt)
    return X, Yt


def set_levels_from_case(mlp, case):
    mlp.set_levels(np.asarray(case.kappa_lev, np.float32),
                   np.asarray(np.asarray(case.alpha) * np.asarray(case.dz), np.float32))


def train(mlp, X, Yt, n_rows, epochs=4, batch=4096, lr0=1e-3, seed=0, log=None):
    """Adam on shuffled minibatches of the first n_rows rows; returns the
    per-epoch mean loss (device losses read once per epoch)."""
    torch = _torch()
    g = torch.Generator(device="cpu").manual_seed(seed)
    nb = n_rows // batch
    total = epochs * nb
    loss = torch.zeros(max(nb, 1), dtype=torch.float32, device="cuda")
    hist = []
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n_rows, generator=g).cuda()
        for b in range(nb):
            idx = perm[b * batch:(b + 1) * batch]
            lr = 0.5 * lr0 * (1.0 + np.cos(np.pi * step / total))
            mlp.train_step(X.index_select(0, idx), Yt.index_select(0, idx), lr, loss=loss[b:])
            step += 1
        hist.append(float(loss[:nb].mean().item()))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    mlp.status()
    return hist


def predict(mlp, X):
    """Physical-unit predictions [rows][116] (H | vdiff rate) of BF16 rows."""
    torch = _torch()
    Y = torch.empty(X.shape[0], wx.MLP_OUT_PAD, dtype=torch.float32, device="cuda")
    mlp.forward(X, Y)
    _, _, mo, so = mlp.get_norm()
    mo = torch.from_numpy(mo).cuda()
    so = torch.from_numpy(so).cuda()
    return Y[:, :wx.MLP_OUT] * so + mo


def tendency_error(mlp, Ts, qs, km, tend):
    """Relative L2 error of the predicted tendencies in physical units over
    all columns: (both halves, heating only, vertical diffusion only)."""
    X, _ = rows(mlp, Ts, qs, km)
    n = Ts.shape[0]
    P = predict(mlp, X)[:n].double()
    Y = tend.reshape(n, -1).double()
    rel = lambda a, b: float((a - b).norm() / b.norm())
    return rel(P, Y), rel(P[:, :NZ], Y[:, :NZ]), rel(P[:, NZ:], Y[:, NZ:])
