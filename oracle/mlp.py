"""FP64 CPU oracle of the column-physics MLP surrogate.

TEST INFRASTRUCTURE ONLY: nothing in the product path imports this module.
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may call it.

The surrogate replaces the two column-physics steps of the time step (the
implicit vertical diffusion of Sec. 2 / Eq. 1 applied per column, and the
top-down optical-depth scan with its radiative heating) by a learned map

    x = [T*_k, q*_k, kappa_v(k), alpha_k dz_k]  (4 x 58 = 232 features)
    h1 = GELU(W1 x + b1), h2 = GELU(W2 h1 + b2), h3 = GELU(W3 h2 + b3)
    y  = W4 h3 + b4 = [H_k, (T**_k - T*_k)/dt]   (2 x 58 = 116 outputs)

with inputs and targets normalised per feature, mean-squared-error loss and
Adam.  GELU is the exact erf form 0.5 z (1 + erf(z / sqrt 2)), evaluated by
calling ``scipy.special.erf``.

``forward(..., bf16=True)`` rounds the weights and each hidden activation to
bfloat16 (round to nearest even, as the tensor-core path stores them), takes
each normalised input (held in FP32) as its two-term bfloat16 expansion
hi + lo, hi = bf16(x), lo = bf16(x - hi), and accumulates in FP64;
``bf16=False`` is the plain FP64 network used by the finite-difference pin.
``backward`` is full FP64.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SQRT_HALF = np.sqrt(0.5)
INV_SQRT_2PI = 1.0 / np.sqrt(2.0 * np.pi)


# --------------------------------------------------------------- rounding
def bf16(x) -> np.ndarray:
    """Round to bfloat16 (round to nearest, ties to even) via FP32: the value
    is first rounded to FP32 (as the device holds it) and then to the 8-bit
    significand.  Returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def bf16_pair(x):
    """Two-term bfloat16 expansion (hi, lo) of FP32(x): hi = bf16(x),
    lo = bf16(x - hi); x - hi is exact in FP32."""
    f = np.asarray(x, dtype=np.float32).astype(np.float64)
    hi = bf16(f)
    return hi, bf16(f - hi)


# --------------------------------------------------------------- network
def gelu(z):
    return 0.5 * z * (1.0 + erf(z * SQRT_HALF))


def gelu_grad(z):
    """d/dz of z Phi(z) = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z * SQRT_HALF)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def forward(Ws, bs, X, bf16_path: bool = True):
    """X [M][232] normalised inputs -> (Y [M][116], cache for backward)."""
    rnd = bf16 if bf16_path else (lambda a: np.asarray(a, dtype=np.float64))
    if bf16_path:
        hi, lo = bf16_pair(X)
        h = hi + lo
    else:
        h = np.asarray(X, dtype=np.float64)
    cache = {"a": [h], "z": []}
    for l in range(4):
        z = h @ rnd(Ws[l]).T + np.asarray(bs[l], dtype=np.float64)
        if l == 3:
            cache["Wr"] = [rnd(W) for W in Ws]
            return z, cache
        cache["z"].append(z)
        h = rnd(gelu(z))
        cache["a"].append(h)


def mse(Y, Yt) -> float:
    """Mean of (Y - Yt)^2 over all M x 116 entries."""
    d = Y - Yt
    return float(np.mean(d * d))


def mse_grad(Y, Yt):
    return 2.0 * (Y - Yt) / Y.size


def backward(cache, dY):
    """Gradients of a scalar loss L(Y) given dL/dY, by the chain rule through
    the four affine layers and three GELUs; returns (dW list, db list)."""
    dW, db = [None] * 4, [None] * 4
    g = np.asarray(dY, dtype=np.float64)
    for l in range(3, -1, -1):
        a = cache["a"][l]
        dW[l] = g.T @ a
        db[l] = g.sum(axis=0)
        if l > 0:
            g = (g @ cache["Wr"][l]) * gelu_grad(cache["z"][l - 1])
    return dW, db


def loss_and_grads(Ws, bs, X, Yt, bf16_path: bool = True):
    Y, cache = forward(Ws, bs, X, bf16_path)
    dW, db = backward(cache, mse_grad(Y, Yt))
    return mse(Y, Yt), dW, db


# --------------------------------------------------------------- Adam
def adam_step(p, g, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) with bias correction;
    t is the 1-based step count.  Returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def cosine_lr(step: int, total: int, lr0: float = 1e-3) -> float:
    return 0.5 * lr0 * (1.0 + np.cos(np.pi * min(step, total) / total))


# --------------------------------------------------------------- features
def raw_features(Ts, qs, kappa_mult, kappa_lev, alpha, dz):
    """[ncol][232] = [T*_k | q*_k | kappa_mult kappa_lev(k) | alpha_k dz_k]."""
    Ts = np.asarray(Ts, dtype=np.float64)
    qs = np.asarray(qs, dtype=np.float64)
    ncol, nz = Ts.shape
    km = np.ones(ncol) if kappa_mult is None else np.asarray(kappa_mult, dtype=np.float64).reshape(ncol)
    kv = km[:, None] * np.asarray(kappa_lev, dtype=np.float64)[None, :]
    adz = np.broadcast_to(np.asarray(alpha) * np.asarray(dz), (ncol, nz))
    return np.concatenate([Ts, qs, kv, adz], axis=1)


def raw_targets(tend):
    """tend [ncol][2][nz] = (H_k, (T**_k - T*_k)/dt) -> [ncol][2 nz]."""
    tend = np.asarray(tend, dtype=np.float64)
    return tend.reshape(tend.shape[0], -1)


def fit_norm(F):
    """Per-feature mean and standard deviation (population) of rows F; a
    constant feature gets a floor of 1e-6 |mean| (or 1 when the mean is 0)."""
    mean = F.mean(axis=0)
    sd = np.sqrt(np.maximum((F * F).mean(axis=0) - mean * mean, 0.0))
    floor = 1e-6 * np.maximum(np.abs(mean), 1e-12)
    sd = np.maximum(sd, floor)
    sd[sd == 0] = 1.0
    return mean, sd


def normalise(F, mean, sd):
    return (F - mean) / sd


def denormalise(Y, mean, sd):
    return Y * sd + mean


# --------------------------------------------------------------- residuals
def residuals(Ts, qs, Tss_hat, H_hat, kappa_mult, kappa_lev, alpha, dz, dt, S0, q_ref):
    """Per-column acceptance checks of a predicted column:

    rho_vd = ||A x - T*|| / ||A T* - T*||, with A = I - dt L_v the implicit
      vertical-diffusion operator of the column and x the predicted T**;
    rho_H  = |sum_k H_k dz_k - S0 (1 - exp(-tau_tot))| / (S0 (1 - exp(-tau_tot))),
      the column energy budget of the beam, which the exact heating meets by
      telescoping.
    """
    from . import vdiff_coeffs  # tridiagonal coefficients of the exact path

    Ts = np.asarray(Ts, dtype=np.float64)
    ncol, nz = Ts.shape
    km = np.ones(ncol) if kappa_mult is None else np.asarray(kappa_mult, dtype=np.float64).reshape(ncol)
    rvd = np.empty(ncol)
    for c in range(ncol):
        a, b, cc = vdiff_coeffs(nz, dt, dz, kappa_lev, km[c])
        x = Tss_hat[c]
        Ax = b * x
        Ax[1:] += a[1:] * x[:-1]
        Ax[:-1] += cc[:-1] * x[1:]
        AT = b * Ts[c]
        AT[1:] += a[1:] * Ts[c, :-1]
        AT[:-1] += cc[:-1] * Ts[c, 1:]
        den = np.linalg.norm(AT - Ts[c])
        num = np.linalg.norm(Ax - Ts[c])
        rvd[c] = num / den if den > 0 else (0.0 if num == 0 else np.inf)
    tau = (np.asarray(alpha) * np.asarray(dz) / q_ref)[None, :] * np.asarray(qs, dtype=np.float64)
    absorbed = S0 * (1.0 - np.exp(-tau.sum(axis=1)))
    rH = np.abs((np.asarray(H_hat) * np.asarray(dz)[None, :]).sum(axis=1) - absorbed) / absorbed
    return rvd, rH
