"""Pins of the FP64 MLP oracle (oracle/mlp.py) to facts outside itself:
finite differences (P11), the closed form of Adam's first steps (P12),
known values of the normal CDF, an independent FP64 network in PyTorch, the
bfloat16 rounding of PyTorch, and the exactness of the residual checks on
the exact column physics of the plain oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
from paper_1802_05839_gb300 import inputs


def small_batch(M=6, seed=5):
    X = inputs.normal(seed, 1, M * 232).reshape(M, 232)
    Yt = inputs.normal(seed, 2, M * 116).reshape(M, 116)
    return X, Yt


def test_gelu_values_and_derivative():
    # GELU(z) = z Phi(z); Phi(1) = 0.8413447460685429 (standard normal CDF)
    phi1 = 0.8413447460685429
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([1.0]))[0] - phi1) < 1e-15
    assert abs(mlp.gelu(np.array([-1.0]))[0] + (1 - phi1)) < 1e-15
    assert abs(mlp.gelu(np.array([8.0]))[0] - 8.0) < 1e-12
    z = np.linspace(-5, 5, 41)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-9


def test_bf16_rounding_ties_to_even_and_matches_torch():
    one = 1.0
    assert mlp.bf16(one)[()] == 1.0
    assert mlp.bf16(1 + 2.0 ** -8)[()] == 1.0                   # tie -> even
    assert mlp.bf16(1 + 3 * 2.0 ** -8)[()] == 1 + 2.0 ** -6     # tie -> even (up)
    assert mlp.bf16(1 + 2.0 ** -8 + 2.0 ** -20)[()] == 1 + 2.0 ** -7
    x = inputs.normal(3, 9, 20000) * 10.0 ** (inputs.uniform(3, 10, 20000) * 8 - 4)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_two_term_bf16_expansion():
    """hi + lo carries FP32(x) to 16 significant bits: |x - hi - lo| <=
    2^-17 |x| (two roundings of 2^-9 each); hi alone only to 2^-9."""
    x = inputs.normal(6, 1, 50000) * 10.0 ** (inputs.uniform(6, 2, 50000) * 6 - 3)
    f = x.astype(np.float32).astype(np.float64)
    hi, lo = mlp.bf16_pair(x)
    assert np.array_equal(hi, mlp.bf16(x))
    assert np.all(np.abs(f - hi - lo) <= 2.0 ** -17 * np.abs(f))
    assert np.max(np.abs(f - hi) / np.abs(f)) > 2.0 ** -10


def test_forward_matches_independent_torch_network():
    Ws, bs = inputs.mlp_init(11)
    bs = [inputs.normal(11, 50 + l, len(b)) * 0.1 for l, b in enumerate(bs)]
    X, _ = small_batch(16)
    Y, _ = mlp.forward(Ws, bs, X, bf16_path=False)
    h = torch.from_numpy(X)
    for l in range(4):
        h = torch.nn.functional.linear(h, torch.from_numpy(Ws[l]), torch.from_numpy(bs[l]))
        if l < 3:
            h = torch.nn.functional.gelu(h, approximate="none")
    assert np.max(np.abs(Y - h.numpy())) < 1e-12 * max(1.0, np.max(np.abs(Y)))


def test_p11_backward_matches_central_differences():
    """P11: every layer's weight and bias gradient of the FP64 network
    against central differences with step 1e-6 (sampled entries)."""
    Ws, bs = inputs.mlp_init(21)
    bs = [inputs.normal(21, 60 + l, len(b)) * 0.1 for l, b in enumerate(bs)]
    X, Yt = small_batch(6, seed=8)
    L0, dW, db = mlp.loss_and_grads(Ws, bs, X, Yt, bf16_path=False)
    h = 1e-6
    rng = np.random.default_rng(0)
    worst = 0.0
    for l in range(4):
        for _ in range(6):
            n, k = rng.integers(Ws[l].shape[0]), rng.integers(Ws[l].shape[1])
            Wp = [W.copy() for W in Ws]
            Wm = [W.copy() for W in Ws]
            Wp[l][n, k] += h
            Wm[l][n, k] -= h
            fd = (mlp.loss_and_grads(Wp, bs, X, Yt, False)[0] -
                  mlp.loss_and_grads(Wm, bs, X, Yt, False)[0]) / (2 * h)
            err = abs(fd - dW[l][n, k]) / (abs(dW[l][n, k]) + 1e-4)
            worst = max(worst, err)
        for _ in range(3):
            n = rng.integers(len(bs[l]))
            bp = [b.copy() for b in bs]
            bm = [b.copy() for b in bs]
            bp[l][n] += h
            bm[l][n] -= h
            fd = (mlp.loss_and_grads(Ws, bp, X, Yt, False)[0] -
                  mlp.loss_and_grads(Ws, bm, X, Yt, False)[0]) / (2 * h)
            worst = max(worst, abs(fd - db[l][n]) / (abs(db[l][n]) + 1e-4))
    assert worst < 1e-6


def test_p11_input_gradient_chain():
    """The chain rule through all layers: d loss / d x by central differences
    equals the backward pass continued to the input."""
    Ws, bs = inputs.mlp_init(4)
    X, Yt = small_batch(3, seed=2)
    Y, cache = mlp.forward(Ws, bs, X, False)
    g = mlp.mse_grad(Y, Yt)
    for l in range(3, -1, -1):
        if l > 0:
            g = (g @ cache["Wr"][l]) * mlp.gelu_grad(cache["z"][l - 1])
        else:
            g = g @ cache["Wr"][0]
    h = 1e-6
    for (r, f) in [(0, 0), (1, 100), (2, 231)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[r, f] += h
        Xm[r, f] -= h
        fd = (mlp.mse(mlp.forward(Ws, bs, Xp, False)[0], Yt) -
              mlp.mse(mlp.forward(Ws, bs, Xm, False)[0], Yt)) / (2 * h)
        assert abs(fd - g[r, f]) <= 1e-6 * abs(g[r, f]) + 1e-10


def test_p12_adam_closed_form():
    """P12: with a constant gradient g, every bias-corrected Adam step moves
    by exactly -lr g / (|g| + eps)."""
    g = np.array([3.0, -2e-3, 1e-9, 0.0])
    p = np.array([1.0, 2.0, 3.0, 4.0])
    m = np.zeros(4)
    v = np.zeros(4)
    lr = 1e-3
    for t in range(1, 6):
        p_new, m, v = mlp.adam_step(p, g, m, v, t, lr)
        np.testing.assert_allclose(p_new - p, -lr * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-18)
        p = p_new


def test_cosine_schedule_ends():
    assert mlp.cosine_lr(0, 100) == 1e-3
    assert abs(mlp.cosine_lr(50, 100) - 5e-4) < 1e-18
    assert mlp.cosine_lr(100, 100) < 1e-18


def test_features_layout_and_normalisation():
    nz, ncol = 58, 40
    Ts = 280 + inputs.normal(1, 1, ncol * nz).reshape(ncol, nz)
    qs = 0.01 * inputs.uniform(1, 2, ncol * nz).reshape(ncol, nz)
    km = 1 + inputs.uniform(1, 3, ncol)
    kl = 0.01 + 0.04 * inputs.uniform(1, 4, nz)
    al = inputs.absorber(nz)
    dz = 1.05 ** np.arange(nz)
    F = mlp.raw_features(Ts, qs, km, kl, al, dz)
    assert F.shape == (ncol, 232)
    assert np.array_equal(F[:, :nz], Ts) and np.array_equal(F[:, nz:2 * nz], qs)
    assert np.allclose(F[7, 2 * nz:3 * nz], km[7] * kl)
    assert np.allclose(F[3, 3 * nz:], al * dz)
    mean, sd = mlp.fit_norm(F)
    Z = mlp.normalise(F, mean, sd)
    varying = np.ptp(F, axis=0) > 0
    assert np.allclose(Z[:, varying].mean(axis=0), 0, atol=1e-10)
    assert np.allclose(Z[:, varying].std(axis=0), 1, atol=1e-10)
    assert np.all(np.abs(Z[:, ~varying]) < 1e-6)
    assert np.allclose(mlp.denormalise(Z, mean, sd), F)


def test_residuals_vanish_on_exact_physics_and_are_one_for_no_mixing():
    """rho_vd of the exact T** is zero (it solves A x = T*), rho_H of the
    exact heating is zero (the flux divergence telescopes, P9); predicting
    no vertical diffusion at all gives rho_vd = 1 exactly by definition."""
    c = inputs.paper_grid_case(24, 10, 58, seed=3, near_singular=True)
    ncol = c.nx * c.ny
    Ts = np.ascontiguousarray(c.T.reshape(58, ncol).T)
    qs = np.ascontiguousarray(c.q.reshape(58, ncol).T)
    km = c.kappa_mult.reshape(ncol) if c.kappa_mult is not None else None
    _, tend = oracle.physics_columns(58, c.dt, c.dz, c.kappa_lev, km, c.alpha, c.S0, c.q_ref,
                                     Ts, qs, with_tend=True)
    H, rate = tend[:, 0, :], tend[:, 1, :]
    rvd, rH = mlp.residuals(Ts, qs, Ts + c.dt * rate, H, km, c.kappa_lev, c.alpha, c.dz,
                            c.dt, c.S0, c.q_ref)
    # x = T* + dt rate rebuilt from the stored rate carries ~1e-16 |T*| of
    # rounding against ||A T* - T*|| ~ 1e-6 |T*|
    assert np.max(rvd) < 1e-7
    assert np.max(rH) < 1e-12
    rvd0, _ = mlp.residuals(Ts, qs, Ts, H, km, c.kappa_lev, c.alpha, c.dz, c.dt, c.S0, c.q_ref)
    assert np.allclose(rvd0, 1.0, rtol=0, atol=1e-15)
    # 1% too much heating everywhere -> rho_H = 0.01
    _, rH1 = mlp.residuals(Ts, qs, Ts + c.dt * rate, 1.01 * H, km, c.kappa_lev, c.alpha, c.dz,
                           c.dt, c.S0, c.q_ref)
    assert np.allclose(rH1, 0.01, rtol=1e-9)


def test_planted_mistakes_are_caught():
    """A transposed weight in backward or a dropped GELU' factor would fail
    the finite-difference pin: plant each in a copy of the oracle's backward
    and check the pin's measure rejects it."""
    Ws, bs = inputs.mlp_init(9)
    X, Yt = small_batch(4, seed=4)
    Y, cache = mlp.forward(Ws, bs, X, False)
    dY = mlp.mse_grad(Y, Yt)

    def bad_backward(cache, dY):
        dW, db = [None] * 4, [None] * 4
        g = dY
        for l in range(3, -1, -1):
            dW[l] = g.T @ cache["a"][l]
            db[l] = g.sum(axis=0)
            if l > 0:
                g = g @ cache["Wr"][l]          # GELU' factor dropped
        return dW, db

    good = mlp.backward(cache, dY)[0][0]
    bad = bad_backward(cache, dY)[0][0]
    h = 1e-6
    n, k = 3, 5
    Wp = [W.copy() for W in Ws]
    Wm = [W.copy() for W in Ws]
    Wp[0][n, k] += h
    Wm[0][n, k] -= h
    fd = (mlp.mse(mlp.forward(Wp, bs, X, False)[0], Yt) -
          mlp.mse(mlp.forward(Wm, bs, X, False)[0], Yt)) / (2 * h)
    assert abs(fd - good[n, k]) <= 1e-6 * abs(good[n, k]) + 1e-12
    assert abs(fd - bad[n, k]) > 1e-3 * abs(fd)
