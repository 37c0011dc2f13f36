"""Seeded synthetic inputs for the weather step (shared by the GPU path's
callers and the oracle's tests; holds none of the step's arithmetic).

The paper ran its reduced weather application and ASUCA on real or
box-shaped initial states (Sec. 3.1: a 300 K box in a 0 K field; Sec. 5:
JMA operational data, not public).  These generators stand in for them
with smooth, seeded states of the same grid shapes:

* T  = 280 K + 8 Fourier modes, amplitude U[0,2] K, horizontal wavenumbers
  1..4, vertical cosine factor cos(pi c (k+1/2)/nz) with c in 0..4;
* q  = U[0, 0.02] i.i.d. (a moisture-like tracer);
* winds from a seeded streamfunction psi at cell corners, differenced onto
  C-grid faces so the discrete divergence is zero (w = 0), scaled so the
  largest face speed is 10;
* absorber alpha_k = 0.01 exp(-k/8), k counted from the bottom;
* layer thickness dz_k = 1 (small grid) or 1.05^k (paper grid);
* kappa_lev = 0.02 (small grid) or U[0.01, 0.05] per level (paper grid);
* kappa_mult = 1, or (mixed-precision case) 10^U[4,5] on a Bernoulli(0.05)
  mask of "near-singular" columns.

Random numbers come from SplitMix64 (Steele, Lea and Flood, 2014) used as a
counter-based generator: value n of stream s is mix64(key(s) + (n+1)*golden),
so any sub-block can be regenerated and the sequence does not depend on the
numpy version.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        base = np.array([np.uint64(seed) * _GOLDEN + np.uint64(stream)], dtype=np.uint64)
    return _mix64(base)[0]


def _uniform_block(k, start: int, n: int, out: np.ndarray) -> None:
    z = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    t = np.empty_like(z)
    with np.errstate(over="ignore"):
        np.multiply(z, _GOLDEN, out=z)
        np.add(z, k, out=z)
        for sh, mul in ((30, _M1), (27, _M2)):
            np.right_shift(z, np.uint64(sh), out=t)
            np.bitwise_xor(z, t, out=z)
            np.multiply(z, mul, out=z)
        np.right_shift(z, np.uint64(31), out=t)
        np.bitwise_xor(z, t, out=z)
        np.right_shift(z, np.uint64(11), out=z)
    np.multiply(z, 1.0 / 9007199254740992.0, out=out)


def uniform(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n doubles in [0, 1) (53-bit), values start..start+n-1 of the stream."""
    k = _key(seed, stream)
    out = np.empty(n, dtype=np.float64)
    blk = 1 << 20
    for b0 in range(0, n, blk):
        m = min(blk, n - b0)
        _uniform_block(k, start + b0, m, out[b0:b0 + m])
    return out


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal doubles by the Box-Muller transform."""
    m = (n + 1) // 2
    u1 = uniform(seed, stream, m)
    u2 = uniform(seed, stream + 0x5151, m)
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1-u1 in (0,1]
    out = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return out[:n]


# stream tags (arbitrary distinct constants)
_S_TMODES, _S_Q, _S_PSI, _S_KLEV, _S_MASK, _S_KMULT, _S_PERT = 11, 12, 13, 14, 15, 16, 17


@dataclasses.dataclass
class Case:
    """One problem instance: sizes, parameters and the initial state.

    Field layouts (C order): T, q [nz][ny][nx]; U, V, kappa_mult [ny][nx];
    dz, kappa_lev, alpha [nz].  U[j][i] sits on the east face of cell (i,j),
    V[j][i] on its north face.
    """
    nx: int
    ny: int
    nz: int
    dt: float
    h: float
    kappa_h: float
    S0: float
    q_ref: float
    dz: np.ndarray
    kappa_lev: np.ndarray
    alpha: np.ndarray
    kappa_mult: Optional[np.ndarray]
    T: np.ndarray
    q: np.ndarray
    U: np.ndarray
    V: np.ndarray
    advection: bool = True
    physics: bool = True
    name: str = ""

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def copy(self) -> "Case":
        return dataclasses.replace(
            self, T=self.T.copy(), q=self.q.copy(), U=self.U.copy(), V=self.V.copy(),
            dz=self.dz.copy(), kappa_lev=self.kappa_lev.copy(), alpha=self.alpha.copy(),
            kappa_mult=None if self.kappa_mult is None else self.kappa_mult.copy())


def temperature(nx: int, ny: int, nz: int, seed: int) -> np.ndarray:
    """280 K plus 8 seeded separable Fourier modes, [nz][ny][nx]."""
    u = uniform(seed, _S_TMODES, 8 * 6)
    A = 2.0 * u[0:8]
    a = 1 + np.floor(4 * u[8:16]).astype(int)
    b = 1 + np.floor(4 * u[16:24]).astype(int)
    c = np.floor(5 * u[24:32]).astype(int)
    ph = 2 * np.pi * u[32:40]
    ii = np.arange(nx)[None, :] / nx
    jj = np.arange(ny)[:, None] / ny
    kk = (np.arange(nz) + 0.5) / nz
    planes = np.stack([A[m] * np.cos(2 * np.pi * (a[m] * ii + b[m] * jj) + ph[m])
                       for m in range(8)]).reshape(8, ny * nx)
    vert = np.stack([np.cos(np.pi * c[m] * kk) for m in range(8)], axis=1)  # [nz][8]
    T = vert @ planes
    T += 280.0
    return T.reshape(nz, ny, nx)


def tracer(nx: int, ny: int, nz: int, seed: int) -> np.ndarray:
    """q ~ U[0, 0.02] i.i.d., [nz][ny][nx]."""
    return 0.02 * uniform(seed, _S_Q, nx * ny * nz).reshape(nz, ny, nx)


def winds(nx: int, ny: int, h: float, seed: int, umax: float = 10.0):
    """Divergence-free C-grid face winds (U, V) from a seeded streamfunction.

    psi[j][i] lives at the corner (i+1/2, j+1/2).  U on the east face of
    cell (i,j) is -(psi[j][i] - psi[j-1][i])/h, V on its north face is
    (psi[j][i] - psi[j][i-1])/h, with periodic wrap.  psi is scaled first so
    the largest |U| or |V| is umax.
    """
    u = uniform(seed, _S_PSI, 8 * 4)
    B = 0.5 + u[0:8]
    a = 1 + np.floor(4 * u[8:16]).astype(int)
    b = 1 + np.floor(4 * u[16:24]).astype(int)
    ph = 2 * np.pi * u[24:32]
    ii = (np.arange(nx)[None, :] + 0.5) / nx
    jj = (np.arange(ny)[:, None] + 0.5) / ny
    psi = np.zeros((ny, nx))
    for m in range(8):
        psi += B[m] * np.sin(2 * np.pi * (a[m] * ii + b[m] * jj) + ph[m])

    def diff(p):
        U = -(p - np.roll(p, 1, axis=0)) / h
        V = (p - np.roll(p, 1, axis=1)) / h
        return U, V

    U, V = diff(psi)
    peak = max(np.abs(U).max(), np.abs(V).max())
    scale = umax / peak if peak > 0 else 0.0  # a 1x1 periodic grid has no wind
    return diff(psi * scale)


def absorber(nz: int) -> np.ndarray:
    return 0.01 * np.exp(-np.arange(nz) / 8.0)


def near_singular_multiplier(nx: int, ny: int, seed: int, frac: float = 0.05):
    """kappa_mult [ny][nx]: 10^U[4,5] on a Bernoulli(frac) mask, else 1."""
    mask = uniform(seed, _S_MASK, nx * ny) < frac
    expo = 4.0 + uniform(seed, _S_KMULT, nx * ny)
    return np.where(mask, 10.0 ** expo, 1.0).reshape(ny, nx)


def small_case(nx=128, ny=128, nz=32, seed=12345) -> Case:
    """128x128x32, uniform dz = 1, kappa_lev = 0.02 (the small plain-method run)."""
    h = 2.5
    U, V = winds(nx, ny, h, seed)
    return Case(nx=nx, ny=ny, nz=nz, dt=0.1, h=h, kappa_h=0.05, S0=1.0, q_ref=0.01,
                dz=np.ones(nz), kappa_lev=np.full(nz, 0.02), alpha=absorber(nz),
                kappa_mult=None, T=temperature(nx, ny, nz, seed),
                q=tracer(nx, ny, nz, seed), U=U, V=V, name=f"small {nx}x{ny}x{nz}")


def paper_grid_case(nx=1581, ny=1301, nz=58, seed=12345, near_singular=False,
                    config_seed=None) -> Case:
    """The paper's ASUCA grid shape (Sec. 5.4): 1581x1301x58 by default.

    dz_k = 1.05^k, kappa_lev ~ U[0.01, 0.05] per level.  With near_singular
    the Bernoulli(0.05) columns get kappa_mult = 10^U[4,5].  The fields and
    winds come from `seed`; kappa_lev from `config_seed` (default: `seed`),
    so that several states can share one model configuration.
    """
    h = 2.5
    U, V = winds(nx, ny, h, seed)
    klev = 0.01 + 0.04 * uniform(seed if config_seed is None else config_seed, _S_KLEV, nz)
    km = near_singular_multiplier(nx, ny, seed) if near_singular else None
    return Case(nx=nx, ny=ny, nz=nz, dt=0.1, h=h, kappa_h=0.05, S0=1.0, q_ref=0.01,
                dz=1.05 ** np.arange(nz), kappa_lev=klev, alpha=absorber(nz),
                kappa_mult=km, T=temperature(nx, ny, nz, seed),
                q=tracer(nx, ny, nz, seed), U=U, V=V,
                name=f"paper-grid {nx}x{ny}x{nz}" + (" near-singular" if near_singular else ""))


def ensemble_sizes(members=16, seed=7):
    """Member grid sizes: first 256x256x40, last 1024x768x58, the rest drawn
    uniformly (nx in [256,1024], ny in [256,768], nz in [40,58])."""
    u = uniform(seed, 21, 3 * members)
    sizes = []
    for m in range(members):
        if m == 0:
            sizes.append((256, 256, 40))
        elif m == members - 1:
            sizes.append((1024, 768, 58))
        else:
            nx = 256 + int(np.floor(u[3 * m] * 769))
            ny = 256 + int(np.floor(u[3 * m + 1] * 513))
            nz = 40 + int(np.floor(u[3 * m + 2] * 19))
            sizes.append((nx, ny, nz))
    return sizes


def ensemble_member(m: int, nx: int, ny: int, nz: int, seed=12345) -> Case:
    """Member m: paper-grid generators at its own size, T perturbed per cell
    by N(0, 0.5^2) with seed 1000+m."""
    c = paper_grid_case(nx, ny, nz, seed=seed)
    c.T = c.T + 0.5 * normal(1000 + m, _S_PERT, nx * ny * nz).reshape(nz, ny, nx)
    c.name = f"member {m} {nx}x{ny}x{nz}"
    return c


def round_to_f32(case: Case) -> Case:
    """The same case with every input rounded once to FP32 (and held in
    float64 again), which is what an FP32 run of the step sees."""
    r = lambda a: None if a is None else np.asarray(a, np.float32).astype(np.float64)
    f = lambda x: float(np.float32(x))
    c = case.copy()
    c.T, c.q, c.U, c.V = r(c.T), r(c.q), r(c.U), r(c.V)
    c.dz, c.kappa_lev, c.alpha, c.kappa_mult = r(c.dz), r(c.kappa_lev), r(c.alpha), r(c.kappa_mult)
    c.dt, c.h, c.kappa_h, c.S0, c.q_ref = f(c.dt), f(c.h), f(c.kappa_h), f(c.S0), f(c.q_ref)
    return c


# ----------------------------------------------------------------- MLP
MLP_SIZES = [(232, 512), (512, 512), (512, 512), (512, 116)]  # (fan_in, fan_out)


def mlp_init(seed: int = 2024):
    """Random initial weights of the column-physics MLP: He/Kaiming-uniform
    W_l ~ U(-sqrt(6/fan_in), sqrt(6/fan_in)) in [fan_out][fan_in] layout,
    biases zero.  Stream 100 + l of `seed` per layer."""
    Ws, bs = [], []
    for l, (fi, fo) in enumerate(MLP_SIZES):
        bound = np.sqrt(6.0 / fi)
        u = uniform(seed, 100 + l, fi * fo)
        Ws.append(((2.0 * u - 1.0) * bound).reshape(fo, fi))
        bs.append(np.zeros(fo))
    return Ws, bs


def column_sample(ncol_total: int, n: int, seed: int, stream: int = 200) -> np.ndarray:
    """n distinct-ish column indices drawn uniformly from [0, ncol_total)."""
    return np.minimum((uniform(seed, stream, n) * ncol_total).astype(np.int64), ncol_total - 1)


# ------------------------------------------------- reduced application
def paper_box_state(nx: int, ny: int, nz: int, T_box: float = 300.0) -> np.ndarray:
    """The reduced application's initial state (Sec. 3.1): 0 K everywhere and
    T_box inside the box from one quarter to three quarters of each
    dimension, read as the interior indices [n/4, 3n/4) (0-based) of each
    axis; the ghost ring starts at 0 K.  Layout [nz][ny+2][nx+2]."""
    E = np.zeros((nz, ny + 2, nx + 2))
    E[nz // 4:(3 * nz) // 4, 1 + ny // 4:1 + (3 * ny) // 4, 1 + nx // 4:1 + (3 * nx) // 4] = T_box
    return E
