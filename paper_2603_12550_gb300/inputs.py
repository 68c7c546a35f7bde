"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module only draws random numbers and names workload sizes; it holds none
of the method's arithmetic and imports nothing else from this package.

Initial condition (Sec. 3.1): every component of bond k is drawn i.i.d. from
N(0, kBT / H_k) -- the Boltzmann distribution of the Hookean potential.
Arrays are drawn in FP64 with ``numpy.random.default_rng(seed)`` and rounded
to FP32 for the device; the oracle receives the same FP32 values widened back
to FP64, so both sides start from identical numbers.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "equilibrium_cloud",
    "ensemble_sizes",
    "snapshot_matrix",
    "WORKLOADS",
    "shear_kappa",
]


def shear_kappa(s: int, rate: float) -> np.ndarray:
    """Simple-shear velocity gradient acting as qdot = kappa q, flow along x1,
    gradient along x2 (kappa[0, 1] = shear rate), s x s."""
    k = np.zeros((s, s))
    k[0, 1] = rate
    return k


def equilibrium_cloud(N: int, nb: int, s: int, H=1.0, kBT: float = 1.0,
                      seed: int = 0, fene_b: float | None = None) -> np.ndarray:
    """N x (nb*s) FP32 cloud with bond k ~ N(0, kBT/H_k) per component.

    With ``fene_b`` set, any particle with some |q_k|^2 >= b is redrawn from
    the same stream until all bonds lie inside the FENE domain.
    """
    H = np.broadcast_to(np.asarray(H, dtype=np.float64), (nb,))
    rng = np.random.default_rng(seed)
    D = nb * s
    scale = np.repeat(np.sqrt(kBT / H), s)
    q = rng.standard_normal((N, D)) * scale
    if fene_b is not None:
        while True:
            n2 = (q.reshape(N, nb, s) ** 2).sum(-1)
            bad = np.nonzero((n2 >= fene_b).any(-1))[0]
            if bad.size == 0:
                break
            q[bad] = rng.standard_normal((bad.size, D)) * scale
    return q.astype(np.float32)


def ensemble_sizes(n_ens: int, seed: int = 0, lo_exp: float = 10.0,
                   hi_exp: float = 14.0, rate_lo: float = -1.0,
                   rate_hi: float = 1.0):
    """Ensemble sizes N_e = round(2^U(lo,hi)) and shear rates 10^U(rate_lo, rate_hi)."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(2.0 ** rng.uniform(lo_exp, hi_exp, n_ens)).astype(np.int64)
    rates = 10.0 ** rng.uniform(rate_lo, rate_hi, n_ens)
    return sizes, rates


def snapshot_matrix(n_rows: int, n_cols: int, rank: int, seed: int = 0,
                    decay: float = 0.5, noise: float = 0.0) -> np.ndarray:
    """Synthetic column-major-ready snapshot matrix (n_rows x n_cols) of a
    prescribed rank with geometrically decaying singular values, plus optional
    small full-rank noise.  Used only where a test needs a known spectrum."""
    rank = min(rank, n_rows, n_cols)
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n_rows, rank))
    B = rng.standard_normal((rank, n_cols))
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B.T)
    sv = decay ** np.arange(rank) * math.sqrt(n_rows)
    X = (Qa * sv) @ Qb.T
    if noise:
        X = X + noise * rng.standard_normal((n_rows, n_cols))
    return X.astype(np.float32)


# Workload recipes (sizes and physical parameters), named by what they are.
WORKLOADS = {
    # 2D Hookean dumbbell: N=512, D=2, h=0.3, shear rate 1, dt=0.01, implicit.
    "dumbbell2d_n512": dict(N=512, nb=1, s=2, H=[1.0], kBT=1.0, zeta=4.0,
                            h=0.3, dt=0.01, rate=1.0, spring=0, b=0.0,
                            scheme=1, steps=50, seed=0),
    # 3D Hookean dumbbell: N=16384, D=3, Silverman h, dt=0.005.
    "dumbbell3d_n16384": dict(N=16384, nb=1, s=3, H=[1.0], kBT=1.0, zeta=4.0,
                              h=None, dt=0.005, rate=1.0, spring=0, b=0.0,
                              scheme=0, steps=1000, seed=0),
    # 4-bead chain in 3D: N=65536, D=9 (3 bonds x 3), shear rate 1, dt=0.005.
    "chain4_n65536_d9": dict(N=65536, nb=3, s=3, H=[1.0, 1.0, 1.0], kBT=1.0,
                             zeta=4.0, h=None, dt=0.005, rate=1.0, spring=0,
                             b=50.0, scheme=0, steps=1000, seed=0),
}


def mlp_init(widths=(9, 256, 256, 256, 9), seed: int = 0, scale: float = 1.0):
    """Seeded initial parameters of an MLP with the given layer widths:
    W_l (out x in) ~ N(0, scale^2 / in), b_l = 0.  Returns a list of (W, b)
    in FP32 (the draws; no arithmetic of the method)."""
    rng = np.random.default_rng(seed)
    layers = []
    for fan_in, fan_out in zip(widths[:-1], widths[1:]):
        W = rng.standard_normal((fan_out, fan_in)) * (scale / math.sqrt(fan_in))
        layers.append((W.astype(np.float32), np.zeros(fan_out, dtype=np.float32)))
    return layers


def dsm_batch(X: np.ndarray, batch: int, seed: int):
    """A training batch for denoising score matching: `batch` rows drawn with
    replacement from X (n x D) and standard normal noise of the same shape."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, X.shape[0], batch)
    eps = rng.standard_normal((batch, X.shape[1])).astype(np.float32)
    return X[idx].astype(np.float32), eps


def dsm_rows(n_pool: int, batch: int, D: int, seed: int):
    """Row indices (batch, with replacement, int32) into a pool of n_pool
    configurations and standard normal noise (batch x D, FP32)."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, n_pool, batch).astype(np.int32),
            rng.standard_normal((batch, D)).astype(np.float32))
