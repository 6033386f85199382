"""Seeded synthetic inputs for the forward-Euler phase-field / reaction-diffusion step.

This module is the only code shared by the CUDA path (its tests and ``bench.py``) and the
FP64 oracle.  It holds no arithmetic of the method itself: only a counter-based random
generator and the recipes that turn its draws into initial fields and model parameters.

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014).  Output ``i`` (0-based) of a stream with key ``K`` is
``mix(K + (i + 1) * GAMMA)`` with the usual SplitMix64 finaliser; the key of stream ``s``
under seed ``S`` is ``mix(S * GAMMA + s)``.  A uniform draw on ``[a, b)`` is
``a + (b - a) * (bits >> 11) * 2**-53``.  All arithmetic is mod 2**64 (numpy uint64).

Layout of every field: dense C order ``[nz][ny][nx]`` (3D) or ``[ny][nx]`` (2D), x fastest,
which is the row-major, x-first grid layout of the paper (Sec. 2.2.1 "Uniform Grid").
Fields are returned as float32: both sides start from the same FP32-representable array.

Recipes (the paper sets initial conditions to uniform noise, Sec. 3; the Gray-Scott
recipe, which the paper does not give, follows the reaction-diffusion workloads):

* ``allen_cahn_init``   phi ~ U(lo, hi) independently per site.
* ``cahn_hilliard_init`` phi ~ U(-amp, amp), then the FP64 sample mean is subtracted.
* ``gray_scott_init``   u = 1, v = 0; ``n_seeds`` axis-aligned cubes (squares in 2D) of
  side ``side`` with origins uniform on the periodic grid are set to u = 0.5, v = 0.25
  (overlaps allowed, wrapping at the edges); then both fields get multiplicative noise
  x <- x * (1 + noise * U(-1, 1)).
* ``batch_instances``   side N = round(exp(U(ln lo, ln hi))), F ~ U(F range),
  k ~ U(k range) per instance; every instance is seeded by ``gray_scott_init``.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


def _mix_int(z: int) -> int:
    """SplitMix64 finaliser on a Python int (mod 2**64)."""
    z &= _MASK
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (numpy wraps mod 2**64)."""
    z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> int:
    """Key of sub-stream ``stream`` under ``seed``."""
    return _mix_int((seed * GAMMA + stream) & _MASK)


def splitmix64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of sub-stream ``stream`` (uint64 array)."""
    key = np.uint64(stream_key(seed, stream))
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + i * np.uint64(GAMMA))


def uniform(seed: int, stream: int, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """``count`` float64 draws on ``[lo, hi)`` from sub-stream ``stream``."""
    bits = splitmix64(seed, stream, count)
    u01 = (bits >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u01


# --------------------------------------------------------------------------- recipes

def allen_cahn_init(shape, seed: int = 1, lo: float = -0.1, hi: float = 0.1) -> np.ndarray:
    """phi_0 ~ U(lo, hi) per site, rounded once to float32."""
    n = int(np.prod(shape))
    return uniform(seed, 0, n, lo, hi).reshape(shape).astype(np.float32)


def cahn_hilliard_init(shape, seed: int = 2, amp: float = 0.05) -> np.ndarray:
    """phi_0 = U(-amp, amp) minus its FP64 sample mean, rounded once to float32."""
    n = int(np.prod(shape))
    x = uniform(seed, 0, n, -amp, amp)
    x -= x.mean()
    return x.reshape(shape).astype(np.float32)


def gray_scott_init(shape, seed: int = 3, n_seeds: int = 20, side: int = 8,
                    noise: float = 0.01, u_in: float = 0.5, v_in: float = 0.25):
    """(u_0, v_0) float32: u=1, v=0 with seeded cubes/squares and multiplicative noise."""
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    u = np.ones(shape, dtype=np.float64)
    v = np.zeros(shape, dtype=np.float64)
    origins = uniform(seed, 1, n_seeds * d)
    for c in range(n_seeds):
        idx = []
        for ax in range(d):
            o = int(origins[c * d + ax] * shape[ax]) % shape[ax]
            idx.append((o + np.arange(min(side, shape[ax]))) % shape[ax])
        sel = np.ix_(*idx)
        u[sel] = u_in
        v[sel] = v_in
    n = u.size
    u *= 1.0 + noise * uniform(seed, 2, n, -1.0, 1.0).reshape(shape)
    v *= 1.0 + noise * uniform(seed, 3, n, -1.0, 1.0).reshape(shape)
    return u.astype(np.float32), v.astype(np.float32)


def batch_instances(n: int = 512, seed: int = 4, side_lo: int = 64, side_hi: int = 512,
                    F_range=(0.02, 0.06), k_range=(0.045, 0.07)):
    """Sizes and parameters of ``n`` independent square 2D Gray-Scott instances.

    Returns a list of dicts with keys ``n`` (side), ``F``, ``k``.
    """
    lsides = uniform(seed, 10, n, math.log(side_lo), math.log(side_hi))
    Fs = uniform(seed, 11, n, *F_range)
    ks = uniform(seed, 12, n, *k_range)
    return [dict(n=int(round(math.exp(ls))), F=float(F), k=float(k))
            for ls, F, k in zip(lsides, Fs, ks)]


def batch_instance_init(side: int, index: int, seed: int = 4):
    """Initial (u, v) of batch instance ``index``: one 8x8 square per 128x128 of area."""
    n_seeds = max(1, (side * side) // (128 * 128))
    return gray_scott_init((side, side), seed=seed * 1_000_003 + index + 1, n_seeds=n_seeds)


def paper_timing_init(model: str, shape, seed: int = 6):
    """Fields seeded uniformly in [-1, 1] (the paper's initial conditions for Models A-C,
    Sec. 3): one field for Model A, (psi, m) for Model C."""
    n = int(np.prod(shape))
    f0 = uniform(seed, 30, n, -1.0, 1.0).reshape(shape).astype(np.float32)
    if model == "ac":
        return (f0,)
    return (f0, uniform(seed, 31, n, -1.0, 1.0).reshape(shape).astype(np.float32))


# The paper's performance workloads (Sec. 3.1 table), run here with both solvers: Models A
# and C on 128^2, 512^2 and 64^3 for 10^4 iterations.  `paper_best_s` is the fastest
# whole-program time the paper reports for that case (min over its three CPUs, semi-implicit
# spectral solver) -- context from other hardware, not a target.
PAPER_TABLE = [
    dict(model="ac", shape=(128, 128), coeffs=(1.0, 1.0), dt=0.05, paper_best_s=1.7),
    dict(model="ac", shape=(512, 512), coeffs=(1.0, 1.0), dt=0.05, paper_best_s=32.6),
    dict(model="ac", shape=(64, 64, 64), coeffs=(1.0, 1.0), dt=0.05, paper_best_s=31.1),
    dict(model="c", shape=(128, 128), coeffs=(1.0,) * 5, dt=0.005, paper_best_s=4.1),
    dict(model="c", shape=(512, 512), coeffs=(1.0,) * 5, dt=0.005, paper_best_s=102.8),
    dict(model="c", shape=(64, 64, 64), coeffs=(1.0,) * 5, dt=0.005, paper_best_s=96.7),
]
PAPER_TABLE_STEPS = 10000


# Concrete workloads: the five configurations the measurements use.
WORKLOADS = {
    "ac2d_128": dict(model="ac", shape=(128, 128), h=1.0, dt=0.05, coeffs=(1.0, 1.0), steps=1000),
    "ch2d_2048": dict(model="ch", shape=(2048, 2048), h=1.0, dt=0.01, coeffs=(1.0, 1.0, 1.0),
                      steps=20000),
    "gs3d_256": dict(model="gs", shape=(256, 256, 256), h=1.0, dt=0.5,
                     coeffs=(0.2, 0.1, 0.04, 0.06), steps=5000),
    "gs2d_batch512": dict(model="gs", n_instances=512, h=1.0, dt=0.5, Du=0.2, Dv=0.1, steps=2000),
    "gs2d_adjoint_512": dict(model="gs", shape=(512, 512), h=1.0, dt=0.5,
                             coeffs=(0.2, 0.1, 0.04, 0.06), steps=2000),
}


def workload_init(name: str, shape=None):
    """Initial fields (tuple of float32 arrays) of a named workload, optionally resized."""
    w = WORKLOADS[name]
    shape = tuple(shape) if shape is not None else w.get("shape")
    if w["model"] == "ac":
        return (allen_cahn_init(shape, seed=1),)
    if w["model"] == "ch":
        return (cahn_hilliard_init(shape, seed=2),)
    if name == "gs3d_256":
        return gray_scott_init(shape, seed=3, n_seeds=20, side=8)
    if name == "gs2d_adjoint_512":
        n_seeds = max(1, (shape[0] * shape[1]) // (128 * 128))
        return gray_scott_init(shape, seed=5, n_seeds=n_seeds, side=8)
    raise KeyError(name)
