"""Seeded synthetic inputs: velocity models, Ricker wavelets and workload lists.

This module holds none of the solver's arithmetic. It produces the inputs that
both the CUDA path and the FP64 oracle consume (numpy only), so the two sides
see bit-identical models, wavelets and source positions. The paper runs on
synthetic grids only (Sec. 4: 256^3 points, space orders 8-24); its workloads
are reproduced here by shape, with the layered and smooth-random velocity
models described beside each function.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

H = 10.0  # grid spacing in metres for every workload


def slowness2(v) -> np.ndarray:
    """Squared slowness m = 1 / v^2 (Eq. 1) as float32."""
    v = np.asarray(v, dtype=np.float64)
    return (1.0 / (v * v)).astype(np.float32)


def pad_edge(v_interior: np.ndarray, nbl: int) -> np.ndarray:
    """Extend an interior model into the absorbing layer by edge replication."""
    return np.pad(v_interior, nbl, mode="edge") if nbl > 0 else np.array(v_interior)


def constant_velocity(interior, nbl: int, v: float) -> np.ndarray:
    shape = tuple(n + 2 * nbl for n in interior)
    return np.full(shape, v, dtype=np.float64)


def layered_velocity(interior, nbl: int, velocities=(1500.0, 2500.0, 3500.0, 4500.0)) -> np.ndarray:
    """Equal-thickness horizontal layers along z (depth), slowest at the top."""
    nx, ny, nz = interior
    v = np.empty((nx, ny, nz), dtype=np.float64)
    nl = len(velocities)
    for i, vel in enumerate(velocities):
        z0 = (i * nz) // nl
        z1 = ((i + 1) * nz) // nl
        v[:, :, z0:z1] = vel
    return pad_edge(v, nbl)


def _gaussian_smooth(a: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian filter (truncated at 4 sigma, reflecting edges)."""
    rad = int(math.ceil(4 * sigma))
    t = np.arange(-rad, rad + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    out = a
    for ax in range(a.ndim):
        pad = [(0, 0)] * a.ndim
        pad[ax] = (rad, rad)
        p = np.pad(out, pad, mode="reflect")
        acc = np.zeros_like(out)
        for i, w in enumerate(k):
            sl = [slice(None)] * a.ndim
            sl[ax] = slice(i, i + out.shape[ax])
            acc += w * p[tuple(sl)]
        out = acc
    return out


def _upsample_linear(a: np.ndarray, factor: int, shape) -> np.ndarray:
    """Separable linear interpolation of a coarse grid (spacing `factor`) onto
    the first shape[ax] points of the fine grid."""
    out = a
    for ax, n in enumerate(shape):
        pos = np.arange(n, dtype=np.float64) / factor
        i0 = np.floor(pos).astype(np.int64)
        w = (pos - i0).reshape([-1 if d == ax else 1 for d in range(a.ndim)])
        lo = np.take(out, i0, axis=ax)
        hi = np.take(out, i0 + 1, axis=ax)
        out = lo * (1.0 - w) + hi * w
    return out


def smooth_random_velocity(interior, nbl: int, rng: np.random.Generator, vmin=1500.0, vmax=4500.0,
                           sigma=8.0) -> np.ndarray:
    """Gaussian-filtered N(0,1) noise (sigma in cells), min-max rescaled to
    [vmin, vmax], edge-replicated into the layer. Fields above 2 M points draw
    the noise on a 4x coarser grid, smooth it with sigma/4 and interpolate
    linearly (the same correlation length at 1/64 of the cost)."""
    interior = tuple(int(n) for n in interior)
    if int(np.prod(interior)) > 2_000_000 and sigma >= 4:
        f = 4
        coarse = tuple(n // f + 2 for n in interior)
        s = _upsample_linear(_gaussian_smooth(rng.standard_normal(coarse), sigma / f), f, interior)
    else:
        s = _gaussian_smooth(rng.standard_normal(interior), sigma)
    s = (s - s.min()) / max(s.max() - s.min(), 1e-30)
    return pad_edge(vmin + (vmax - vmin) * s, nbl)


def ricker(f0: float, dt: float, nt: int, amplitude: float = 1.0) -> np.ndarray:
    """Ricker wavelet (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = n dt - 1/f0."""
    t = np.arange(nt, dtype=np.float64) * dt - 1.0 / f0
    a = (math.pi * f0 * t) ** 2
    return (amplitude * (1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


# ---- workloads ----------------------------------------------------------------

@dataclass
class ShotSpec:
    interior: tuple
    nbl: int
    space_order: int
    velocity: np.ndarray = field(repr=False)  # over the computational domain (float64)
    source: tuple                             # interior node
    f0: float
    nt: int
    dt: float = 0.0                           # filled by the caller from the stability limit
    storage: str = "f32"
    arrival: float = 0.0

    @property
    def shape(self):
        return tuple(n + 2 * self.nbl for n in self.interior)

    @property
    def points(self) -> int:
        return int(np.prod(self.shape))

    @property
    def m(self) -> np.ndarray:
        return slowness2(self.velocity)

    @property
    def vmax(self) -> float:
        return float(self.velocity.max())


def plain_shot() -> ShotSpec:
    """64^3 interior + 10-cell layer, space order 4, v = 1.5 km/s, 10 Hz Ricker at
    the centre (32, 32, 32), 100 steps."""
    return ShotSpec((64, 64, 64), 10, 4, constant_velocity((64, 64, 64), 10, 1500.0),
                    (32, 32, 32), 10.0, 100)


def sweep_shot(space_order: int, n: int = 256, nbl: int = 10, nt: int = 500) -> ShotSpec:
    """n^3 interior + nbl layer, 4 horizontal layers 1.5/2.5/3.5/4.5 km/s along z,
    15 Hz Ricker at (n/2, n/2, 20 n/256), nt steps (the paper's 256^3 workload)."""
    interior = (n, n, n)
    return ShotSpec(interior, nbl, space_order, layered_velocity(interior, nbl),
                    (n // 2, n // 2, max(1, (20 * n) // 256)), 15.0, nt)


def batched_shots(seed: int = 0, count: int = 64, lo: int = 96, hi: int = 256, nbl: int = 10,
                  space_order: int = 8, nt: int = 300, sigma: float = 8.0) -> list[ShotSpec]:
    """Uneven shots: each axis drawn independently from U{lo..hi}, smooth random
    velocity (sigma cells), 10 Hz Ricker at a random interior node."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        interior = tuple(int(v) for v in rng.integers(lo, hi + 1, size=3))
        vel = smooth_random_velocity(interior, nbl, rng, sigma=sigma)
        src = tuple(int(rng.integers(0, n)) for n in interior)
        out.append(ShotSpec(interior, nbl, space_order, vel, src, 10.0, nt))
    return out


def precision_shot(n: int = 384, nbl: int = 20, nt: int = 1000, space_order: int = 12) -> ShotSpec:
    """n^3 interior + nbl layer, space order 12 (by default), 4-layer model (n/4-cell layers)."""
    interior = (n, n, n)
    return ShotSpec(interior, nbl, space_order, layered_velocity(interior, nbl),
                    (n // 2, n // 2, max(1, (20 * n) // 256)), 15.0, nt)


def serving_trace(seed: int = 0, count: int = 200, rate: float = 20.0, lo: int = 128,
                  hi: int = 512, nbl: int = 10, steps=(200, 2000), orders=(8, 16),
                  smooth_sigma: float = 8.0, max_interior: int | None = None) -> list[ShotSpec]:
    """Poisson arrivals (rate per second) of cubic shots n ~ U{lo..hi}, space order
    drawn from `orders`, FP32 or BF16 storage at 50/50, steps ~ U{steps}.
    Velocity models are generated lazily by the caller (see velocity_for)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += rng.exponential(1.0 / rate)
        n = int(rng.integers(lo, hi + 1))
        if max_interior:
            n = min(n, max_interior)
        so = int(rng.choice(orders))
        st = "f32" if rng.random() < 0.5 else "bf16"
        nt = int(rng.integers(steps[0], steps[1] + 1))
        src = tuple(int(rng.integers(0, n)) for _ in range(3))
        spec = ShotSpec((n, n, n), nbl, so, None, src, 10.0, nt, storage=st, arrival=t)
        spec.velocity_seed = int(rng.integers(0, 2 ** 31))
        out.append(spec)
    return out


def velocity_for(spec: ShotSpec, sigma: float = 8.0) -> np.ndarray:
    """Smooth random velocity for a serving request (seeded per request)."""
    rng = np.random.default_rng(spec.velocity_seed)
    return smooth_random_velocity(spec.interior, spec.nbl, rng, sigma=sigma)
