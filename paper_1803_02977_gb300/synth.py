"""Seeded synthetic inputs for the landscape-evolution workloads.

Holds none of the method's arithmetic: only the random initial surfaces and
parameter draws that both the CUDA path and the oracle consume.

The paper's test data are square rasters of uniform noise with fixed seeds
(Section "Test Data").  Noise here comes from SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator: draw i of stream s is mix(s + (i+1) * GOLDEN), and
u = (draw >> 11) * 2^-53 lies in [0, 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Draws start..start+count-1 of the SplitMix64 stream seeded with `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform [0, 1) doubles with 53 random bits."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def noise_surface(nx: int, ny: int, seed: int, lo: float = 0.0, hi: float = 1.0,
                  south_tilt: float = 0.0, dx: float = 100.0) -> np.ndarray:
    """(ny, nx) float64 surface: row-major uniform [lo, hi) noise, plus
    south_tilt * dx * (ny-1-y) (a gradient falling toward row ny-1), with the
    perimeter set to base level 0."""
    if nx < 1 or ny < 1:
        raise ValueError("grid must be non-empty")
    h = lo + (hi - lo) * uniform01(seed, nx * ny).reshape(ny, nx)
    if south_tilt:
        y = np.arange(ny, dtype=np.float64)[:, None]
        h = h + south_tilt * dx * (ny - 1 - y)
    h[0, :] = 0.0
    h[-1, :] = 0.0
    h[:, 0] = 0.0
    h[:, -1] = 0.0
    return np.ascontiguousarray(h)


def signed_field(nx: int, ny: int, seed: int) -> np.ndarray:
    """(ny, nx) uniform [-1, 1) field."""
    return np.ascontiguousarray((2.0 * uniform01(seed, nx * ny) - 1.0).reshape(ny, nx))


@dataclass
class GridWorkload:
    """One grid run: size, stream-power parameters, initial surface recipe."""
    name: str
    nx: int
    ny: int
    dx: float = 100.0
    K: float = 1e-5
    m: float = 0.5
    U: float = 1e-3
    dt: float = 1000.0
    steps: int = 100
    seed: int = 1
    noise_hi: float = 1.0
    south_tilt: float = 0.0
    dtype: str = "f64"
    area_dtype: str = "i32"

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def initial(self) -> np.ndarray:
        return noise_surface(self.nx, self.ny, self.seed, 0.0, self.noise_hi,
                             self.south_tilt, self.dx)


def workload(name: str) -> GridWorkload:
    """The named synthetic workloads (uniform-noise squares, Section "Test Data")."""
    table = {
        # 256 x 256, FP64, noise [0,1), 100 steps
        "grid256_f64": GridWorkload("grid256_f64", 256, 256, steps=100, seed=1),
        # 2048 x 2048 with a 1e-4 tilt toward the south edge, 500 steps
        "grid2048_f64": GridWorkload("grid2048_f64", 2048, 2048, steps=500, seed=2,
                                     south_tilt=1e-4),
        "grid2048_f32": GridWorkload("grid2048_f32", 2048, 2048, steps=500, seed=2,
                                     south_tilt=1e-4, dtype="f32"),
        # the paper's 10,000 x 10,000 size, FP32 elevations, int64 areas
        "grid10000_f32": GridWorkload("grid10000_f32", 10000, 10000, K=2e-5, m=0.45,
                                      dt=500.0, steps=100, seed=3, noise_hi=10.0,
                                      dtype="f32", area_dtype="i64"),
        "grid10000_f64": GridWorkload("grid10000_f64", 10000, 10000, K=2e-5, m=0.45,
                                      dt=500.0, steps=100, seed=3, noise_hi=10.0,
                                      dtype="f64", area_dtype="i64"),
        # adjoint workload: 1024 x 1024 FP64, 50 steps
        "grid1024_adjoint": GridWorkload("grid1024_adjoint", 1024, 1024, steps=50, seed=5),
    }
    if name not in table:
        raise KeyError(f"unknown workload {name!r}; known: {sorted(table)}")
    return table[name]


@dataclass
class BatchWorkload:
    """Many independent realizations of uneven size and parameters."""
    name: str
    sides: list = field(default_factory=list)
    K: list = field(default_factory=list)
    m: list = field(default_factory=list)
    seeds: list = field(default_factory=list)
    dx: float = 100.0
    U: float = 1e-3
    dt: float = 1000.0
    steps: int = 200

    @property
    def count(self) -> int:
        return len(self.sides)

    @property
    def cells(self) -> int:
        return int(sum(s * s for s in self.sides))

    def initial(self, r: int) -> np.ndarray:
        s = self.sides[r]
        return noise_surface(s, s, self.seeds[r], 0.0, 1.0, 0.0, self.dx)


def batch_workload(count: int = 512, side_lo: int = 128, side_hi: int = 1024,
                   seed: int = 4, steps: int = 200) -> BatchWorkload:
    """Realization r: side uniform on {side_lo..side_hi}, K log-uniform on
    [1e-6, 1e-4] /yr, m uniform on [0.4, 0.6], surface seed 1000 + r."""
    u = uniform01(seed, 3 * count).reshape(count, 3)
    span = side_hi - side_lo + 1
    sides = [int(side_lo + min(span - 1, math.floor(u[r, 0] * span))) for r in range(count)]
    K = [float(10.0 ** (-6.0 + 2.0 * u[r, 1])) for r in range(count)]
    m = [float(0.4 + 0.2 * u[r, 2]) for r in range(count)]
    seeds = [1000 + r for r in range(count)]
    return BatchWorkload(f"batch{count}_f32", sides, K, m, seeds, steps=steps)
