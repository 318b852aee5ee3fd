"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: only the workload shapes
(lattice sizes, relaxation times, driven shells, amplitudes, seeds) and
seeded generators of initial macroscopic fields (energy density and
3-velocity on the lattice).  Both the CUDA library and the CPU oracle consume
these inputs; neither is imported here.

The shapes follow the runs of the paper (Sec. 5: periodic N x N lattices,
N = 128 ... 1024, flat start at rest, stirring on a wavenumber band near
k_f = 6, filtered velocities ~0.01-0.015) scaled up to the sizes a GB300
holds.  The paper uses no public dataset; these generators stand in for its
runs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    tau: float
    dtype: str            # storage form: "f64", "f32", "bf16", "f16"
    kmin: int = 0
    kmax: int = 0
    amp: float = 0.0
    seed: int = 0
    redraw: int = 100
    steps: int = 100
    init: str = "rest"    # "rest" or "shear"
    extra: dict = field(default_factory=dict)

    @property
    def forced(self) -> bool:
        return self.amp > 0.0 and self.kmax > 0


SEED = 2101061870

# Shear-wave decay: 128^2, FP64 form, tau = 0.8, eps = 1, v_x = 0.01 sin(2 pi y/128), no force, 2000 steps.
SHEAR_128 = Workload("shear_wave_128x128_f64_tau0.8", 128, 128, 0.8, "f64", steps=2000, init="shear",
                     extra={"u0": 0.01})
# Stirred turbulence: 1024^2, FP32 populations (and the same run in FP64 form), tau = 0.52,
# shell 4 <= |k| <= 6, amplitude 1e-5, redraw every 100 steps, 50k steps.
STIRRED_1024 = Workload("stirred_1024x1024_tau0.52_shell4-6", 1024, 1024, 0.52, "f32", kmin=4, kmax=6, amp=1e-5,
                        seed=SEED, redraw=100, steps=50000)
# Precision forms: 4096^2, BF16 / FP16 deviation storage, tau = 0.51, shell 8..10, amplitude 5e-6, 20k steps.
PRECISION_4096 = Workload("stirred_4096x4096_tau0.51_shell8-10", 4096, 4096, 0.51, "bf16", kmin=8, kmax=10,
                          amp=5e-6, seed=SEED + 1, redraw=100, steps=20000)
# Large steady turbulence: 8192^2, FP32, tau = 0.505, shell 16..18, amplitude 2e-6.
LARGE_8192 = Workload("stirred_8192x8192_tau0.505_shell16-18", 8192, 8192, 0.505, "f32", kmin=16, kmax=18,
                      amp=2e-6, seed=SEED + 2, redraw=100, steps=100000)

ENSEMBLE_SIDES = (256, 384, 512, 768, 1024)


def shear_wave(nx: int, ny: int, u0: float = 0.01):
    """eps = 1, v_x = u0 sin(2 pi y / ny), v_y = 0."""
    y = np.arange(ny, dtype=np.float64)
    vx = np.repeat((u0 * np.sin(2.0 * np.pi * y / ny))[:, None], nx, axis=1)
    return np.ones((ny, nx)), vx, np.zeros((ny, nx))


def rest(nx: int, ny: int, eps0: float = 1.0):
    return np.full((ny, nx), eps0), np.zeros((ny, nx)), np.zeros((ny, nx))


def random_smooth(nx: int, ny: int, seed: int, deps: float = 0.05, vmax: float = 0.05, nmodes: int = 4):
    """Seeded smooth periodic fields: eps = 1 + deps * (sum of a few low
    Fourier modes), and a 3-velocity of comparable smoothness with |v| up to
    about vmax.  Periodic on the lattice, so any size is valid."""
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")

    def field_():
        out = np.zeros((ny, nx))
        for _ in range(nmodes):
            kx = int(rng.integers(-3, 4))
            ky = int(rng.integers(-3, 4))
            ph = rng.uniform(0, 2 * np.pi)
            a = rng.uniform(-1, 1)
            out += a * np.cos(2 * np.pi * (kx * x / nx + ky * y / ny) + ph)
        return out / nmodes

    eps = 1.0 + deps * field_()
    vx = vmax * field_()
    vy = vmax * field_()
    return eps, vx, vy


def random_smooth3d(nx: int, ny: int, nz: int, seed: int, deps: float = 0.05, vmax: float = 0.05,
                    nmodes: int = 4):
    """Seeded smooth periodic fields on an nx x ny x nz lattice ([z][y][x]):
    eps = 1 + deps * (a few low 3D Fourier modes) and three velocity
    components of comparable smoothness, |v| up to about vmax."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")

    def field_():
        out = np.zeros((nz, ny, nx))
        for _ in range(nmodes):
            kx, ky, kz = (int(rng.integers(-2, 3)) for _ in range(3))
            ph = rng.uniform(0, 2 * np.pi)
            a = rng.uniform(-1, 1)
            out += a * np.cos(2 * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ph)
        return out / nmodes

    eps = 1.0 + deps * field_()
    return eps, vmax * field_(), vmax * field_(), vmax * field_()


def random_tiled(nx: int, ny: int, period: int, seed: int, deps: float = 0.05, vmax: float = 0.05):
    """Fields periodic with a small period (period | nx, ny): the tile of
    `random_smooth(period, period)` repeated over the lattice.  A large
    lattice started from it must stay an exact tiling of the small one."""
    e, a, b = random_smooth(period, period, seed, deps, vmax)
    ry, rx = ny // period, nx // period
    return np.tile(e, (ry, rx)), np.tile(a, (ry, rx)), np.tile(b, (ry, rx))


def random_nodes(n: int, seed: int, vmax: float = 0.6):
    """n random (eps, v) pairs: eps in [0.5, 2], |v| <= vmax, isotropic in 3D
    (for node-level tests)."""
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.5, 2.0, size=n)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    s = vmax * rng.uniform(0, 1, size=n) ** (1.0 / 3.0)
    return eps, d * s[:, None]


def ensemble(nruns: int = 64, seed: int = SEED + 3, sides=ENSEMBLE_SIDES):
    """The batched-ensemble workload: per run a square side drawn from
    `sides`, tau ~ U[0.51, 0.7], a driven band [c-1, c+1] with centre
    c ~ U[4, 12] rounded to an integer band, amplitude 1e-5 and its own seed."""
    rng = np.random.default_rng(seed)
    runs = []
    for r in range(nruns):
        n = int(sides[int(rng.integers(0, len(sides)))])
        tau = float(rng.uniform(0.51, 0.7))
        c = float(rng.uniform(4.0, 12.0))
        kmin = max(1, int(np.floor(c - 1.0)))
        kmax = int(np.ceil(c + 1.0))
        runs.append(Workload("ens%02d" % r, n, n, tau, "f32", kmin=kmin, kmax=kmax, amp=1e-5,
                             seed=int(seed * 1000 + r), redraw=100, steps=100))
    return runs


def philox_pin_inputs(n_random: int = 4096, seed: int = 11):
    """Counter and key words (uint32, shapes (n, 4) and (n, 2)) on which a
    Philox4x32-10 implementation is compared with an independent one: the
    counters the stirring force draws with ({epoch, mode, stream, 0} for
    epochs 0..3, modes 0..255, streams 0..2) under the keys of the
    workloads' seeds (low word, high word), the all-zero and all-one words,
    and n_random seeded uniform draws."""
    ctr, key = [], []
    for s in (SEED, SEED + 1, SEED + 2):
        k = (s & 0xFFFFFFFF, (s >> 32) & 0xFFFFFFFF)
        for epoch in range(4):
            for mode in range(256):
                for stream in range(3):
                    ctr.append((epoch, mode, stream, 0))
                    key.append(k)
    ctr += [(0, 0, 0, 0), (0xFFFFFFFF,) * 4]
    key += [(0, 0), (0xFFFFFFFF, 0xFFFFFFFF)]
    rng = np.random.default_rng(seed)
    c = np.concatenate([np.array(ctr, dtype=np.uint64),
                        rng.integers(0, 1 << 32, size=(n_random, 4), dtype=np.uint64)]).astype(np.uint32)
    k = np.concatenate([np.array(key, dtype=np.uint64),
                        rng.integers(0, 1 << 32, size=(n_random, 2), dtype=np.uint64)]).astype(np.uint32)
    return c, k
