"""Seeded synthetic inputs and the named workload configurations.

This module holds no lattice Boltzmann arithmetic: it only draws the inputs
that the library, its tests and the benchmark feed to the method (inlet
density profiles, perturbations of the rest state, regions of interest) and
records the workload sizes.  The library and the CPU oracle both consume
these inputs; neither is imported here.

Stand-ins for the paper's data (the paper's 2D packings and its CT-scanned
Hamburg sand are not available): grain packings come from the seeded
geometry recipe of the library (disks for D2Q9, spheres for D3Q19), and the
unknown inlet profile is a smooth random 4-mode sine series.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def inlet_profile(n: int, seed: int, amplitude: float = 1e-3, modes: int = 4) -> np.ndarray:
    """Inlet density excess delta(y) = rho_in(y) - rho_out, shape [n].

    delta(y) = A (1 + s(y) / max_y |s|),  s(y) = sum_{m=1..modes} a_m sin(m pi (y + 1/2) / n + phi_m),
    a_m ~ U[-1, 1], phi_m ~ U[0, 2 pi), drawn from numpy's PCG64 seeded with ``seed``.
    The profile is positive (between 0 and 2A) and smooth across the inlet.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.uniform(-1.0, 1.0, modes)
    phi = rng.uniform(0.0, 2.0 * math.pi, modes)
    y = np.arange(n, dtype=np.float64)
    s = np.zeros(n)
    for m in range(1, modes + 1):
        s += a[m - 1] * np.sin(m * math.pi * (y + 0.5) / n + phi[m - 1])
    return amplitude * (1.0 + s / np.max(np.abs(s)))


def perturbation(shape, seed: int, scale: float = 1e-3) -> np.ndarray:
    """Seeded uniform noise in [-scale, scale) of the given shape (float64).

    Used as a shifted population state f - w (a perturbed rest state), as an
    adjoint direction, or as a test direction."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-scale, scale, size=shape)


def roi_band(shape, axis: int, start: int) -> np.ndarray:
    """uint8 region of interest: 1 where the index along ``axis`` is >= start
    (the paper observes only a band near the outlet or the top)."""
    roi = np.zeros(shape, np.uint8)
    sl = [slice(None)] * len(shape)
    sl[axis] = slice(start, None)
    roi[tuple(sl)] = 1
    return roi


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named synthetic workload: lattice, sizes, geometry recipe and step count."""

    name: str
    q: int
    nx: int
    ny: int
    nz: int
    precision: int          # bytes per real: 4 (FP32) or 8 (FP64)
    steps: int              # T
    tau: float
    geom_kind: int          # 0 channel/duct, 1 disks, 2 spheres
    seed: int
    r_min: int
    r_max: int
    porosity: float
    inlet: str              # "const" or "profile"
    rho_out: float = 1.0
    delta_rho: float = 1e-3  # constant head rho_in - rho_out (const inlet)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz


WORKLOADS = {
    # D2Q9 FP64 64x32 channel, walls top/bottom, no grains, rho_in 1.001 / rho_out 1.0, 1000 steps.
    "channel64x32": Workload("channel64x32", 9, 64, 32, 1, 8, 1000, 0.8, 0, 0, 6, 12, 1.0, "const"),
    # D2Q9 FP32 512x256 disks r 6-12 lu, porosity 0.6, 20000 steps, 256-entry inlet profile.
    "disks512x256": Workload("disks512x256", 9, 512, 256, 1, 4, 20000, 0.8, 1, 1000, 6, 12, 0.6, "profile"),
    # D3Q19 FP32 128x64x64 duct, spheres r 6 lu, porosity 0.45, 10000 steps, constant head + tau.
    "spheres128x64x64": Workload("spheres128x64x64", 19, 128, 64, 64, 4, 10000, 0.8, 2, 3000, 6, 6, 0.45,
                                 "const"),
    # Lattices larger than L2, for the HBM roofline of the step kernels.
    "disks8192x4096": Workload("disks8192x4096", 9, 8192, 4096, 1, 4, 20, 0.8, 1, 7000, 6, 12, 0.6, "profile"),
    "disks4096x2048": Workload("disks4096x2048", 9, 4096, 2048, 1, 4, 20, 0.8, 1, 7001, 6, 12, 0.6, "profile"),
    "spheres256x128x128": Workload("spheres256x128x128", 19, 256, 128, 128, 4, 10, 0.8, 2, 8001, 6, 6, 0.45,
                                   "const"),
    "spheres512x256x256": Workload("spheres512x256x256", 19, 512, 256, 256, 4, 10, 0.8, 2, 8000, 6, 6, 0.45,
                                   "const"),
}


def batch_sizes(count: int = 64, seed: int = 4000):
    """Sizes for the batched inversions: nx = 32 * U{4..32}, ny = nx / 2, porosity U[0.5, 0.7]."""
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(seed + i))
        nx = 32 * int(rng.integers(4, 33))
        out.append((nx, nx // 2, float(rng.uniform(0.5, 0.7)), seed + i))
    return out
