"""Synthetic workloads shaped like the paper's runs (no method arithmetic here).

Each workload is a list of cavity descriptions (grid, geometry, Re, n, lid
speed). Nothing here computes any part of the method; the seeded random
draws of the batched sweep are plain NumPy generator calls.

* cavity65   65 x 65, theta = 60 deg, n = 0.75, Re = 100 (the plain FP64
             validation case; Sec. 5.1 parameters c = 1, CFL = 0.5, U = 0.1)
* sweep257   the power-law sweep: 257 x 257, theta = 60 deg,
             n in {0.5, 0.75, 1.0, 1.25, 1.5} x Re in {100, 1000}
             (10 cavities advanced together; the paper's production grid
             is 256^2 cells, Sec. 5.3)
* unsteady1025  1025 x 1025, theta = 75 deg, n = 0.75, Re in {3000, 5000, 8000}
* batch64    64 cavities, N in {129, 257, 385, 513}, theta in
             {30, 45, 60, 75, 90} deg, n ~ U[0.5, 1.5], Re in {100, 400, 1000},
             drawn with numpy.random.default_rng(230607603) in that order
* adjoint257 257 x 257, theta = 60 deg, n = 0.75, Re = 400
* roof2049 / roof4097  one large cavity for HBM-roofline measurements
* quad257    10 cavities of 257 x 257 on general quadrilaterals (per-node
             metrics): the unit square's corners moved by U[-0.2, 0.2] in x and
             y, drawn with numpy.random.default_rng(230607604), n and Re as in
             sweep257
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class CavitySpec:
    nx: int
    ny: int
    Re: float
    n: float
    theta_deg: float = 60.0
    U_lid: float = 0.1
    L: float = 1.0
    H: float = 1.0

    @property
    def nodes(self) -> int:
        return self.nx * self.ny


@dataclass(frozen=True)
class QuadSpec:
    """A cavity on a general quadrilateral: corners ((x, y) bottom-left,
    bottom-right, top-left, top-right); the lid is the top edge."""
    nx: int
    ny: int
    corners: tuple
    Re: float
    n: float
    U_lid: float = 0.1
    H: float = 1.0

    @property
    def nodes(self) -> int:
        return self.nx * self.ny


def cavity65():
    return [CavitySpec(65, 65, 100.0, 0.75, 60.0)]


def sweep257():
    return [CavitySpec(257, 257, Re, n, 60.0) for n in (0.5, 0.75, 1.0, 1.25, 1.5)
            for Re in (100.0, 1000.0)]


def unsteady1025():
    return [CavitySpec(1025, 1025, Re, 0.75, 75.0) for Re in (3000.0, 5000.0, 8000.0)]


def batch64(seed=230607603):
    rng = np.random.default_rng(seed)
    N = rng.choice([129, 257, 385, 513], size=64)
    theta = rng.choice([30.0, 45.0, 60.0, 75.0, 90.0], size=64)
    n = rng.uniform(0.5, 1.5, size=64)
    Re = rng.choice([100.0, 400.0, 1000.0], size=64)
    return [CavitySpec(int(N[k]), int(N[k]), float(Re[k]), float(n[k]), float(theta[k]))
            for k in range(64)]


def adjoint257():
    return [CavitySpec(257, 257, 400.0, 0.75, 60.0)]


def quad257(seed=230607604):
    rng = np.random.default_rng(seed)
    out = []
    for n in (0.5, 0.75, 1.0, 1.25, 1.5):
        for Re in (100.0, 1000.0):
            d = rng.uniform(-0.2, 0.2, size=(4, 2))
            c = tuple((float(x0 + d[k, 0]), float(y0 + d[k, 1]))
                      for k, (x0, y0) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))))
            out.append(QuadSpec(257, 257, c, Re, n))
    return out


def roof(N):
    return [CavitySpec(N, N, 1000.0, 0.75, 60.0)]


# Library options a workload needs beyond the defaults (none at present:
# the default contravariant Courant rule for dt covers every workload).
WORKLOAD_OPTIONS = {}

WORKLOADS = {
    "cavity65": cavity65,
    "sweep257": sweep257,
    "unsteady1025": unsteady1025,
    "batch64": batch64,
    "adjoint257": adjoint257,
    "roof2049": lambda: roof(2049),
    "roof4097": lambda: roof(4097),
    "quad257": quad257,
}


def smooth_noise(shape, seed, modes=4, amplitude=1.0):
    """Seeded smooth random field: a sum of a few random Fourier modes."""
    rng = np.random.default_rng(seed)
    ny, nx = shape[-2], shape[-1]
    y = np.linspace(0.0, 1.0, ny)[:, None]
    x = np.linspace(0.0, 1.0, nx)[None, :]
    out = np.zeros(shape)
    for idx in np.ndindex(*shape[:-2]):
        f = np.zeros((ny, nx))
        for _ in range(modes):
            kx, ky = rng.integers(1, 4, size=2)
            ph = rng.uniform(0, 2 * np.pi, size=2)
            f += rng.standard_normal() * np.sin(np.pi * kx * x + ph[0]) * np.sin(np.pi * ky * y + ph[1])
        out[idx] = amplitude * f / modes
    return out
