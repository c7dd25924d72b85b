"""Seeded synthetic inputs for the projection step (Sec. 5.4 of the paper).

This module holds no arithmetic of the method itself: it only draws the fields
the projection consumes -- the predicted velocity u*, v*, w* on the staggered
MAC faces (Sec. 5, uniform staggered Cartesian mesh), the divergence source
S = div u^{n+1} of Eq. (31), the one-fluid density rho^{n+1} and the two old
pressures p^n, p^{n-1} that enter p_hat = 2p^n - p^{n-1} of Eq. (32).  Both the
oracle and the CUDA path receive exactly these arrays.

Layout (C order, x fastest):
  cell fields   [Nz][Ny][Nx]      index (k*Ny + j)*Nx + i
  u  (x-faces)  [Nz][Ny][Nx]      face i sits between cells i-1 and i (periodic)
  v  (y-faces)  [Nz][Ny+1][Nx]    face j between cells j-1 and j; j=0, Ny are walls
  w  (z-faces)  [Nz][Ny][Nx]      face k between cells k-1 and k (periodic)

Recipes (the paper's jets, periodic in x and z with walls in y, stand-in):
  * interface height eta(x, z): either pi + 0.1 sin(2x) cos(z) ("single") or
    pi + sum_{m=1..8} 0.05 cos(kx_m x + kz_m z + phi_m) with (kx_m, kz_m) drawn
    from {0..8}^2 \\ {(0,0)} and phi_m ~ U[0, 2pi) ("multimode");
  * rho = rho_g + (rho_l - rho_g) * 0.5 * (1 - tanh(2 (y - eta) / (w dy))) at
    cell centres: liquid below eta, a tanh layer about w cells wide;
  * u*, v*, w* ~ N(0, 1), v* = 0 on the two wall planes (no penetration);
  * S ~ N(0, 0.1) on cells with |y_j - eta(x_i, z_k)| <= 3 dy, zero elsewhere,
    its mean over those support cells removed (so mean(S) = 0 over the grid);
  * p^n, p^{n-1} ~ N(0, 1), each minus its own mean;
  * dt = 1e-3.

Random draws come from numpy.random.default_rng(seed) in this fixed order:
(multimode: kx_m, kz_m, phi_m), u, v, w, S, p^n, p^{n-1}.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass
class Fields:
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    S: np.ndarray
    rho: np.ndarray
    p_n: np.ndarray
    p_nm1: np.ndarray
    dt: float
    recipe: str
    seed: int

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    def arrays(self):
        return dict(u=self.u, v=self.v, w=self.w, S=self.S, rho=self.rho,
                    p_n=self.p_n, p_nm1=self.p_nm1)


def _centres(n: int, length: float) -> np.ndarray:
    h = length / n
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def _modes(rng: np.random.Generator, count: int = 8):
    kx = np.empty(count, dtype=np.int64)
    kz = np.empty(count, dtype=np.int64)
    for m in range(count):
        while True:
            a, b = rng.integers(0, 9, size=2)
            if a != 0 or b != 0:
                break
        kx[m], kz[m] = a, b
    phi = rng.uniform(0.0, TWO_PI, size=count)
    return kx, kz, phi


def make_fields(nx: int, ny: int, nz: int, *, seed: int = 0, recipe: str = "single",
                width: float = 2.0, rho_l: float = 640.0, rho_g: float = 120.0,
                lx: float = TWO_PI, ly: float = TWO_PI, lz: float = TWO_PI,
                dt: float = 1e-3) -> Fields:
    """Draw one synthetic projection problem (see the module docstring)."""
    rng = np.random.default_rng(seed)
    x = _centres(nx, lx)[None, None, :]
    y = _centres(ny, ly)[None, :, None]
    z = _centres(nz, lz)[:, None, None]
    dy = ly / ny
    if recipe == "single":
        eta = math.pi + 0.1 * np.sin(2.0 * x) * np.cos(z)
    elif recipe == "multimode":
        kx, kz, phi = _modes(rng)
        eta = np.full((nz, 1, nx), math.pi)
        for m in range(len(kx)):
            eta = eta + 0.05 * np.cos(kx[m] * x + kz[m] * z + phi[m])
    else:
        raise ValueError(f"unknown recipe {recipe!r}")
    rho = rho_g + (rho_l - rho_g) * 0.5 * (1.0 - np.tanh(2.0 * (y - eta) / (width * dy)))
    rho = np.array(np.broadcast_to(rho, (nz, ny, nx)), dtype=np.float64)  # owned, writable copy

    u = rng.standard_normal((nz, ny, nx))
    v = rng.standard_normal((nz, ny + 1, nx))
    v[:, 0, :] = 0.0
    v[:, ny, :] = 0.0
    w = rng.standard_normal((nz, ny, nx))

    support = np.abs(np.broadcast_to(y, (nz, ny, nx)) - eta) <= 3.0 * dy
    S = np.where(support, 0.1 * rng.standard_normal((nz, ny, nx)), 0.0)
    n_sup = int(support.sum())
    if n_sup:
        S = np.where(support, S - S[support].mean(), 0.0)

    p_n = rng.standard_normal((nz, ny, nx))
    p_n -= p_n.mean()
    p_nm1 = rng.standard_normal((nz, ny, nx))
    p_nm1 -= p_nm1.mean()
    return Fields(nx, ny, nz, lx, ly, lz, u, v, w, np.ascontiguousarray(S), rho,
                  p_n, p_nm1, dt, recipe, seed)


# The five workloads, by what they are.
def small_single_interface(seed: int = 0) -> Fields:
    """32^3, single-mode interface, tanh width 2 cells, density 640/120."""
    return make_fields(32, 32, 32, seed=seed, recipe="single", width=2.0)


def multimode_128(seed: int = 1) -> Fields:
    """128^3, 8 seeded interface modes, 6-cell layer, density 640/120."""
    return make_fields(128, 128, 128, seed=seed, recipe="multimode", width=6.0)


def multimode_256(seed: int = 2, rho_g: float = 60.0) -> Fields:
    """256^3, 8 seeded interface modes, 6-cell layer, density 640/60."""
    return make_fields(256, 256, 256, seed=seed, recipe="multimode", width=6.0, rho_g=rho_g)


BATCH_DIMS = (32, 48, 64, 96, 128, 192)


def batch_shapes(count: int = 64, seed: int = 3):
    """Grid shapes (nx, ny, nz) for the uneven batch, each dimension drawn from
    {32, 48, 64, 96, 128, 192}."""
    rng = np.random.default_rng(seed)
    dims = np.asarray(BATCH_DIMS)
    return [tuple(int(d) for d in rng.choice(dims, size=3)) for _ in range(count)]


def smooth_field(nx: int, ny: int, nz: int, *, seed: int = 0, modes: int = 4, amplitude: float = 1.0,
                 lx: float = TWO_PI, lz: float = TWO_PI) -> np.ndarray:
    """A smooth zero-mean cell field: `modes` products of a Fourier mode in x and
    z (wavenumbers 1..3) and a cosine mode in y (1..3) with random phases and
    N(0, 1) weights, scaled to max |.| = amplitude.  A stand-in for a pressure
    field that varies slowly in space (the time signal of the split study)."""
    rng = np.random.default_rng(seed)
    x = _centres(nx, lx)[None, None, :]
    zc = _centres(nz, lz)[:, None, None]
    jj = (np.arange(ny, dtype=np.float64) + 0.5)[None, :, None]
    out = np.zeros((nz, ny, nx))
    for _ in range(modes):
        a, b, c = rng.integers(1, 4, size=3)
        px, pz = rng.uniform(0.0, TWO_PI, size=2)
        out += rng.standard_normal() * (np.cos(TWO_PI * a * x / lx + px) * np.cos(math.pi * b * jj / ny)
                                        * np.cos(TWO_PI * c * zc / lz + pz))
    out -= out.mean()
    return amplitude * out / np.abs(out).max()
