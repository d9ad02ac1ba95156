"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle, the tests and the bench.

This module holds none of the imaging method's arithmetic: no stencil, sponge, injection,
probe projection or imaging condition.  It only builds what a user would hand to the
method: velocity models shaped like the paper's case studies (layered media with a smooth
random perturbation and a high-velocity salt body, Sec. 3 "Synthetic case studies"), TTI
Thomsen-parameter fields, source/receiver positions, the source wavelet, and the random
probing matrix Z whose entries the method draws (Rademacher +-1, Eq. 1 and the sentence
after it).  Random numbers come from SplitMix64 (Steele, Lea & Flood 2014), implemented
here from its published definition so that every consumer sees the same Z.

Grid convention used everywhere in this package: a model of `nx` (x), `ny` (y, 3-D only)
and `nz` (z, depth) interior points is padded by `nbl` absorbing cells on every side; the
padded field is stored with x fastest, then y, then z: index = (z*NY + y)*NX + x.
Coordinates are metres measured from the first interior point.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_MASK64 = (1 << 64) - 1


# ----------------------------------------------------------------------------------------
# SplitMix64 and Rademacher probes
# ----------------------------------------------------------------------------------------
def splitmix64(seed: int, n: int) -> np.ndarray:
    """First `n` outputs of SplitMix64 started from state `seed` (uint64).

    Published definition: state += 0x9E3779B97F4A7C15; z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) * 0x94D049BB133111EB;
    output z ^ (z >> 31); all arithmetic modulo 2^64.
    """
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def rademacher(seed: int, nt: int, r: int) -> np.ndarray:
    """Rademacher probing matrix Z (nt x r, float32 entries +-1), Eq. 1.

    Entry (t, i) takes the (t*r + i)-th SplitMix64 output of stream `seed`; bit 63 set
    gives -1, clear gives +1.  Independent shots use seed = base_seed + shot.
    """
    z = splitmix64(seed, nt * r)
    s = np.where((z >> np.uint64(63)) == 1, -1.0, 1.0).astype(np.float32)
    return s.reshape(nt, r)


def rademacher_shots(base_seed: int, nshots: int, nt: int, r: int) -> np.ndarray:
    """Independent probing matrices for `nshots` shots: (nshots, nt, r)."""
    return np.stack([rademacher(base_seed + s, nt, r) for s in range(nshots)])


# ----------------------------------------------------------------------------------------
# Source wavelet
# ----------------------------------------------------------------------------------------
def ricker(nt: int, dt: float, f0: float, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = t - t0,
    sampled at t = n*dt, n = 0..nt-1; t0 defaults to 1.5/f0."""
    if t0 is None:
        t0 = 1.5 / f0
    t = np.arange(nt, dtype=np.float64) * dt
    a = (math.pi * f0 * (t - t0)) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float64)


# ----------------------------------------------------------------------------------------
# Velocity models
# ----------------------------------------------------------------------------------------
def pad_edge(field: np.ndarray, nbl: int) -> np.ndarray:
    """Extend an interior model into the absorbing layer by repeating its edge values."""
    return np.pad(field, nbl, mode="edge")


def _smooth(field: np.ndarray, sigma_cells: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(field, sigma_cells, mode="nearest")


def two_layer(nz: int, nx: int, dz: float, v_top: float = 1500.0, v_bot: float = 2500.0,
              z_interface: float = 1000.0) -> np.ndarray:
    """Two-layer 2-D model (nz, nx): v_top above depth z_interface, v_bot at and below."""
    z = np.arange(nz) * dz
    v = np.where(z >= z_interface, v_bot, v_top)[:, None] * np.ones((1, nx))
    return v.astype(np.float64)


def layered_salt(shape: tuple, spacing: float, seed: int, v_min: float = 1500.0,
                 v_max: float = 4500.0, nlayers: int = 10, pert: float = 0.05,
                 pert_sigma: float = 200.0, salt_v: float = 4500.0, v_cap: float = 4725.0
                 ) -> np.ndarray:
    """Layered model with a smooth random perturbation and an elliptical salt body.

    `shape` is (nz, nx) or (nz, ny, nx), depth first.  Recipe: `nlayers` equal-thickness
    layers with velocities evenly spaced from v_min to v_max; times (1 + p) with p an
    N(0,1) field (seed `seed`) Gaussian-smoothed with sigma `pert_sigma` metres and scaled
    to max|p| = `pert`; an ellipse (ellipsoid) of velocity `salt_v` centred in the model
    with semi-axes 15 % of the lateral extents and 16 % of the depth extent; finally
    v <= v_cap.
    """
    shape = tuple(int(s) for s in shape)
    nz = shape[0]
    layer = np.minimum((np.arange(nz) * nlayers) // nz, nlayers - 1)
    vz = v_min + (v_max - v_min) * layer / (nlayers - 1)
    v = vz.reshape((nz,) + (1,) * (len(shape) - 1)) * np.ones(shape)
    rng = np.random.default_rng(seed)
    p = _smooth(rng.standard_normal(shape), pert_sigma / spacing)
    p *= pert / np.abs(p).max()
    v = v * (1.0 + p)
    grids = np.meshgrid(*[np.arange(n) * spacing for n in shape], indexing="ij")
    rad = 0.0
    for axis, g in enumerate(grids):
        extent = (shape[axis] - 1) * spacing
        semi = (0.16 if axis == 0 else 0.15) * extent
        rad = rad + ((g - 0.5 * extent) / semi) ** 2
    v = np.where(rad <= 1.0, salt_v, v)
    return np.minimum(v, v_cap)


def smoothed(v: np.ndarray, sigma: float, spacing: float) -> np.ndarray:
    """Gaussian-smoothed copy of a model (the background model of a gradient)."""
    return _smooth(v, sigma / spacing)


def tti_fields(shape: tuple, spacing: float, seeds=(2, 3, 4, 5), sigma: float = 200.0):
    """Thomsen epsilon in [0, 0.25], delta in [0, 0.1], tilt theta in [0, 40] deg and
    azimuth phi in [0, 90] deg (radians returned), each a smoothed uniform random field
    rescaled to its range; delta is then capped at epsilon.  The pseudo-acoustic system
    has a growing mode wherever delta > epsilon (its 2 x 2 symbol has determinant
    2 (eps - delta) |k_perp|^2 |k_par|^2), so models, like the BP 2007 TTI model, keep
    delta <= eps."""
    out = []
    for seed, (lo, hi) in zip(seeds, [(0.0, 0.25), (0.0, 0.1), (0.0, math.radians(40.0)),
                                      (0.0, math.radians(90.0))]):
        f = _smooth(np.random.default_rng(seed).random(shape), sigma / spacing)
        f = (f - f.min()) / max(f.max() - f.min(), 1e-30)
        out.append(lo + (hi - lo) * f)
    out[1] = np.minimum(out[1], out[0])
    return tuple(out)


def slowness_squared(v: np.ndarray) -> np.ndarray:
    """m = 1/v^2 (s^2/m^2), the model parameter of the gradient."""
    return 1.0 / (v.astype(np.float64) ** 2)


# ----------------------------------------------------------------------------------------
# Configurations shaped like the paper's workloads
# ----------------------------------------------------------------------------------------
@dataclasses.dataclass
class Survey:
    """One seeded workload: grid, models, wavelet and acquisition geometry."""
    name: str
    ndim: int
    nx: int
    ny: int
    nz: int
    spacing: float
    nbl: int
    nt: int
    dt: float
    f0: float
    v_true: np.ndarray        # interior, depth first
    v_background: np.ndarray  # interior, depth first
    src: np.ndarray           # (nshots, 3) metres (x, y, z)
    rec: np.ndarray           # (nshots, nrec, 3) metres
    r: int
    probe_seed: int = 0

    @property
    def shape_padded(self):
        if self.ndim == 2:
            return (self.nz + 2 * self.nbl, self.nx + 2 * self.nbl)
        return (self.nz + 2 * self.nbl, self.ny + 2 * self.nbl, self.nx + 2 * self.nbl)

    @property
    def npoints(self) -> int:
        return int(np.prod(self.shape_padded))

    @property
    def damp_v(self) -> float:
        """Velocity that sets the absorbing-layer strength (the true model's maximum)."""
        return float(self.v_true.max())

    @property
    def nshots(self) -> int:
        return int(self.src.shape[0])

    def m_padded(self, which: str = "background") -> np.ndarray:
        v = self.v_background if which == "background" else self.v_true
        return pad_edge(slowness_squared(v), self.nbl).astype(np.float32)

    def wavelet(self) -> np.ndarray:
        return ricker(self.nt, self.dt, self.f0)

    def probes(self, r: int | None = None) -> np.ndarray:
        return rademacher_shots(self.probe_seed, self.nshots, self.nt, r or self.r)


def _line(n, spacing, depth, nshots):
    x = np.arange(n) * spacing
    rec = np.stack([x, np.zeros(n), np.full(n, depth)], axis=1)
    return np.broadcast_to(rec, (nshots, n, 3)).copy()


def config_two_layer(nx=201, nz=201, nt=1000, nbl=40, r=8, nshots=1,
                     src_x: float | None = None) -> Survey:
    """2-D two-layer 1.5/2.5 km/s (interface 1 km), 10 m grid, 10 Hz Ricker at
    (1 km, 20 m), receivers every 10 m at 20 m depth, dt at CFL 0.4 of v_max."""
    dx = 10.0
    v = two_layer(nz, nx, dx)
    vb = np.full_like(v, 1500.0)
    dt = 0.4 * dx / v.max()
    if nshots == 1:
        xs = np.array([src_x if src_x is not None else min(1000.0, 0.5 * (nx - 1) * dx)])
    else:
        xs = np.linspace(0.0, (nx - 1) * dx, nshots + 2)[1:-1]
    src = np.stack([xs, np.zeros_like(xs), np.full_like(xs, 20.0)], axis=1)
    rec = _line(nx, dx, 20.0, len(xs))
    return Survey("two_layer_2d", 2, nx, 1, nz, dx, nbl, nt, dt, 10.0, v, vb, src, rec, r)


def config_salt_2d(nx=1601, nz=401, nt=4000, nbl=40, r=64, nshots=64) -> Survey:
    """2-D 1601x401 at 12.5 m, layered 1.5-4.5 km/s + 5 % smoothed perturbation + salt,
    15 Hz Ricker, 1601 receivers at 12.5 m depth, `nshots` shots evenly spaced in x."""
    dx = 12.5
    v = layered_salt((nz, nx), dx, seed=1)
    vb = smoothed(v, 400.0, dx)
    dt = 0.4 * dx / v.max()
    xs = (np.arange(nshots) + 0.5) * ((nx - 1) * dx / nshots)
    src = np.stack([xs, np.zeros_like(xs), np.full_like(xs, 12.5)], axis=1)
    rec = _line(nx, dx, 12.5, nshots)
    return Survey("salt_2d", 2, nx, 1, nz, dx, nbl, nt, dt, 15.0, v, vb, src, rec, r)


def config_salt_3d(nx=512, ny=512, nz=256, nt=2500, nbl=40, r=32, nshots=1,
                   rec_stride=2, dx=10.0, f0=12.0, eps_max=0.0) -> Survey:
    """3-D layered + salt model at `dx` (10 m), `f0` Ricker (12 Hz), receiver carpet every
    `rec_stride` cells at 20 m depth, one shot at the surface centre.  dt is at CFL 0.4 of
    the fastest velocity, sqrt(1 + 2 eps_max) faster for an anisotropic model."""
    v = layered_salt((nz, ny, nx), dx, seed=1)
    vb = smoothed(v, 400.0, dx)
    dt = 0.4 * dx / (v.max() * math.sqrt(1.0 + 2.0 * eps_max))
    src = np.array([[0.5 * (nx - 1) * dx, 0.5 * (ny - 1) * dx, 20.0]] * nshots)
    gx, gy = np.meshgrid(np.arange(0, nx, rec_stride) * dx, np.arange(0, ny, rec_stride) * dx)
    rec = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 20.0)], axis=1)
    rec = np.broadcast_to(rec, (nshots,) + rec.shape).copy()
    return Survey("salt_3d", 3, nx, ny, nz, dx, nbl, nt, dt, f0, v, vb, src, rec, r)
