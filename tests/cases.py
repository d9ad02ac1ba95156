"""Seeded cases shared by the tests: each builds inputs with paper_2201_06914_gb300.inputs
and can run either the CPU oracle or (in GPU tests) the CUDA path on them."""
from __future__ import annotations

import dataclasses

import numpy as np

from paper_2201_06914_gb300 import inputs as I


@dataclasses.dataclass
class Case:
    ndim: int
    nx: int
    ny: int
    nz: int
    nbl: int
    nt: int
    h: float
    dt: float
    f0: float
    damp_v: float
    m_true: np.ndarray     # padded float32
    m0: np.ndarray         # padded float32
    src: np.ndarray        # (S, nsrc, 3)
    rec: np.ndarray        # (S, nrec, 3)
    wavelet: np.ndarray    # (nt,) float64

    @property
    def shape(self):
        nb = 2 * self.nbl
        return (self.nz + nb, self.nx + nb) if self.ndim == 2 else \
            (self.nz + nb, self.ny + nb, self.nx + nb)

    @property
    def N(self):
        return int(np.prod(self.shape))

    @property
    def nshots(self):
        return self.src.shape[0]

    def oracle_grid(self):
        from oracle.oracle import Grid
        return Grid(self.ndim, self.nx, self.ny, self.nz, self.nbl, self.nt, self.h, self.h,
                    self.h, self.dt, self.damp_v)


def layered_case(ndim=2, nx=67, ny=1, nz=45, nbl=10, nt=240, h=10.0, f0=15.0, nshots=1,
                 nrec=None, off_grid=False, seed=0, salt=False, zi=0.55, background="smooth"):
    """Two-layer (or layered + salt) model, interface at depth fraction `zi`; background
    either the smoothed true model or the constant top velocity; sources near the top."""
    shape = (nz, nx) if ndim == 2 else (nz, ny, nx)
    if salt:
        v = I.layered_salt(shape, h, seed=seed + 1, v_min=1500.0, v_max=3000.0, nlayers=4,
                           pert_sigma=3 * h, salt_v=3200.0, v_cap=3300.0)
    else:
        z = np.arange(nz) * h
        v = np.where(z >= zi * (nz - 1) * h, 2500.0, 1500.0)
        v = v.reshape((nz,) + (1,) * (ndim - 1)) * np.ones(shape)
    v0 = I.smoothed(v, 3 * h, h) if background == "smooth" else np.full_like(v, v.min())
    dt = 0.4 * h / v.max()
    m_true = I.pad_edge(I.slowness_squared(v), nbl).astype(np.float32)
    m0 = I.pad_edge(I.slowness_squared(v0), nbl).astype(np.float32)
    rng = np.random.default_rng(seed)
    xs = np.linspace(0.2, 0.8, nshots) * (nx - 1) * h if nshots > 1 else np.array([0.5 * (nx - 1) * h])
    ys = np.full(nshots, 0.5 * (ny - 1) * h if ndim == 3 else 0.0)
    zs = np.full(nshots, 2 * h)
    if off_grid:
        xs = xs + rng.uniform(0.1, 0.9, nshots) * h
        zs = zs + rng.uniform(0.1, 0.9, nshots) * h
        if ndim == 3:
            ys = ys + rng.uniform(0.1, 0.9, nshots) * h
    src = np.stack([xs, ys, zs], axis=1)[:, None, :]
    if ndim == 2:
        nr = nrec or nx
        rx = np.linspace(0, (nx - 1) * h, nr)
        rec = np.stack([rx, np.zeros(nr), np.full(nr, 2 * h + (0.37 * h if off_grid else 0))], 1)
    else:
        gx, gy = np.meshgrid(np.arange(0, nx, 3) * h, np.arange(0, ny, 3) * h)
        rec = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 2 * h + (0.37 * h if off_grid else 0))], 1)
    rec = np.ascontiguousarray(np.broadcast_to(rec, (nshots,) + rec.shape))
    w = I.ricker(nt, dt, f0)
    return Case(ndim, nx, ny, nz, nbl, nt, h, dt, f0, float(v.max()), m_true, m0, src, rec, w)


def oracle_shot(case, s, m, Q=None, want_udd=False):
    from oracle import oracle as O
    return O.forward(case.oracle_grid(), m.astype(np.float64), case.src[s], case.wavelet,
                     case.rec[s], Q=Q, want_udd=want_udd)


def oracle_data(case, which="true"):
    m = case.m_true if which == "true" else case.m0
    return np.stack([oracle_shot(case, s, m)["d"] for s in range(case.nshots)])


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def relmax(a, b):
    """Largest pointwise difference relative to the largest reference value: a localised
    error (one tile edge, one source cell) that the L2 norm would average away."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def close(a, b, tol):
    """Relative L2 and per-element relative maximum both within tol; returns both (for the
    assertion message)."""
    e2, em = rel(a, b), relmax(a, b)
    return e2 < tol and em < tol, (e2, em)


def tti_case(ndim=2, nx=31, ny=1, nz=27, nbl=6, nt=120, h=10.0, f0=20.0, nshots=1, seed=0,
             scale=1.0, off_grid=True):
    """Layered case plus smooth Thomsen fields (scaled by `scale`; 0 gives isotropy)."""
    from oracle.oracle import Thomsen
    base = layered_case(ndim=ndim, nx=nx, ny=ny, nz=nz, nbl=nbl, nt=nt, h=h, f0=f0,
                        nshots=nshots, off_grid=off_grid, seed=seed, zi=0.35,
                        background="const")
    shape = base.m0.shape
    inner = (nz, nx) if ndim == 2 else (nz, ny, nx)
    e, d, t, p = I.tti_fields(inner, h, sigma=3 * h)
    fields = [I.pad_edge(f * scale, nbl) for f in (e, d, t, p)]
    th = Thomsen(*fields)
    # stability of the anisotropic operator: dt from v_max * sqrt(1 + 2 eps_max)
    vmax = base.damp_v * np.sqrt(1 + 2 * fields[0].max())
    dt = 0.4 * h / vmax
    base.dt = dt
    base.wavelet = I.ricker(nt, dt, f0)
    assert fields[0].shape == shape
    return base, th
