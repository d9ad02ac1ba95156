"""Python wrapper of the FP64 CPU oracle (oracle/wp_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
leg are the only callers.  The product path (paper_2201_06914_gb300) never imports this
module, and this module imports nothing from the product package.

Every function follows the paper's notation: u_tt the second time derivative of the
forward wavefield, v the adjoint wavefield, Q the probing matrix (nt x r), Pu = Q^T u_tt
and Pv = Q^T v the probed projections (Eq. 3), dm = sum_t u_tt[t] v[t] the exact gradient
(Eq. 2).  The discrete scheme and its readings are described at the top of wp_oracle.c.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, IEEE FP64, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("nbl", ctypes.c_int), ("nt", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("dt", ctypes.c_double), ("damp_v", ctypes.c_double)]


@dataclasses.dataclass
class Grid:
    """Padded-grid description: interior sizes, absorbing width, spacing, dt, nt and the
    velocity that sets the absorbing-layer strength."""
    ndim: int
    nx: int
    ny: int
    nz: int
    nbl: int
    nt: int
    dx: float
    dy: float
    dz: float
    dt: float
    damp_v: float

    @property
    def shape(self):
        nb = 2 * self.nbl
        if self.ndim == 2:
            return (self.nz + nb, self.nx + nb)
        return (self.nz + nb, self.ny + nb, self.nx + nb)

    @property
    def npoints(self):
        return int(np.prod(self.shape))

    def c(self):
        return _Grid(self.ndim, self.nx, self.ny if self.ndim == 3 else 1, self.nz, self.nbl,
                     self.nt, self.dx, self.dy, self.dz, self.dt, self.damp_v)


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        g = ctypes.POINTER(_Grid)
        _lib.orc_forward.argtypes = [g, d, ctypes.c_int, d, d, d, ctypes.c_int, d, d,
                                     ctypes.c_int, d, d, d, d]
        _lib.orc_adjoint.argtypes = [g, d, ctypes.c_int, d, d, ctypes.c_int, d, d, d, d, d,
                                     ctypes.c_int, d, d]
        _lib.orc_sponge.argtypes = [g, d]
        _lib.orc_weights.argtypes = [g, d, ctypes.POINTER(ctypes.c_long), d]
        _lib.orc_probed_image.argtypes = [ctypes.c_long, ctypes.c_int, d, d, ctypes.c_double, d]
        _lib.orc_apply_laplacian.argtypes = [g, d, d]
        _lib.orc_apply_hz.argtypes = [g, d, d, d, d]
        _lib.orc_tti_forward.argtypes = [g, d, d, d, d, d, ctypes.c_int, d, d, d, ctypes.c_int,
                                         d, d, ctypes.c_int, d, d, d]
        _lib.orc_tti_adjoint.argtypes = [g, d, d, d, d, d, ctypes.c_int, d, d, ctypes.c_int, d,
                                         d, d, d, ctypes.c_int, d, d]
        _lib.orc_npoints.argtypes = [g]
        _lib.orc_npoints.restype = ctypes.c_long
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def sponge(grid: Grid) -> np.ndarray:
    out = np.empty(grid.npoints)
    _L().orc_sponge(ctypes.byref(grid.c()), _p(out))
    return out.reshape(grid.shape)


def laplacian(grid: Grid, u):
    """8th-order Laplacian of a padded field (zero values beyond the grid)."""
    u = _f64(u)
    out = np.empty_like(u)
    _L().orc_apply_laplacian(ctypes.byref(grid.c()), _p(u), _p(out))
    return out


def history_bytes(npoints, nt, bytes_per_value=4, fields=1):
    """Memory of the full forward time history that the adjoint-state imaging condition
    (Eq. 2) correlates with the adjoint wavefield: nt snapshots of every field."""
    return nt * npoints * bytes_per_value * fields


def probe_bytes(npoints, r, bytes_per_value=4, fields=1):
    """Memory of the probed forward wavefield of Eq. 3: r projections per field instead of
    nt snapshots (Sec. 2.2, "storage of the compressed wavefields for only r << nt")."""
    return r * npoints * bytes_per_value * fields


def weights(grid: Grid, xyz) -> tuple[np.ndarray, np.ndarray]:
    idx = (ctypes.c_long * 8)()
    w = np.zeros(8)
    nc = _L().orc_weights(ctypes.byref(grid.c()), _p(_f64(xyz)), idx, _p(w))
    if nc < 0:
        raise ValueError("point outside the grid")
    return np.array(idx[:nc]), w[:nc]


def forward(grid: Grid, m, src, wavelet, rec, Q=None, want_udd=False, want_u=False,
            vol_src=None):
    """One shot: returns dict(d=(nt, nrec), Pu=(r, *shape) or None, udd, u)."""
    m = _f64(m).ravel()
    src = _f64(np.reshape(src, (-1, 3)))
    rec = _f64(np.reshape(rec, (-1, 3)))
    N, nt = grid.npoints, grid.nt
    d = np.zeros((nt, rec.shape[0]))
    r = 0 if Q is None else Q.shape[1]
    Q = _f64(Q)
    Pu = np.zeros((r, N)) if r else None
    udd = np.zeros((nt, N)) if want_udd else None
    uh = np.zeros((nt + 1, N)) if want_u else None
    rc = _L().orc_forward(ctypes.byref(grid.c()), _p(m), src.shape[0], _p(src),
                          _p(_f64(wavelet)), _p(_f64(vol_src)), rec.shape[0], _p(rec), _p(d),
                          r, _p(Q), _p(Pu), _p(udd), _p(uh))
    if rc:
        raise ValueError("source or receiver outside the grid")
    sh = grid.shape
    return dict(d=d, Pu=None if Pu is None else Pu.reshape((r,) + sh),
                udd=None if udd is None else udd.reshape((nt,) + sh),
                u=None if uh is None else uh.reshape((nt + 1,) + sh))


def adjoint(grid: Grid, m, rec, res, Q=None, udd=None, want_v=False, points=None):
    """One shot: returns dict(Pv, g (exact gradient, needs udd), v, vpt)."""
    m = _f64(m).ravel()
    rec = _f64(np.reshape(rec, (-1, 3)))
    N, nt = grid.npoints, grid.nt
    r = 0 if Q is None else Q.shape[1]
    Q = _f64(Q)
    Pv = np.zeros((r, N)) if r else None
    g = np.zeros(N) if udd is not None else None
    vh = np.zeros((nt, N)) if want_v else None
    pts = None if points is None else _f64(np.reshape(points, (-1, 3)))
    npt = 0 if pts is None else pts.shape[0]
    vpt = np.zeros((nt, npt)) if npt else None
    rc = _L().orc_adjoint(ctypes.byref(grid.c()), _p(m), rec.shape[0], _p(rec),
                          _p(_f64(res)), r, _p(Q), _p(Pv),
                          _p(None if udd is None else _f64(udd).reshape(-1)), _p(g), _p(vh),
                          npt, _p(pts), _p(vpt))
    if rc:
        raise ValueError("receiver or sample point outside the grid")
    sh = grid.shape
    return dict(Pv=None if Pv is None else Pv.reshape((r,) + sh),
                g=None if g is None else g.reshape(sh),
                v=None if vh is None else vh.reshape((nt,) + sh), vpt=vpt)


def probed_image(Pu, Pv, scale):
    """Eq. 3: scale * sum_i Pu[i] * Pv[i]."""
    r = Pu.shape[0]
    Pu = _f64(Pu)
    Pv = _f64(Pv)
    N = Pu.size // max(r, 1)
    out = np.zeros(N)
    _L().orc_probed_image(N, r, _p(Pu), _p(Pv), float(scale), _p(out))
    return out.reshape(Pu.shape[1:])


def range_finder(A, Z):
    """Sec. 2.1: [Q, ~] = qr(A Z), the orthonormal basis of the sketch A Z (columns of Q
    with the signs that make diag(R) non-negative).  A: (nt, nt) matrix, Z: (nt, r)."""
    Y = np.asarray(A, np.float64) @ np.asarray(Z, np.float64)
    Q, R = np.linalg.qr(Y)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d


def offset_image(Pu, Pv, nh, scale):
    """Eq. 4, the subsurface-offset image volume from the probed projections:
        out[h + nh][..., x] = scale * sum_i Pu[i][..., x + h] * Pv[i][..., x - h],
    h = -nh .. nh along x (the last axis), zero where x + h or x - h leaves the row.
    Pu, Pv: (r, *shape).  With Pu, Pv the full histories (u_tt and v, i.e. Q = I) and
    scale 1 this is the exact offset image sum_t u_tt[t][x + h] v[t][x - h]."""
    Pu = np.asarray(Pu, np.float64)
    Pv = np.asarray(Pv, np.float64)
    nx = Pu.shape[-1]
    out = np.zeros((2 * nh + 1,) + Pu.shape[1:])
    for h in range(-nh, nh + 1):
        lo, hi = max(0, -h, h), min(nx, nx - h, nx + h)   # x with x+h and x-h in [0, nx)
        if lo >= hi:
            continue
        prod = Pu[..., lo + h:hi + h] * Pv[..., lo - h:hi - h]
        out[h + nh][..., lo:hi] = scale * prod.sum(axis=0)
    return out


def misfit(d, d_obs):
    """J = 1/2 sum_t |R u[t] - d_obs[t]|^2 (no time-step weighting)."""
    return 0.5 * float(np.sum((np.asarray(d, np.float64) - d_obs) ** 2))


def exact_gradient(grid: Grid, m, src, wavelet, rec, d_obs):
    """Full-history adjoint-state gradient of one shot (Eq. 2): returns (J, g, fwd)."""
    f = forward(grid, m, src, wavelet, rec, want_udd=True)
    res = f["d"] - d_obs
    a = adjoint(grid, m, rec, res, udd=f["udd"])
    return misfit(f["d"], d_obs), a["g"], f


def probed_gradient(grid: Grid, m, src, wavelet, rec, d_obs, Q, scale):
    """Probed gradient of one shot (Eq. 3): forward with Pu, adjoint with Pv, image.
    Returns dict(J, g_hat, Pu, Pv, d)."""
    f = forward(grid, m, src, wavelet, rec, Q=Q)
    res = f["d"] - d_obs
    a = adjoint(grid, m, rec, res, Q=Q)
    return dict(J=misfit(f["d"], d_obs), g_hat=probed_image(f["Pu"], a["Pv"], scale),
                Pu=f["Pu"], Pv=a["Pv"], d=f["d"])


# ----------------------------------------------------------------------------------------
# Pseudo-acoustic TTI (see the TTI block of wp_oracle.c for the reading of the equations)
# ----------------------------------------------------------------------------------------
@dataclasses.dataclass
class Thomsen:
    """Padded Thomsen fields: epsilon, delta, tilt theta and azimuth phi (radians)."""
    eps: np.ndarray
    delta: np.ndarray
    theta: np.ndarray
    phi: np.ndarray

    def ptrs(self):
        self._keep = [_f64(a).ravel() for a in (self.eps, self.delta, self.theta, self.phi)]
        return [_p(a) for a in self._keep]


def apply_hz(grid: Grid, theta, phi, w):
    """Hz w = -Dr^T Dr w for the tilted-axis first derivative Dr."""
    w = _f64(w)
    out = np.empty_like(w)
    _L().orc_apply_hz(ctypes.byref(grid.c()), _p(_f64(theta)), _p(None if phi is None else _f64(phi)),
                      _p(w), _p(out))
    return out


def tti_forward(grid: Grid, m, th: Thomsen, src, wavelet, rec, Q=None, want_udd=False,
                vol_src=None):
    """One TTI shot: d (nt, nrec) of the p field, Pu (2, r, *shape), udd (nt, 2, *shape)."""
    m = _f64(m).ravel()
    src = _f64(np.reshape(src, (-1, 3)))
    rec = _f64(np.reshape(rec, (-1, 3)))
    N, nt = grid.npoints, grid.nt
    d = np.zeros((nt, rec.shape[0]))
    r = 0 if Q is None else Q.shape[1]
    Q = _f64(Q)
    Pu = np.zeros((2, r, N)) if r else None
    udd = np.zeros((nt, 2, N)) if want_udd else None
    e, dl, t, ph = th.ptrs()
    rc = _L().orc_tti_forward(ctypes.byref(grid.c()), _p(m), e, dl, t, ph, src.shape[0], _p(src),
                              _p(_f64(wavelet)), _p(_f64(vol_src)), rec.shape[0], _p(rec), _p(d),
                              r, _p(Q), _p(Pu), _p(udd))
    if rc:
        raise ValueError("source or receiver outside the grid")
    sh = grid.shape
    return dict(d=d, Pu=None if Pu is None else Pu.reshape((2, r) + sh),
                udd=None if udd is None else udd.reshape((nt, 2) + sh))


def tti_adjoint(grid: Grid, m, th: Thomsen, rec, res, Q=None, udd=None, points=None):
    """One TTI shot adjoint: Pv (2, r, *shape), g (exact, needs udd), vpt (nt, npt, 2)."""
    m = _f64(m).ravel()
    rec = _f64(np.reshape(rec, (-1, 3)))
    N, nt = grid.npoints, grid.nt
    r = 0 if Q is None else Q.shape[1]
    Q = _f64(Q)
    Pv = np.zeros((2, r, N)) if r else None
    g = np.zeros(N) if udd is not None else None
    pts = None if points is None else _f64(np.reshape(points, (-1, 3)))
    npt = 0 if pts is None else pts.shape[0]
    vpt = np.zeros((nt, npt, 2)) if npt else None
    e, dl, t, ph = th.ptrs()
    rc = _L().orc_tti_adjoint(ctypes.byref(grid.c()), _p(m), e, dl, t, ph, rec.shape[0], _p(rec),
                              _p(_f64(res)), r, _p(Q), _p(Pv),
                              _p(None if udd is None else _f64(udd).reshape(-1)), _p(g), npt,
                              _p(pts), _p(vpt))
    if rc:
        raise ValueError("receiver or sample point outside the grid")
    sh = grid.shape
    return dict(Pv=None if Pv is None else Pv.reshape((2, r) + sh),
                g=None if g is None else g.reshape(sh), vpt=vpt)


def tti_exact_gradient(grid: Grid, m, th: Thomsen, src, wavelet, rec, d_obs):
    f = tti_forward(grid, m, th, src, wavelet, rec, want_udd=True)
    a = tti_adjoint(grid, m, th, rec, f["d"] - d_obs, udd=f["udd"])
    return misfit(f["d"], d_obs), a["g"], f


def tti_probed_gradient(grid: Grid, m, th: Thomsen, src, wavelet, rec, d_obs, Q, scale):
    """Eq. 3 summed over the two wavefields: scale * sum_f sum_i Pu[f,i] Pv[f,i]."""
    f = tti_forward(grid, m, th, src, wavelet, rec, Q=Q)
    a = tti_adjoint(grid, m, th, rec, f["d"] - d_obs, Q=Q)
    img = probed_image(f["Pu"][0], a["Pv"][0], scale) + probed_image(f["Pu"][1], a["Pv"][1], scale)
    return dict(J=misfit(f["d"], d_obs), g_hat=img, Pu=f["Pu"], Pv=a["Pv"], d=f["d"])
