"""Thin Python binding of libwp.so (include/wp.h): argument marshalling only.

Every function keeps the C name and forwards to the library; every step of the imaging
path runs in the library's CUDA kernels.  PyTorch supplies device memory and streams.
Importing this module loads the compiled library and raises if it is missing: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libwp.so")

WP_OK, WP_ERR_INVALID, WP_ERR_UNSTABLE, WP_ERR_OOM, WP_ERR_CUDA, WP_ERR_NONFINITE, \
    WP_ERR_TIMEOUT = range(7)
WP_PHYS_ISO, WP_PHYS_TTI = 0, 1
WP_MODE_PROBED, WP_MODE_EXACT_FULL, WP_MODE_EXACT_CHECKPOINT = 0, 1, 2
WP_PROBES_DENSE, WP_PROBES_ALIGNED = 0, 1
STATUS_NAMES = ["WP_OK", "WP_ERR_INVALID", "WP_ERR_UNSTABLE", "WP_ERR_OOM", "WP_ERR_CUDA",
                "WP_ERR_NONFINITE", "WP_ERR_TIMEOUT"]

EXPORTS = ["wp_model", "wp_model_free", "wp_model_npoints", "wp_model_vmax",
           "wp_workspace_bytes", "wp_probe_forward", "wp_adjoint_image", "wp_exact_gradient",
           "wp_residual", "wp_residual_workspace_bytes", "wp_probe_accumulate",
           "wp_probe_accumulate_workspace_bytes", "wp_stream_status", "wp_last_error",
           "wp_kernel_launches", "wp_profile_enable", "wp_profile_read",
           "wp_probe_accumulate_static", "wp_offset_image", "wp_check_bounded_wait",
           "wp_range_finder", "wp_range_finder_workspace_bytes", "wp_static_status",
           "wp_offset_status", "wp_set_probe_layout", "wp_probe_layout"]


class WpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class wp_model_desc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("nbl", ctypes.c_int), ("space_order", ctypes.c_int),
                ("physics", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("dt", ctypes.c_double), ("nt", ctypes.c_int),
                ("damp_v", ctypes.c_double), ("m", ctypes.c_void_p), ("eps", ctypes.c_void_p),
                ("delta", ctypes.c_void_p), ("theta", ctypes.c_void_p),
                ("phi", ctypes.c_void_p)]


class wp_geom(ctypes.Structure):
    _fields_ = [("nshots", ctypes.c_int), ("nsrc", ctypes.c_int), ("nrec", ctypes.c_int),
                ("src_xyz", ctypes.c_void_p), ("rec_xyz", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libwp.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, LL, D, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double, ctypes.c_size_t
    sig = {
        "wp_model": ([ctypes.POINTER(wp_model_desc), ctypes.POINTER(P)], I),
        "wp_model_free": ([P], None),
        "wp_model_npoints": ([P], LL),
        "wp_model_vmax": ([P], D),
        "wp_workspace_bytes": ([P, ctypes.POINTER(wp_geom), I, I, I], SZ),
        "wp_probe_forward": ([P, ctypes.POINTER(wp_geom), P, P, I, I, P, P, P, SZ, P], I),
        "wp_adjoint_image": ([P, ctypes.POINTER(wp_geom), P, P, I, I, ctypes.c_float, P, P, P,
                              P, SZ, P], I),
        "wp_exact_gradient": ([P, ctypes.POINTER(wp_geom), P, P, P, P, P, I, I, P, SZ, P], I),
        "wp_residual": ([P, P, P, LL, P, P, SZ, P], I),
        "wp_residual_workspace_bytes": ([LL], SZ),
        "wp_probe_accumulate": ([P, I, LL, I, P, I, I, I, ctypes.c_float, P, P, SZ, P], I),
        "wp_probe_accumulate_workspace_bytes": ([I, I, I], SZ),
        "wp_stream_status": ([P, P, D], I),
        "wp_last_error": ([], ctypes.c_char_p),
        "wp_kernel_launches": ([], LL),
        "wp_profile_enable": ([I, I], None),
        "wp_profile_read": ([I, ctypes.POINTER(D), ctypes.POINTER(LL)], I),
        "wp_probe_accumulate_static": ([P, I, LL, I, P, I, I, I, ctypes.c_float, P, P], I),
        "wp_offset_image": ([P, P, P, I, I, ctypes.c_float, I, P, P], I),
        "wp_check_bounded_wait": ([P, SZ, P], I),
        "wp_range_finder": ([P, I, I, I, I, I, P, I, P, P, SZ, P], I),
        "wp_range_finder_workspace_bytes": ([I, I, I, I, I], SZ),
        "wp_static_status": ([P, D], I),
        "wp_offset_status": ([P, D], I),
        "wp_set_probe_layout": ([P, I], I),
        "wp_probe_layout": ([P, ctypes.POINTER(I), ctypes.POINTER(LL), ctypes.POINTER(I)], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def _check(status):
    if status != WP_OK:
        raise WpError(status, _lib.wp_last_error().decode())


def _ptr(t, dtype="float32"):
    """Device address of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    want = {"float32": torch.float32, "float64": torch.float64, "uint8": torch.uint8}[dtype]
    if t.dtype != want:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return t.data_ptr()


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


# --------------------------------------------------------------------------------------
# Same-name wrappers of the C ABI
# --------------------------------------------------------------------------------------
def wp_last_error() -> str:
    return _lib.wp_last_error().decode()


def wp_kernel_launches() -> int:
    return int(_lib.wp_kernel_launches())


def wp_profile_enable(on: bool, capacity: int = 0) -> None:
    _lib.wp_profile_enable(1 if on else 0, int(capacity))


def wp_profile_read(cls: int):
    """(total_ms, count) of the recorded launches of a kernel class (0 one-step stencil,
    1 probe contraction, 2 other, 3 two-step stencil, 4 two-step exact imaging adjoint)."""
    t = ctypes.c_double()
    n = ctypes.c_longlong()
    if _lib.wp_profile_read(cls, ctypes.byref(t), ctypes.byref(n)) != 0:
        raise WpError(WP_ERR_CUDA, "wp_profile_read failed")
    return t.value, n.value


def wp_model(desc: wp_model_desc) -> int:
    h = ctypes.c_void_p()
    _check(_lib.wp_model(ctypes.byref(desc), ctypes.byref(h)))
    return h.value


def wp_model_free(handle) -> None:
    _lib.wp_model_free(handle)


def wp_model_npoints(handle) -> int:
    return int(_lib.wp_model_npoints(handle))


def wp_model_vmax(handle) -> float:
    return float(_lib.wp_model_vmax(handle))


def wp_set_probe_layout(handle, layout: int) -> None:
    _check(_lib.wp_set_probe_layout(handle, int(layout)))


def wp_probe_layout(handle):
    """(layout, floats between probe rows, x pitch) of the model's P_u / P_v layout."""
    lay, rf, xp = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_int()
    _check(_lib.wp_probe_layout(handle, ctypes.byref(lay), ctypes.byref(rf), ctypes.byref(xp)))
    return lay.value, rf.value, xp.value


def wp_workspace_bytes(handle, geom: wp_geom, r: int, Tb: int, mode: int) -> int:
    return int(_lib.wp_workspace_bytes(handle, ctypes.byref(geom), r, Tb, mode))


def wp_probe_forward(handle, geom, wavelet, Q, r, Tb, P_u, d_syn, ws, stream=None):
    _check(_lib.wp_probe_forward(handle, ctypes.byref(geom), _ptr(wavelet), _ptr(Q), r, Tb,
                                 _ptr(P_u), _ptr(d_syn), _ptr(ws, "uint8"), ws.numel(),
                                 _stream(stream)))


def wp_adjoint_image(handle, geom, residual, Q, r, Tb, scale, P_u, g, P_v, ws, stream=None):
    _check(_lib.wp_adjoint_image(handle, ctypes.byref(geom), _ptr(residual), _ptr(Q), r, Tb,
                                 float(scale), _ptr(P_u), _ptr(g), _ptr(P_v),
                                 _ptr(ws, "uint8"), ws.numel(), _stream(stream)))


def wp_exact_gradient(handle, geom, wavelet, d_obs, g, misfit, d_syn, mode, ncheck, ws,
                      stream=None):
    _check(_lib.wp_exact_gradient(handle, ctypes.byref(geom), _ptr(wavelet), _ptr(d_obs),
                                  _ptr(g), _ptr(misfit, "float64"), _ptr(d_syn), mode, ncheck,
                                  _ptr(ws, "uint8"), ws.numel(), _stream(stream)))


def wp_offset_image(handle, P_u, P_v, r, nshots, scale, nh, out, stream=None):
    """Subsurface-offset image volume (Eq. 4): out (2*nh+1, N) from P_u, P_v (nshots, r rows
    in the model's probe layout)."""
    _check(_lib.wp_offset_image(handle, _ptr(P_u), _ptr(P_v), r, nshots, scale, nh, _ptr(out),
                                _stream(stream)))


def wp_residual(d_syn, d_obs, res, n, misfit, ws, stream=None):
    _check(_lib.wp_residual(_ptr(d_syn), _ptr(d_obs), _ptr(res), n, _ptr(misfit, "float64"),
                            _ptr(ws, "uint8"), 0 if ws is None else ws.numel(),
                            _stream(stream)))


def wp_residual_workspace_bytes(n: int) -> int:
    return int(_lib.wp_residual_workspace_bytes(n))


def wp_probe_accumulate(A, cnt, npoints, nshots, Q, nt, t0, r, scale, P, ws, stream=None):
    _check(_lib.wp_probe_accumulate(_ptr(A), cnt, npoints, nshots, _ptr(Q), nt, t0, r,
                                    float(scale), _ptr(P), _ptr(ws, "uint8"), ws.numel(),
                                    _stream(stream)))


def wp_probe_accumulate_static(A, cnt, npoints, nshots, Q, nt, t0, r, scale, P, stream=None):
    """wp_probe_accumulate without a workspace: for callers that may not allocate device
    memory; the library's fixed 16 MiB device array holds the scratch (see include/wp.h)."""
    _check(_lib.wp_probe_accumulate_static(_ptr(A), cnt, npoints, nshots, _ptr(Q), nt, t0, r,
                                           float(scale), _ptr(P), _stream(stream)))


def wp_probe_accumulate_workspace_bytes(nshots: int, nt: int, r: int) -> int:
    return int(_lib.wp_probe_accumulate_workspace_bytes(nshots, nt, r))


def wp_range_finder_workspace_bytes(nt: int, ncols: int, nshots: int, d_shared: bool, r: int) -> int:
    return int(_lib.wp_range_finder_workspace_bytes(nt, ncols, nshots, int(bool(d_shared)), r))


def wp_range_finder(D, nt, ncols, nshots, d_shared, power, Z, r, Q, ws, stream=None):
    _check(_lib.wp_range_finder(_ptr(D), nt, ncols, nshots, int(bool(d_shared)), power, _ptr(Z), r,
                                _ptr(Q), _ptr(ws, "uint8"), ws.numel(), _stream(stream)))


def wp_offset_status(stream=None, timeout_s: float = 60.0) -> None:
    _check(_lib.wp_offset_status(_stream(stream), float(timeout_s)))


def wp_static_status(stream=None, timeout_s: float = 60.0) -> None:
    _check(_lib.wp_static_status(_stream(stream), float(timeout_s)))


def wp_check_bounded_wait(ws, stream=None) -> None:
    _check(_lib.wp_check_bounded_wait(_ptr(ws, "uint8"), ws.numel(), _stream(stream)))


def wp_stream_status(ws, stream=None, timeout_s: float = 60.0) -> None:
    _check(_lib.wp_stream_status(None if ws is None else _ptr(ws, "uint8"), _stream(stream),
                                 float(timeout_s)))


# --------------------------------------------------------------------------------------
# Marshalling helpers (no arithmetic of the method)
# --------------------------------------------------------------------------------------
class Model:
    """Owns a wp_model_t handle and keeps the borrowed device model alive."""

    def __init__(self, ndim, nx, ny, nz, nbl, dx, dy, dz, dt, nt, m, damp_v=0.0, eps=None,
                 delta=None, theta=None, phi=None):
        self.m = m
        self.tti = (eps, delta, theta, phi)   # kept alive while the handle exists
        phys = WP_PHYS_TTI if eps is not None else WP_PHYS_ISO
        self.desc = wp_model_desc(ndim, nx, ny if ndim == 3 else 1, nz, nbl, 8, phys,
                                  dx, dy, dz, dt, nt, damp_v, _ptr(m), _ptr(eps), _ptr(delta),
                                  _ptr(theta), _ptr(phi))
        self.handle = wp_model(self.desc)
        self.nt = nt
        self.N = wp_model_npoints(self.handle)

    @classmethod
    def from_survey(cls, survey, m):
        return cls(survey.ndim, survey.nx, survey.ny, survey.nz, survey.nbl, survey.spacing,
                   survey.spacing, survey.spacing, survey.dt, survey.nt, m, survey.damp_v)

    def use_aligned_probes(self) -> int:
        """Switch P_u / P_v of this handle to the row-aligned layout (no copy into the dense
        layout); returns the floats per probe row."""
        wp_set_probe_layout(self.handle, WP_PROBES_ALIGNED)
        return wp_probe_layout(self.handle)[1]

    def close(self):
        if self.handle:
            wp_model_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Geometry:
    """Host-side acquisition arrays kept alive for the wp_geom view."""

    def __init__(self, src, rec):
        self.src = np.ascontiguousarray(np.asarray(src, np.float64).reshape(-1, np.shape(src)[-2] if np.ndim(src) == 3 else 1, 3))
        self.rec = np.ascontiguousarray(np.asarray(rec, np.float64))
        nshots = self.src.shape[0]
        if self.rec.ndim == 2:
            self.rec = np.ascontiguousarray(np.broadcast_to(self.rec, (nshots,) + self.rec.shape))
        self.c = wp_geom(nshots, self.src.shape[1], self.rec.shape[1],
                         self.src.ctypes.data, self.rec.ctypes.data)

    @property
    def nshots(self):
        return self.c.nshots

    @property
    def nrec(self):
        return self.c.nrec


def workspace(nbytes: int, device="cuda"):
    """Caller-owned device workspace (torch allocation)."""
    import torch
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)
