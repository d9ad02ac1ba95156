"""Probing matrices for the randomized trace estimate (Sec. 2.1, Eq. 1 and 3).

`rademacher` is the plain Hutchinson choice (entries +-1, estimator scale 1/r).  The
paper also approximates the range of the traced matrix with a partial QR factorisation,
[Q, ~] = qr(A Z) with Z Rademacher; the estimate with an orthonormal Q uses scale 1.  The
paper does not say which A; two readings are offered, both operators on the time axis:

  - "wavelet": A = (W W^T)^p with W the causal convolution by the source wavelet.  Every
    trace of the forward wavefield is a sum of delayed, scaled copies of the wavelet, so
    its temporal covariance is shaped by the wavelet's autocorrelation; the power p
    sharpens the captured band (a power-iteration step of the randomized range finder).
  - "data": A = D D^T with D the shot's nt x nrec observed data.

Z comes from the same SplitMix64 streams as the Rademacher probes (seed = base + shot).
Everything here runs on the host once per shot; the CUDA kernels take Q as an input.
"""
from __future__ import annotations

import numpy as np

from . import inputs as I


def rademacher(base_seed: int, nshots: int, nt: int, r: int) -> tuple[np.ndarray, float]:
    """(Q (nshots, nt, r) float32 +-1, estimator scale 1/r)."""
    return I.rademacher_shots(base_seed, nshots, nt, r), 1.0 / r


def _conv(x: np.ndarray, w: np.ndarray, transpose: bool) -> np.ndarray:
    """Causal convolution of each column of x (nt, k) with w, or its transpose
    (correlation), truncated to nt samples."""
    nt = x.shape[0]
    n = 1 << int(np.ceil(np.log2(2 * nt)))
    W = np.fft.rfft(w, n)
    if transpose:
        W = np.conj(W)
    y = np.fft.irfft(np.fft.rfft(x, n, axis=0) * W[:, None], n, axis=0)
    return y[:nt] if not transpose else y[:nt]


def _orth(Y: np.ndarray) -> np.ndarray:
    """Q of the thin QR of Y with the signs fixed so that diag(R) >= 0."""
    Q, R = np.linalg.qr(Y)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def wavelet_operator(wavelet: np.ndarray, power: int = 2):
    """x -> (W W^T)^power x for x of shape (nt, k)."""
    w = np.asarray(wavelet, np.float64)

    def apply(x):
        y = np.asarray(x, np.float64)
        for _ in range(power):
            y = _conv(_conv(y, w, True), w, False)
        return y
    return apply


def data_operator(d_obs: np.ndarray):
    """x -> D D^T x for one shot's data D (nt, nrec)."""
    D = np.asarray(d_obs, np.float64)
    return lambda x: D @ (D.T @ np.asarray(x, np.float64))


def range_finder(op, nt: int, r: int, seed: int) -> np.ndarray:
    """[Q, ~] = qr(A Z) (Sec. 2.1) for one shot: Q (nt, r) orthonormal, float32."""
    Z = I.rademacher(seed, nt, r).astype(np.float64)
    return _orth(op(Z)).astype(np.float32)


def range_finder_shots(base_seed: int, nt: int, r: int, ops) -> tuple[np.ndarray, float]:
    """Per-shot range-finder probes: ops[s] is the operator of shot s.
    Returns (Q (nshots, nt, r) float32, estimator scale 1)."""
    return np.stack([range_finder(op, nt, r, base_seed + s) for s, op in enumerate(ops)]), 1.0
