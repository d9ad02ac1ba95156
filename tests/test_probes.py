"""Range-finder probes (Sec. 2.1, [Q, ~] = qr(A Z)).

Oracle pins: Q is orthonormal; for an A of rank k <= r the sketch captures its range
exactly; with r = nt, Q Q^T = I (so the estimate is exact).  The product's host-side
construction (FFT Toeplitz products, its own QR call) is compared with the oracle's
dense-matrix definition for both readings of A, and on a small propagation case the
wavelet range finder beats Rademacher probes at the same r.
"""
import numpy as np
import scipy.linalg as sl

from oracle import oracle as O
from paper_2201_06914_gb300 import inputs as I
from paper_2201_06914_gb300 import probes as P
from tests.cases import layered_case, rel


def test_oracle_range_finder_orthonormal_and_exact_on_low_rank():
    rng = np.random.default_rng(0)
    nt, r, k = 50, 12, 7
    A = rng.standard_normal((nt, k)) @ rng.standard_normal((k, nt))
    Z = I.rademacher(3, nt, r)
    Q = O.range_finder(A, Z)
    assert np.max(np.abs(Q.T @ Q - np.eye(r))) < 1e-12
    assert np.linalg.norm(A - Q @ (Q.T @ A)) < 1e-12 * np.linalg.norm(A)
    Qf = O.range_finder(np.eye(nt), I.rademacher(4, nt, nt))
    assert np.max(np.abs(Qf @ Qf.T - np.eye(nt))) < 1e-12


def _dense_conv(w, nt):
    return sl.toeplitz(np.asarray(w, np.float64)[:nt], np.zeros(nt))


def test_wavelet_range_finder_matches_oracle():
    nt, r = 180, 16
    w = I.ricker(nt, 2e-3, 12.0)
    W = _dense_conv(w, nt)
    A = np.linalg.matrix_power(W @ W.T, 2)
    ref = O.range_finder(A, I.rademacher(9, nt, r))
    got = P.range_finder(P.wavelet_operator(w, 2), nt, r, 9)
    assert got.dtype == np.float32
    assert np.max(np.abs(got - ref)) < 1e-5


def test_data_range_finder_matches_oracle():
    rng = np.random.default_rng(2)
    nt, nrec, r = 120, 30, 10
    D = rng.standard_normal((nt, nrec))
    ref = O.range_finder(D @ D.T, I.rademacher(5, nt, r))
    got = P.range_finder(P.data_operator(D), nt, r, 5)
    assert np.max(np.abs(got - ref)) < 1e-5


def test_wavelet_probes_beat_rademacher_on_a_small_case():
    case = layered_case(ndim=2, nx=41, nz=35, nbl=8, nt=200, zi=0.3, background="const")
    g = case.oracle_grid()
    d_obs = O.forward(g, case.m_true, case.src[0], case.wavelet, case.rec[0])["d"]
    _, g_exact, _ = O.exact_gradient(g, case.m0, case.src[0], case.wavelet, case.rec[0], d_obs)
    r = 24
    Qr = I.rademacher(1, g.nt, r)
    e_rad = rel(O.probed_gradient(g, case.m0, case.src[0], case.wavelet, case.rec[0], d_obs,
                                  Qr, 1.0 / r)["g_hat"], g_exact)
    Qw = P.range_finder(P.wavelet_operator(case.wavelet, 2), g.nt, r, 1)
    e_rf = rel(O.probed_gradient(g, case.m0, case.src[0], case.wavelet, case.rec[0], d_obs,
                                 Qw.astype(np.float64), 1.0)["g_hat"], g_exact)
    assert e_rf < e_rad, (e_rf, e_rad)
