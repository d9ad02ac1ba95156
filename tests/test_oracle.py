"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible mistake in the oracle (a dropped term, a wrong
sign, index or time alignment, a transposed operand) fails at least one of them:
  - FD weights: exact second derivatives of polynomials up to degree 9 (8th order);
  - symmetry of the Laplacian with zero values beyond the grid;
  - interpolation weights: partition of unity, exact for linear fields;
  - forward/adjoint dot test and Born (linearised) dot test to 1e-12 (Eq. 2's adjoint);
  - Taylor test of J(m): second-order remainder (sign and scale of Eq. 2);
  - Eq. 3 with an orthonormal nt x nt basis equals Eq. 2 (time alignment of u_tt and v);
  - Eq. 1 brute force: the mean over all 2^nt sign vectors equals the exact gradient;
  - closed-form variance of the Hutchinson estimator and its 1/r decay (Eq. 1);
  - the 2-D homogeneous Green's function (amplitude, arrival time, source scaling);
  - Table 1's memory accounting (golden values printed in the paper).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2201_06914_gb300 import inputs as I
from tests.cases import layered_case, oracle_data, rel

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def small_grid(ndim=2, nt=60, nbl=6):
    return O.Grid(ndim, 23, 17 if ndim == 3 else 1, 19, nbl, nt, 10.0, 9.0, 11.0, 1.3e-3, 2500.0)


def test_fd_weights_are_eighth_order():
    g = small_grid()
    NZ, NX = g.shape
    x = np.arange(NX) * g.dx
    for p in range(10):
        u = np.tile((x / 50.0) ** p, (NZ, 1))
        L = O.laplacian(g, u)
        want = p * (p - 1) * (x / 50.0) ** max(p - 2, 0) / 50.0 ** 2 if p >= 2 else 0 * x
        inner = L[6:-6, 6:-6]
        w = np.tile(want, (NZ, 1))[6:-6, 6:-6]
        assert np.max(np.abs(inner - w)) <= 1e-9 * max(1.0, np.max(np.abs(w))), p


def test_laplacian_symmetric_with_zero_exterior():
    rng = np.random.default_rng(0)
    for ndim in (2, 3):
        g = small_grid(ndim)
        u, w = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
        a, b = np.sum(O.laplacian(g, u) * w), np.sum(u * O.laplacian(g, w))
        assert abs(a - b) <= 1e-13 * abs(a)


def test_interpolation_weights_linear_exact():
    rng = np.random.default_rng(1)
    g = small_grid(3)
    NZ, NY, NX = g.shape
    zz, yy, xx = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
    f = 2.0 + 0.3 * xx - 0.7 * yy + 1.1 * zz
    for _ in range(20):
        p = rng.uniform([0, 0, 0], [(g.nx - 1) * g.dx, (g.ny - 1) * g.dy, (g.nz - 1) * g.dz])
        idx, w = O.weights(g, p)
        assert abs(w.sum() - 1.0) < 1e-14
        gx, gy, gz = g.nbl + p[0] / g.dx, g.nbl + p[1] / g.dy, g.nbl + p[2] / g.dz
        assert abs(np.dot(w, f.ravel()[idx]) - (2.0 + 0.3 * gx - 0.7 * gy + 1.1 * gz)) < 1e-12
    with pytest.raises(ValueError):
        O.weights(g, [1e5, 0.0, 0.0])


def test_sponge_profile():
    g = small_grid()
    s = O.sponge(g)
    s0 = 3 * g.damp_v * math.log(1000.0) / (2 * g.nbl * g.dx)
    assert np.all(s[g.nbl:-g.nbl, g.nbl:-g.nbl] == 0.0)
    row = s[g.nbl + 3]
    assert row[0] == pytest.approx(s0)              # d = nbl at the outer edge (x only)
    assert row[1] == pytest.approx(s0 * ((g.nbl - 1) / g.nbl) ** 2)
    assert row[-1] == pytest.approx(s0)


@pytest.mark.parametrize("ndim", [2, 3])
def test_forward_adjoint_dot_test(ndim):
    """<F s, d'> = <s, F^T d'> with F^T d' = -(sampled v) (the adjoint of Sec. 2.2)."""
    case = layered_case(ndim=ndim, nx=21, ny=15, nz=17, nbl=5, nt=70, off_grid=True)
    g = case.oracle_grid()
    rng = np.random.default_rng(2)
    s = rng.standard_normal(g.nt)
    d = O.forward(g, case.m0, case.src[0], s, case.rec[0])["d"]
    dd = rng.standard_normal(d.shape)
    a = O.adjoint(g, case.m0, case.rec[0], dd, points=case.src[0])
    lhs, rhs = np.sum(d * dd), -np.sum(s * a["vpt"][:, 0])
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_born_dot_test():
    """<J dm, dd> = <dm, g(dd)>: the exact gradient of Eq. 2 is the adjoint of the
    linearised modelling operator (u_tt as the m-derivative of the discrete operator)."""
    case = layered_case(ndim=2, nx=25, nz=21, nbl=5, nt=90, off_grid=True, zi=0.3,
                        background="const")
    g = case.oracle_grid()
    rng = np.random.default_rng(3)
    m0 = case.m0.astype(np.float64)
    f = O.forward(g, m0, case.src[0], case.wavelet, case.rec[0], want_udd=True)
    dm = rng.standard_normal(m0.shape) * m0
    vol = -(dm[None] * f["udd"]).reshape(g.nt, -1)
    dlin = O.forward(g, m0, case.src[0], 0 * case.wavelet, case.rec[0], vol_src=vol)["d"]
    dd = rng.standard_normal(dlin.shape)
    gT = O.adjoint(g, m0, case.rec[0], dd, udd=f["udd"])["g"]
    lhs, rhs = np.sum(dlin * dd), np.sum(dm * gT)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_taylor_second_order():
    case = layered_case(ndim=2, nx=31, nz=25, nbl=6, nt=150, zi=0.3, background="const")
    g = case.oracle_grid()
    m0 = case.m0.astype(np.float64)
    d_obs = oracle_data(case, "true")[0]
    J, grad, _ = O.exact_gradient(g, m0, case.src[0], case.wavelet, case.rec[0], d_obs)
    dm = np.random.default_rng(4).standard_normal(m0.shape) * m0 * 0.01
    errs = []
    for h in (0.1, 0.05, 0.025):
        Jh = O.misfit(O.forward(g, m0 + h * dm, case.src[0], case.wavelet, case.rec[0])["d"], d_obs)
        errs.append(abs(Jh - J - h * np.sum(grad * dm)))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(order - 2.0) < 0.1), order


def test_orthonormal_full_basis_recovers_exact_gradient():
    case = layered_case(ndim=2, nx=21, nz=17, nbl=5, nt=64, zi=0.3, background="const")
    g = case.oracle_grid()
    d_obs = oracle_data(case, "true")[0]
    Q = np.linalg.qr(np.random.default_rng(5).standard_normal((g.nt, g.nt)))[0]
    out = O.probed_gradient(g, case.m0, case.src[0], case.wavelet, case.rec[0], d_obs, Q, 1.0)
    _, gx, _ = O.exact_gradient(g, case.m0, case.src[0], case.wavelet, case.rec[0], d_obs)
    assert rel(out["g_hat"], gx) < 1e-11


def test_rademacher_brute_force_mean_is_exact():
    """Eq. 1: averaging z^T A z over all 2^nt sign vectors gives tr(A) exactly."""
    case = layered_case(ndim=2, nx=9, nz=9, nbl=4, nt=12, zi=0.3, background="const", f0=60.0)
    g = case.oracle_grid()
    d_obs = oracle_data(case, "true")[0]
    bits = (np.arange(2 ** g.nt)[:, None] >> np.arange(g.nt)[None, :]) & 1
    Q = (1.0 - 2.0 * bits).T.astype(np.float64)  # nt x 2^nt, every sign vector once
    out = O.probed_gradient(g, case.m0, case.src[0], case.wavelet, case.rec[0], d_obs, Q,
                            1.0 / Q.shape[1])
    _, gx, _ = O.exact_gradient(g, case.m0, case.src[0], case.wavelet, case.rec[0], d_obs)
    assert rel(out["g_hat"], gx) < 1e-12


@pytest.fixture(scope="module")
def histories():
    case = layered_case(ndim=2, nx=21, nz=17, nbl=5, nt=80, zi=0.3, background="const")
    g = case.oracle_grid()
    d_obs = oracle_data(case, "true")[0]
    f = O.forward(g, case.m0, case.src[0], case.wavelet, case.rec[0], want_udd=True)
    a = O.adjoint(g, case.m0, case.rec[0], f["d"] - d_obs, udd=f["udd"], want_v=True)
    return case, g, f, a


def _seed_estimates(case, g, f, a, r, seeds):
    """g_hat for `seeds` independent Rademacher probe sets of width r (one oracle call with
    all probes stacked: columns are independent, so each group is one estimate)."""
    Z = np.concatenate([I.rademacher(100 + s, g.nt, r) for s in range(seeds)], axis=1)
    Pu = np.tensordot(Z.T, f["udd"], axes=(1, 0)).reshape(seeds, r, -1)
    Pv = np.tensordot(Z.T, a["v"], axes=(1, 0)).reshape(seeds, r, -1)
    return np.einsum("sip,sip->sp", Pu, Pv) / r


def test_oracle_projection_matches_history_contraction(histories):
    """The on-the-fly projections equal Q^T applied to the stored histories (Eq. 3)."""
    case, g, f, a = histories
    Z = I.rademacher(7, g.nt, 6).astype(np.float64)
    fo = O.forward(g, case.m0, case.src[0], case.wavelet, case.rec[0], Q=Z)
    ao = O.adjoint(g, case.m0, case.rec[0], f["d"] - oracle_data(case, "true")[0], Q=Z)
    assert rel(fo["Pu"], np.tensordot(Z.T, f["udd"], axes=(1, 0))) < 1e-13
    assert rel(ao["Pv"], np.tensordot(Z.T, a["v"], axes=(1, 0))) < 1e-13


def test_estimator_variance_closed_form(histories):
    """Var[g_hat(x)] = (1/r)(|a|^2|b|^2 + (a.b)^2 - 2 sum_t a_t^2 b_t^2) for Rademacher
    probes, a = u_tt[., x], b = v[., x]."""
    case, g, f, a = histories
    A = f["udd"].reshape(g.nt, -1)
    B = a["v"].reshape(g.nt, -1)
    r, seeds = 4, 3000
    est = _seed_estimates(case, g, f, a, r, seeds)
    var_emp = est.var(axis=0)
    var_th = (np.sum(A ** 2, 0) * np.sum(B ** 2, 0) + np.sum(A * B, 0) ** 2
              - 2 * np.sum(A ** 2 * B ** 2, 0)) / r
    assert abs(var_emp.sum() / var_th.sum() - 1.0) < 0.08
    mean_err = rel(est.mean(axis=0), a["g"].ravel())
    assert mean_err < 4 * math.sqrt(var_th.sum() / seeds) / np.linalg.norm(a["g"])


def test_estimator_error_decays_like_inverse_sqrt_r(histories):
    case, g, f, a = histories
    gx = a["g"].ravel()
    rs = [2, 4, 8, 16, 32]
    errs = []
    for r in rs:
        est = _seed_estimates(case, g, f, a, r, 200)
        errs.append(np.sqrt(np.mean(np.sum((est - gx) ** 2, axis=1))) / np.linalg.norm(gx))
    slope = np.polyfit(np.log(rs), np.log(errs), 1)[0]
    assert abs(slope + 0.5) < 0.08, slope


def test_greens_function_2d_homogeneous():
    """m u_tt - Lap u = w(t) delta(x - xs) * (dx dz) in 2-D has the solution
    u(R, t) = (dx dz / 2 pi) * int_0^{acosh(v t / R)} w(t - (R/v) cosh xi) dxi."""
    v, h, f0, nt = 1500.0, 5.0, 15.0, 320
    dt = 0.4 * h / v
    n = 121
    g = O.Grid(2, n, 1, n, 20, nt, h, h, h, dt, v)
    m = np.full(g.shape, 1.0 / v ** 2)
    xs = np.array([[300.0, 0.0, 300.0]])
    R = 200.0
    rec = np.array([[300.0 + R, 0.0, 300.0]])
    w = I.ricker(nt, dt, f0)
    d = O.forward(g, m, xs, w, rec)["d"][:, 0]

    def ricker_t(t):
        a = (math.pi * f0 * (t - 1.5 / f0)) ** 2
        return (1 - 2 * a) * np.exp(-a)

    t = (np.arange(nt) + 1) * dt   # row n records u^{n+1}
    ana = np.zeros(nt)
    for k, tk in enumerate(t):
        if v * tk > R:
            xi = np.linspace(0.0, math.acosh(v * tk / R), 4001)
            ana[k] = h * h / (2 * math.pi) * np.trapezoid(ricker_t(tk - (R / v) * np.cosh(xi)), xi)
    win = slice(0, int((R / v + 3.0 / f0) / dt))
    assert rel(d[win], ana[win]) < 2e-2


def test_greens_function_3d_homogeneous():
    """m u_tt - Lap u = w(t) delta(x - xs) * (dx dy dz) in 3-D has the solution
    u(R, t) = (dx dy dz / (4 pi R)) w(t - R / v): no tail, amplitude 1/R.  Checked along x, y
    and z and at half the distance (2 %; a one-sample shift of the record gives 14 %)."""
    v, h, f0, R = 1500.0, 10.0, 8.0, 200.0
    dt = 0.4 * h / v
    nt = int((R / v + 3.5 / f0) / dt) + 5
    n = 81
    g = O.Grid(3, n, n, n, 16, nt, h, h, h, dt, v)
    m = np.full(g.shape, 1.0 / v ** 2)
    c = 0.5 * (n - 1) * h
    xs = np.array([[c, c, c]])
    rec = np.array([[c + R, c, c], [c, c + R, c], [c, c, c + R], [c + R / 2, c, c]])
    d = O.forward(g, m, xs, I.ricker(nt, dt, f0), rec)["d"]

    def ricker_t(t):
        a = (math.pi * f0 * (t - 1.5 / f0)) ** 2
        return (1 - 2 * a) * np.exp(-a)

    t = (np.arange(nt) + 1) * dt   # row n records u^{n+1}
    for j, Rj in enumerate((R, R, R, R / 2)):
        ana = h ** 3 / (4 * math.pi * Rj) * ricker_t(t - Rj / v)
        win = slice(0, int((Rj / v + 2.5 / f0) / dt))
        assert rel(d[win, j], ana[win]) < 2e-2, j


def test_table1_memory_accounting():
    gold = json.load(open(os.path.join(GOLD, "table1_memory.json")))
    for name, row in gold["rows"].items():
        # gain = history bytes / probe bytes = nt / r (same grid, same precision)
        assert row["standard_full"] / row["probed_r64"] == pytest.approx(row["gain_hi"], abs=1.0)
        assert row["standard_4ms"] / row["probed_r32"] == pytest.approx(row["gain_lo"], abs=1.0)
        # probe memory is linear in r
        assert row["probed_r64"] / row["probed_r32"] == pytest.approx(2.0)
        # the accounting reproduces the table for the implied grid and step count
        N = row["probed_r64"] * 1e9 / O.probe_bytes(1, 64)
        nt = row["standard_full"] * 1e9 / O.history_bytes(N, 1)
        assert O.history_bytes(N, nt) / O.probe_bytes(N, 64) == pytest.approx(nt / 64)
        assert nt / 64 == pytest.approx(row["gain_hi"], rel=5e-3)
    assert all(r["probed_r64"] < gold["text_claim"]["max_footprint_gb"] + 0.2
               for r in gold["rows"].values())


def test_splitmix64_published_outputs():
    gold = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    assert [int(x) for x in I.splitmix64(0, 3)] == [int(s, 16) for s in gold["seed_0"]]
    assert [int(x) for x in I.splitmix64(1234567, 3)] == gold["seed_1234567"]
    Z = I.rademacher(0, 400, 50)
    assert set(np.unique(Z)) == {-1.0, 1.0}
    C = Z.T @ Z / Z.shape[0]                 # E[z z^T] = I (Eq. 1's condition)
    assert np.max(np.abs(np.diag(C) - 1)) == 0 and np.max(np.abs(C - np.eye(50))) < 0.25
