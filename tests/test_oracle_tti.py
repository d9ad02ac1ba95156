"""Pins of the FP64 oracle's pseudo-acoustic TTI physics (the paper's second physics,
Sec. 3 "2007 BP TTI"; the equations are a reading, described in wp_oracle.c).

  - Hz = -Dr^T Dr is symmetric and negative semi-definite;
  - with zero tilt Hz is the composed 8th-order d/dz d/dz: exact (=2) on z^2;
  - eps = delta = 0 reduces the two-field system to the isotropic equation (p = q);
  - forward/adjoint and Born dot tests to 1e-12, Taylor test (sign and scale of Eq. 2);
  - Eq. 3 summed over both fields with an orthonormal nt x nt basis equals Eq. 2;
  - in a homogeneous medium waves travel at v (1 + 2 eps)^(1/2) across the symmetry axis
    and at v along it (elliptic eps = delta, and eps > delta): measured as the time shift
    between traces 500 m from the source along x and along z.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests.cases import layered_case, rel, tti_case


def test_hz_symmetric_negative_semidefinite():
    rng = np.random.default_rng(0)
    for ndim in (2, 3):
        g = O.Grid(ndim, 15, 13, 11, 4, 10, 10.0, 11.0, 9.0, 1e-3, 2000.0)
        theta = rng.uniform(0, 0.7, g.shape)
        phi = rng.uniform(0, 1.5, g.shape)
        u, w = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
        a = np.sum(O.apply_hz(g, theta, phi, u) * w)
        b = np.sum(u * O.apply_hz(g, theta, phi, w))
        assert abs(a - b) <= 1e-13 * abs(a)
        assert np.sum(O.apply_hz(g, theta, phi, u) * u) < 0


def test_hz_zero_tilt_is_second_z_derivative():
    g = O.Grid(2, 21, 1, 31, 4, 10, 10.0, 10.0, 10.0, 1e-3, 2000.0)
    NZ, NX = g.shape
    z = np.arange(NZ)[:, None] * g.dz * np.ones((1, NX))
    out = O.apply_hz(g, np.zeros(g.shape), None, (z / 100.0) ** 2)
    inner = out[8:-8, :]
    assert np.max(np.abs(inner - 2.0 / 100.0 ** 2)) < 1e-12


def test_isotropic_limit_matches_acoustic():
    case, th = tti_case(ndim=2, scale=0.0)
    g = case.oracle_grid()
    d_tti = O.tti_forward(g, case.m0, th, case.src[0], case.wavelet, case.rec[0])["d"]
    d_iso = O.forward(g, case.m0, case.src[0], case.wavelet, case.rec[0])["d"]
    assert rel(d_tti, d_iso) < 1e-12
    th_tilt = O.Thomsen(th.eps, th.delta, th.theta + 0.5, th.phi)   # tilt alone is isotropic too
    d_tilt = O.tti_forward(g, case.m0, th_tilt, case.src[0], case.wavelet, case.rec[0])["d"]
    assert rel(d_tilt, d_iso) < 1e-12
    case2, th2 = tti_case(ndim=2, scale=1.0)
    d_ani = O.tti_forward(g, case.m0, th2, case.src[0], case.wavelet, case.rec[0])["d"]
    assert rel(d_ani, d_iso) > 1e-3


@pytest.mark.parametrize("ndim", [2, 3])
def test_tti_dot_test(ndim):
    case, th = tti_case(ndim=ndim, nx=17, ny=13, nz=15, nbl=5, nt=60)
    g = case.oracle_grid()
    rng = np.random.default_rng(1)
    s = rng.standard_normal(g.nt)
    d = O.tti_forward(g, case.m0, th, case.src[0], s, case.rec[0])["d"]
    dd = rng.standard_normal(d.shape)
    a = O.tti_adjoint(g, case.m0, th, case.rec[0], dd, points=case.src[0])
    lhs = np.sum(d * dd)
    rhs = -np.sum(s * (a["vpt"][:, 0, 0] + a["vpt"][:, 0, 1]))  # source fires in both fields
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_tti_born_dot_and_taylor():
    case, th = tti_case(ndim=2, nx=23, nz=21, nbl=5, nt=100)
    g = case.oracle_grid()
    m0 = case.m0.astype(np.float64)
    rng = np.random.default_rng(2)
    f = O.tti_forward(g, m0, th, case.src[0], case.wavelet, case.rec[0], want_udd=True)
    dm = rng.standard_normal(m0.shape) * m0
    vol = -(dm[None, None] * f["udd"]).reshape(g.nt * 2, -1)
    dlin = O.tti_forward(g, m0, th, case.src[0], 0 * case.wavelet, case.rec[0], vol_src=vol)["d"]
    dd = rng.standard_normal(dlin.shape)
    gT = O.tti_adjoint(g, m0, th, case.rec[0], dd, udd=f["udd"])["g"]
    lhs, rhs = np.sum(dlin * dd), np.sum(dm * gT)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # Taylor test of the misfit against data from the true model
    d_obs = O.tti_forward(g, case.m_true, th, case.src[0], case.wavelet, case.rec[0])["d"]
    J, grad, _ = O.tti_exact_gradient(g, m0, th, case.src[0], case.wavelet, case.rec[0], d_obs)
    dmm = dm * 0.01
    errs = []
    for h in (0.1, 0.05, 0.025):
        Jh = O.misfit(O.tti_forward(g, m0 + h * dmm, th, case.src[0], case.wavelet,
                                    case.rec[0])["d"], d_obs)
        errs.append(abs(Jh - J - h * np.sum(grad * dmm)))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(order - 2.0) < 0.15), order


def test_tti_orthonormal_basis_recovers_exact():
    case, th = tti_case(ndim=2, nx=19, nz=17, nbl=5, nt=48)
    g = case.oracle_grid()
    d_obs = O.tti_forward(g, case.m_true, th, case.src[0], case.wavelet, case.rec[0])["d"]
    Q = np.linalg.qr(np.random.default_rng(3).standard_normal((g.nt, g.nt)))[0]
    out = O.tti_probed_gradient(g, case.m0, th, case.src[0], case.wavelet, case.rec[0], d_obs, Q, 1.0)
    _, gx, _ = O.tti_exact_gradient(g, case.m0, th, case.src[0], case.wavelet, case.rec[0], d_obs)
    assert rel(out["g_hat"], gx) < 1e-11


def _axis_lag(eps, delta, theta):
    """Arrival delay of the trace 500 m below the source relative to the trace 500 m beside
    it (cross-correlation peak), homogeneous 2 km/s medium with constant Thomsen fields."""
    from paper_2201_06914_gb300 import inputs as I
    n, nbl, h, v, nt = 141, 20, 10.0, 2000.0, 300
    dt = 0.4 * h / (v * np.sqrt(1 + 2 * eps))
    g = O.Grid(2, n, 1, n, nbl, nt, h, h, h, dt, v)
    full = lambda a: np.full(g.shape, float(a))
    th = O.Thomsen(full(eps), full(delta), full(theta), full(0.0))
    c = 0.5 * (n - 1) * h
    rec = np.array([[c + 500.0, 0.0, c], [c, 0.0, c + 500.0]])
    d = O.tti_forward(g, full(1.0 / v ** 2), th, np.array([[c, 0.0, c]]), I.ricker(nt, dt, 15.0), rec)["d"]
    cc = np.correlate(d[:, 1], d[:, 0], mode="full")
    k = int(np.argmax(cc))
    frac = 0.5 * (cc[k - 1] - cc[k + 1]) / (cc[k - 1] - 2 * cc[k] + cc[k + 1])
    return (k + frac - (nt - 1)) * dt


def test_thomsen_eps_sets_velocity_across_the_axis():
    v, r, eps = 2000.0, 500.0, 0.2
    want = r / v - r / (v * np.sqrt(1 + 2 * eps))       # 38.7 ms
    vti = _axis_lag(eps, 0.1, 0.0)                       # symmetry axis along z
    assert abs(vti - want) < 0.02 * want, (vti, want)
    hti = _axis_lag(eps, 0.1, np.pi / 2)                 # axis along x: the fast direction is z
    assert abs(hti + want) < 0.02 * want, (hti, want)
    ell = _axis_lag(eps, eps, 0.0)                       # elliptic anisotropy
    assert abs(ell - want) < 0.02 * want, (ell, want)
    assert abs(_axis_lag(0.0, 0.0, 0.0)) < 1e-4
