"""Pins of the oracle's subsurface-offset image volume (Eq. 4).

  - offset 0 is the randomized image of Eq. 3 computed by the C oracle;
  - a tiny case against a brute-force triple loop;
  - with an orthonormal nt x nt basis the probed volume equals the exact one built from
    the stored u_tt and v histories (the trace identity behind Eq. 4);
  - the mean over all 2^T Rademacher sign vectors (r = 1, scale 1) equals the exact volume;
  - exchanging P_u and P_v mirrors the offset axis.
"""
import itertools

import numpy as np

from oracle import oracle as O
from tests.cases import layered_case, rel


def test_offset_zero_is_probed_image():
    rng = np.random.default_rng(0)
    Pu, Pv = rng.standard_normal((2, 5, 7, 13))
    vol = O.offset_image(Pu, Pv, 3, 0.2)
    img = O.probed_image(Pu, Pv, 0.2)
    assert np.max(np.abs(vol[3] - img)) < 1e-13


def test_brute_force_tiny():
    rng = np.random.default_rng(1)
    r, nz, nx, nh = 3, 2, 9, 4
    Pu, Pv = rng.standard_normal((2, r, nz, nx))
    vol = O.offset_image(Pu, Pv, nh, 0.5)
    ref = np.zeros_like(vol)
    for h in range(-nh, nh + 1):
        for z in range(nz):
            for x in range(nx):
                if 0 <= x + h < nx and 0 <= x - h < nx:
                    ref[h + nh, z, x] = 0.5 * sum(Pu[i, z, x + h] * Pv[i, z, x - h] for i in range(r))
    assert np.max(np.abs(vol - ref)) < 1e-13
    # entries whose shifted points leave the row are zero
    assert np.all(vol[0, :, :nh] == 0) and np.all(vol[-1, :, nx - nh:] == 0)


def test_orthonormal_basis_recovers_exact_offsets():
    case = layered_case(ndim=2, nx=23, nz=19, nbl=5, nt=60)
    g = case.oracle_grid()
    f = O.forward(g, case.m0, case.src[0], case.wavelet, case.rec[0], want_udd=True)
    d_obs = O.forward(g, case.m_true, case.src[0], case.wavelet, case.rec[0])["d"]
    a = O.adjoint(g, case.m0, case.rec[0], f["d"] - d_obs, want_v=True)
    exact = O.offset_image(f["udd"], a["v"], 6, 1.0)
    assert rel(exact[6], O.adjoint(g, case.m0, case.rec[0], f["d"] - d_obs, udd=f["udd"])["g"]) < 1e-12
    Q = np.linalg.qr(np.random.default_rng(2).standard_normal((g.nt, g.nt)))[0]
    Pu = np.tensordot(Q.T, f["udd"], axes=1)
    Pv = np.tensordot(Q.T, a["v"], axes=1)
    assert rel(O.offset_image(Pu, Pv, 6, 1.0), exact) < 1e-11


def test_rademacher_mean_over_all_signs_is_exact():
    rng = np.random.default_rng(3)
    T, nz, nx, nh = 6, 3, 8, 2
    udd, v = rng.standard_normal((2, T, nz, nx))
    exact = O.offset_image(udd, v, nh, 1.0)
    acc = np.zeros_like(exact)
    for signs in itertools.product((-1.0, 1.0), repeat=T):
        z = np.array(signs)
        acc += O.offset_image(np.tensordot(z, udd, axes=1)[None], np.tensordot(z, v, axes=1)[None], nh, 1.0)
    assert np.max(np.abs(acc / 2 ** T - exact)) < 1e-12


def test_swap_mirrors_offsets():
    rng = np.random.default_rng(4)
    Pu, Pv = rng.standard_normal((2, 4, 5, 11))
    a = O.offset_image(Pu, Pv, 3, 1.0)
    b = O.offset_image(Pv, Pu, 3, 1.0)
    assert np.max(np.abs(a - b[::-1])) < 1e-13
