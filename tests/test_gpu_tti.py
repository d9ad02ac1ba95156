"""GPU parity of the pseudo-acoustic TTI path (two wavefields per shot) against the FP64
oracle: recorded data and both fields' probed projections (relative L2 1e-5), the
randomized gradient summed over both fields (1e-4), the exact gradient (1e-4) and the
bit-identity of the checkpointed recomputation."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.cases import close, rel, tti_case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _run(ndim, nx, ny, nz, nbl, nt, r, Tb, nshots=2):
    from paper_2201_06914_gb300 import wp
    from paper_2201_06914_gb300.inputs import rademacher_shots
    case, th = tti_case(ndim=ndim, nx=nx, ny=ny, nz=nz, nbl=nbl, nt=nt, nshots=nshots)
    grid = case.oracle_grid()
    Q = rademacher_shots(0, nshots, nt, r)
    ref = dict(d=[], Pu=[], Pv=[], res=[], g=0.0, gx=0.0, d_obs=[])
    for s in range(nshots):
        d_obs = O.tti_forward(grid, case.m_true, th, case.src[s], case.wavelet, case.rec[s])["d"]
        f = O.tti_forward(grid, case.m0, th, case.src[s], case.wavelet, case.rec[s], Q=Q[s],
                          want_udd=True)
        res = f["d"] - d_obs
        a = O.tti_adjoint(grid, case.m0, th, case.rec[s], res, Q=Q[s], udd=f["udd"])
        ref["d"].append(f["d"]); ref["res"].append(res); ref["d_obs"].append(d_obs)
        ref["Pu"].append(f["Pu"].reshape(2, r, -1)); ref["Pv"].append(a["Pv"].reshape(2, r, -1))
        ref["g"] = ref["g"] + (O.probed_image(f["Pu"][0], a["Pv"][0], 1.0 / r) +
                               O.probed_image(f["Pu"][1], a["Pv"][1], 1.0 / r))
        ref["gx"] = ref["gx"] + a["g"]
    for k in ("d", "Pu", "Pv", "res", "d_obs"):
        ref[k] = np.stack(ref[k])
    M = wp.Model(ndim, nx, ny, nz, nbl, case.h, case.h, case.h, case.dt, nt, _t(case.m0.ravel()),
                 case.damp_v, eps=_t(th.eps.ravel()), delta=_t(th.delta.ravel()),
                 theta=_t(th.theta.ravel()), phi=_t(th.phi.ravel()))
    G = wp.Geometry(case.src, case.rec)
    N = case.N
    ws = wp.workspace(wp.wp_workspace_bytes(M.handle, G.c, r, Tb, wp.WP_MODE_PROBED))
    Pu = torch.full((nshots, 2, r, N), float("nan"), device="cuda")
    d = torch.full((nshots, nt, G.nrec), float("nan"), device="cuda")
    wp.wp_probe_forward(M.handle, G.c, _t(case.wavelet), _t(Q), r, Tb, Pu, d, ws)
    g = torch.full((N,), float("nan"), device="cuda")
    Pv = torch.full((nshots, 2, r, N), float("nan"), device="cuda")
    wp.wp_adjoint_image(M.handle, G.c, _t(ref["res"]), _t(Q), r, Tb, 1.0 / r, _t(ref["Pu"]), g, Pv, ws)
    wp.wp_stream_status(ws)
    out = dict(d=d.cpu().numpy(), Pu=Pu.cpu().numpy(), Pv=Pv.cpu().numpy(), g=g.cpu().numpy())
    gx = torch.full((N,), float("nan"), device="cuda")
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    wse = wp.workspace(wp.wp_workspace_bytes(M.handle, G.c, 0, 1, wp.WP_MODE_EXACT_FULL))
    wp.wp_exact_gradient(M.handle, G.c, _t(case.wavelet), _t(ref["d_obs"]), gx, J, None,
                         wp.WP_MODE_EXACT_FULL, 1, wse)
    wp.wp_stream_status(wse)
    out["gx"] = gx.cpu().numpy()
    gc = torch.full((N,), float("nan"), device="cuda")
    wsc = wp.workspace(wp.wp_workspace_bytes(M.handle, G.c, 0, 23, wp.WP_MODE_EXACT_CHECKPOINT))
    wp.wp_exact_gradient(M.handle, G.c, _t(case.wavelet), _t(ref["d_obs"]), gc, J, None,
                         wp.WP_MODE_EXACT_CHECKPOINT, 23, wsc)
    wp.wp_stream_status(wsc)
    out["gc"] = gc.cpu().numpy()
    return ref, out


@pytest.mark.parametrize("ndim,nx,ny,nz,nbl,nt,r,Tb", [(2, 41, 1, 33, 6, 150, 8, 32),
                                                       (3, 23, 19, 21, 5, 90, 6, 48)])
def test_tti_parity(ndim, nx, ny, nz, nbl, nt, r, Tb):
    ref, out = _run(ndim, nx, ny, nz, nbl, nt, r, Tb)
    ok, err = close(out["d"], ref["d"], 1e-5)
    assert ok, err
    ok, err = close(out["Pu"], ref["Pu"], 1e-5)
    assert ok, err
    ok, err = close(out["Pv"], ref["Pv"], 1e-5)
    assert ok, err
    ok, err = close(out["g"], ref["g"].ravel(), 1e-4)
    assert ok, err
    ok, err = close(out["gx"], ref["gx"].ravel(), 1e-4)
    assert ok, err
    np.testing.assert_array_equal(out["gc"], out["gx"])


def test_model_rejects_delta_above_eps():
    """Where delta > eps the 2 x 2 symbol of the pseudo-acoustic system has determinant
    2 (eps - delta) |k_perp|^2 |k_par|^2 < 0: a growing mode.  wp_model refuses such a
    model (WP_ERR_UNSTABLE) and accepts the elliptic limit delta = eps."""
    from paper_2201_06914_gb300 import wp
    nx, nz, nbl = 20, 16, 4
    N = (nx + 2 * nbl) * (nz + 2 * nbl)
    m = _t(np.full(N, 1 / 2000.0 ** 2))
    eps = np.full(N, 0.1)
    zero = _t(np.zeros(N))
    wp.Model(2, nx, 1, nz, nbl, 10.0, 10.0, 10.0, 1e-3, 10, m, 2000.0,
             eps=_t(eps), delta=_t(eps), theta=zero, phi=zero).close()
    bad = eps.copy()
    bad[N // 2] = 0.2
    with pytest.raises(wp.WpError) as err:
        wp.Model(2, nx, 1, nz, nbl, 10.0, 10.0, 10.0, 1e-3, 10, m, 2000.0,
                 eps=_t(eps), delta=_t(bad), theta=zero, phi=zero)
    assert err.value.status == wp.WP_ERR_UNSTABLE
