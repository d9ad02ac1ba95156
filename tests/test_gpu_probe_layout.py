"""GPU checks of the row-aligned probe layout (WP_PROBES_ALIGNED, include/wp.h): the
projections P_u, P_v (Eq. 3) the library writes in it are bitwise those of the dense
layout once the padding is dropped, the image is bitwise the same, and the offset volume
(Eq. 4) read from aligned rows (TMA-staged, MN-major operands) matches the oracle's definition on
ragged rows, odd offset counts and partial contraction chunks.  The padding entries of
the aligned inputs are NaN: the volume must not read them."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.cases import layered_case, oracle_data, rel, tti_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wp():
    from paper_2201_06914_gb300 import wp as _wp
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return _wp


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _to_aligned(P, shape, RS, XP):
    """(S, r, *shape) dense -> (S, r, RS) aligned rows, NaN in every padding entry."""
    S, r = P.shape[:2]
    NX = shape[-1]
    rows = int(np.prod(shape[:-1]))
    A = np.full((S, r, RS), np.nan, np.float32)
    A[:, :, :rows * XP].reshape(S, r, rows, XP)[..., :NX] = P.reshape(S, r, rows, NX)
    return A


def _from_aligned(A, shape, XP):
    S, r = A.shape[:2]
    NX = shape[-1]
    rows = int(np.prod(shape[:-1]))
    return A[:, :, :rows * XP].reshape(S, r, rows, XP)[..., :NX].reshape((S, r) + tuple(shape))


def _model(wp, ndim, nx, ny, nz, nbl):
    NX, NY, NZ = nx + 2 * nbl, (ny + 2 * nbl if ndim == 3 else 1), nz + 2 * nbl
    m = _t(np.full(NX * NY * NZ, 1 / 1500.0 ** 2))
    shape = (NZ, NY, NX) if ndim == 3 else (NZ, NX)
    return wp.Model(ndim, nx, ny, nz, nbl, 10.0, 10.0, 10.0, 1e-3, 16, m, 1500.0), shape


def test_layout_query_and_switch(wp):
    M, shape = _model(wp, 2, 61, 1, 9, 8)     # NX = 77: x pitch 80
    N = int(np.prod(shape))
    assert wp.wp_probe_layout(M.handle) == (wp.WP_PROBES_DENSE, N, shape[-1])
    wp.wp_set_probe_layout(M.handle, wp.WP_PROBES_ALIGNED)
    lay, RS, XP = wp.wp_probe_layout(M.handle)
    assert lay == wp.WP_PROBES_ALIGNED and XP == 80 and RS % 128 == 0 and RS >= shape[0] * XP
    with pytest.raises(wp.WpError):
        wp.wp_set_probe_layout(M.handle, 2)


@pytest.mark.parametrize("ndim,nx,ny,nz,r,S,nh", [
    (2, 290, 1, 7, 17, 2, 40),    # rows of 306 (pitch 308): two full tiles and a partial one
    (2, 130, 1, 5, 64, 1, 64),    # largest offset range, 4 probe chunks
    (2, 100, 1, 4, 1, 3, 0),      # offset 0 only, one probe
    (2, 57, 1, 6, 33, 1, 7),      # odd nh: the b window starts 2 points early
    (2, 61, 1, 5, 24, 2, 3),      # K = 48: one partial chunk; odd nh
    (3, 40, 6, 5, 16, 2, 21),     # 3-D: offsets along x within each (z, y) row
])
def test_offset_volume_aligned_parity(wp, ndim, nx, ny, nz, r, S, nh):
    M, shape = _model(wp, ndim, nx, ny, nz, 8)
    wp.wp_set_probe_layout(M.handle, wp.WP_PROBES_ALIGNED)
    _, RS, XP = wp.wp_probe_layout(M.handle)
    N = int(np.prod(shape))
    rng = np.random.default_rng(nx + r + nh + 1)
    Pu = rng.standard_normal((S, r) + shape)
    Pv = rng.standard_normal((S, r) + shape)
    out = torch.full((2 * nh + 1, N), float("nan"), device="cuda")
    wp.wp_offset_image(M.handle, _t(_to_aligned(Pu, shape, RS, XP)), _t(_to_aligned(Pv, shape, RS, XP)),
                       r, S, 0.25, nh, out)
    wp.wp_offset_status()
    got = out.cpu().numpy().reshape((2 * nh + 1,) + shape)
    ref = sum(O.offset_image(Pu[s], Pv[s], nh, 0.25) for s in range(S))
    assert np.all(np.isfinite(got))
    assert rel(got, ref) < 1e-5
    if nh > 0:
        assert np.all(got[0][..., :nh] == 0) and np.all(got[-1][..., -nh:] == 0)


def _probed(wp, M, G, case, Q, r, Tb, S, N, rows_floats, tti=False):
    ws = wp.workspace(wp.wp_workspace_bytes(M.handle, G.c, r, Tb, wp.WP_MODE_PROBED))
    nv = 2 if tti else 1
    Pu = torch.full((S, nv * r, rows_floats), float("nan"), device="cuda")
    Pv = torch.full((S, nv * r, rows_floats), float("nan"), device="cuda")
    d = torch.empty((S, case.nt, G.nrec), device="cuda")
    g = torch.empty(N, device="cuda")
    wp.wp_probe_forward(M.handle, G.c, _t(case.wavelet), _t(Q), r, Tb, Pu, d, ws)
    res = (d - d.flip(0)).contiguous() if S > 1 else d
    wp.wp_adjoint_image(M.handle, G.c, res, _t(Q), r, Tb, 1.0 / r, Pu, g, Pv, ws)
    wp.wp_stream_status(ws)
    return Pu.cpu().numpy(), Pv.cpu().numpy(), g.cpu().numpy(), d.cpu().numpy()


@pytest.mark.parametrize("ndim", [2, 3])
def test_probed_gradient_aligned_equals_dense(wp, ndim):
    from paper_2201_06914_gb300 import inputs as I
    if ndim == 2:
        case = layered_case(ndim=2, nx=71, nz=41, nbl=8, nt=150, nshots=2, zi=0.3, background="const")
    else:
        case = layered_case(ndim=3, nx=23, ny=18, nz=21, nbl=6, nt=90, nshots=2, zi=0.3, background="const")
    r, Tb, nh, S = 24, 32, 5, case.nshots
    Q = I.rademacher_shots(7, S, case.nt, r)
    G = wp.Geometry(case.src, case.rec)
    N = case.N
    outs = {}
    for lay in (wp.WP_PROBES_DENSE, wp.WP_PROBES_ALIGNED):
        M = wp.Model(case.ndim, case.nx, case.ny, case.nz, case.nbl, case.h, case.h, case.h, case.dt,
                     case.nt, _t(case.m0.ravel()), case.damp_v)
        wp.wp_set_probe_layout(M.handle, lay)
        _, RS, XP = wp.wp_probe_layout(M.handle)
        Pu, Pv, g, d = _probed(wp, M, G, case, Q, r, Tb, S, N, RS)
        out = torch.empty((2 * nh + 1, N), device="cuda")
        wp.wp_offset_image(M.handle, _t(Pu), _t(Pv), r, S, 1.0 / r, nh, out)
        wp.wp_offset_status()
        if lay == wp.WP_PROBES_ALIGNED:
            Pu, Pv = _from_aligned(Pu, case.shape, XP), _from_aligned(Pv, case.shape, XP)
        outs[lay] = (Pu.reshape((S, r) + case.shape), Pv.reshape((S, r) + case.shape), g, d,
                     out.cpu().numpy())
    dn, al = outs[wp.WP_PROBES_DENSE], outs[wp.WP_PROBES_ALIGNED]
    for k in range(4):   # P_u, P_v, image, data: the same kernels on the same values
        assert np.array_equal(dn[k], al[k]), k
    ref = sum(O.offset_image(dn[0][s].astype(np.float64), dn[1][s].astype(np.float64), nh, 1.0 / r)
              for s in range(S))
    assert rel(al[4].reshape(ref.shape), ref) < 1e-5
    assert rel(al[4][nh], dn[2]) < 1e-5


def test_tti_projections_aligned_equal_dense(wp):
    from paper_2201_06914_gb300 import inputs as I
    case, th = tti_case(ndim=2, nx=31, nz=27, nbl=6, nt=100, nshots=2)
    r, Tb, S = 16, 32, case.nshots
    Q = I.rademacher_shots(3, S, case.nt, r)
    G = wp.Geometry(case.src, case.rec)
    got = {}
    for lay in (wp.WP_PROBES_DENSE, wp.WP_PROBES_ALIGNED):
        M = wp.Model(2, case.nx, 1, case.nz, case.nbl, case.h, case.h, case.h, case.dt, case.nt,
                     _t(case.m0.ravel()), case.damp_v, eps=_t(th.eps.ravel()), delta=_t(th.delta.ravel()),
                     theta=_t(th.theta.ravel()), phi=_t(th.phi.ravel()))
        wp.wp_set_probe_layout(M.handle, lay)
        _, RS, XP = wp.wp_probe_layout(M.handle)
        Pu, Pv, g, _ = _probed(wp, M, G, case, Q, r, Tb, S, case.N, RS, tti=True)
        if lay == wp.WP_PROBES_ALIGNED:
            Pu, Pv = _from_aligned(Pu, case.shape, XP), _from_aligned(Pv, case.shape, XP)
        got[lay] = (Pu.reshape(S, 2 * r, -1), Pv.reshape(S, 2 * r, -1), g)
    for k in range(3):
        assert np.array_equal(got[wp.WP_PROBES_DENSE][k], got[wp.WP_PROBES_ALIGNED][k]), k


def test_bench_shaped_aligned_equals_dense(wp):
    """The bench's own configuration — 1601 x 401 salt model, 64 shots, r = 64, Tb = 256
    (four 64-step chunks per block, a partial last block) — in both probe layouts: the
    projections, the image and the data are bitwise the same, and the offset volumes of the
    two layouts' kernels (MN-major in-place and K-major register-load) agree within the
    split's accuracy."""
    from paper_2201_06914_gb300 import inputs as I
    sv = I.config_salt_2d(nx=1601, nz=401, nt=300, r=64, nshots=64)
    S, r, Tb, nt, N = sv.nshots, 64, 256, sv.nt, sv.npoints
    G = wp.Geometry(sv.src, sv.rec)
    nrec = G.nrec
    wav = _t(sv.wavelet())
    Q = _t(I.rademacher_shots(0, S, nt, r))
    m0 = _t(sv.m_padded("background").ravel())
    mt = _t(sv.m_padded("true").ravel())
    Mt = wp.Model.from_survey(sv, mt)
    ws0 = wp.workspace(wp.wp_workspace_bytes(Mt.handle, G.c, 0, Tb, wp.WP_MODE_PROBED))
    dobs = torch.empty((S, nt, nrec), device="cuda")
    wp.wp_probe_forward(Mt.handle, G.c, wav, None, 0, Tb, None, dobs, ws0)
    wp.wp_stream_status(ws0)
    del ws0
    got = {}
    for lay in (wp.WP_PROBES_DENSE, wp.WP_PROBES_ALIGNED):
        M = wp.Model.from_survey(sv, m0)
        wp.wp_set_probe_layout(M.handle, lay)
        _, RS, XP = wp.wp_probe_layout(M.handle)
        ws = wp.workspace(wp.wp_workspace_bytes(M.handle, G.c, r, Tb, wp.WP_MODE_PROBED))
        Pu = torch.empty((S, r, RS), device="cuda")
        Pv = torch.empty((S, r, RS), device="cuda")
        d = torch.empty((S, nt, nrec), device="cuda")
        g = torch.empty(N, device="cuda")
        wp.wp_probe_forward(M.handle, G.c, wav, Q, r, Tb, Pu, d, ws)
        res = (d - dobs).contiguous()
        wp.wp_adjoint_image(M.handle, G.c, res, Q, r, Tb, 1.0 / r, Pu, g, Pv, ws)
        vol = torch.empty((81, N), device="cuda")
        wp.wp_offset_image(M.handle, Pu, Pv, r, S, 1.0 / r, 40, vol)
        wp.wp_stream_status(ws)
        wp.wp_offset_status()
        del ws
        shape = (sv.nz + 2 * sv.nbl, sv.nx + 2 * sv.nbl)
        if lay == wp.WP_PROBES_ALIGNED:
            # compare the aligned rows' points on the device, row by row of the grid
            Pu = Pu[:, :, :shape[0] * XP].reshape(S, r, shape[0], XP)[..., :shape[1]].reshape(S, r, -1)
            Pv = Pv[:, :, :shape[0] * XP].reshape(S, r, shape[0], XP)[..., :shape[1]].reshape(S, r, -1)
        got[lay] = (Pu.contiguous(), Pv.contiguous(), g, d, vol)
        M.close()
    dn, al = got[wp.WP_PROBES_DENSE], got[wp.WP_PROBES_ALIGNED]
    for k in range(4):
        assert torch.equal(dn[k], al[k]), k
    err = float(torch.linalg.vector_norm((al[4] - dn[4]).double()) / torch.linalg.vector_norm(dn[4].double()))
    assert err < 1e-5, err
    assert float(torch.linalg.vector_norm((al[4][40] - al[2]).double()) / torch.linalg.vector_norm(al[2].double())) < 1e-4
