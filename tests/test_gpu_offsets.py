"""GPU parity of the subsurface-offset image volume (Eq. 4) against the oracle's
definition: seeded random projections on ragged 2-D/3-D grids (rows spanning several
128-point tiles and a partial one, shot x probe counts across the 64-wide contraction
chunks, offsets 0 .. 64, so the accumulator spans one or two tcgen05 N halves), and the
volume of a real probed gradient whose offset-0 slice is the image."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.cases import layered_case, oracle_data, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wp():
    from paper_2201_06914_gb300 import wp as _wp
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return _wp


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _model(wp, ndim, nx, ny, nz, nbl):
    NX, NY, NZ = nx + 2 * nbl, (ny + 2 * nbl if ndim == 3 else 1), nz + 2 * nbl
    m = _t(np.full(NX * NY * NZ, 1 / 1500.0 ** 2))
    return wp.Model(ndim, nx, ny, nz, nbl, 10.0, 10.0, 10.0, 1e-3, 16, m, 1500.0), (NZ, NY, NX) if ndim == 3 else (NZ, NX)


def _oracle_volume(Pu, Pv, nh, scale):
    return sum(O.offset_image(Pu[s], Pv[s], nh, scale) for s in range(Pu.shape[0]))


@pytest.mark.parametrize("ndim,nx,ny,nz,r,S,nh", [
    (2, 290, 1, 7, 17, 2, 40),    # rows of 306: two full tiles and a partial one
    (2, 130, 1, 5, 64, 1, 64),    # largest offset range, 4 probe chunks
    (2, 100, 1, 4, 1, 3, 0),      # offset 0 only, one probe
    (2, 57, 1, 6, 33, 1, 7),      # a single partial tile, ragged probe chunk
    (3, 40, 6, 5, 16, 2, 21),     # 3-D: offsets along x within each (z, y) row
])
def test_offset_volume_random_parity(wp, ndim, nx, ny, nz, r, S, nh):
    M, shape = _model(wp, ndim, nx, ny, nz, 8)
    N = int(np.prod(shape))
    rng = np.random.default_rng(nx + r + nh)
    Pu = rng.standard_normal((S, r) + shape)
    Pv = rng.standard_normal((S, r) + shape)
    out = torch.full((2 * nh + 1, N), float("nan"), device="cuda")
    wp.wp_offset_image(M.handle, _t(Pu), _t(Pv), r, S, 0.25, nh, out)
    wp.wp_offset_status()
    got = out.cpu().numpy().reshape((2 * nh + 1,) + shape)
    ref = _oracle_volume(Pu, Pv, nh, 0.25)
    assert np.all(np.isfinite(got))
    assert rel(got, ref) < 1e-5
    # cells whose shifted points leave the row are exactly zero
    if nh > 0:
        assert np.all(got[0][..., :nh] == 0) and np.all(got[-1][..., -nh:] == 0)


def test_offset_volume_of_a_probed_gradient(wp):
    case = layered_case(ndim=2, nx=71, nz=41, nbl=8, nt=160, nshots=2, zi=0.3, background="const")
    d_obs = oracle_data(case, "true")
    from paper_2201_06914_gb300 import inputs as I
    r, Tb, nh = 24, 32, 10
    Q = I.rademacher_shots(5, case.nshots, case.nt, r)
    m = _t(case.m0.ravel())
    M = wp.Model(case.ndim, case.nx, case.ny, case.nz, case.nbl, case.h, case.h, case.h, case.dt,
                 case.nt, m, case.damp_v)
    G = wp.Geometry(case.src, case.rec)
    ws = wp.workspace(wp.wp_workspace_bytes(M.handle, G.c, r, Tb, wp.WP_MODE_PROBED))
    S, N = case.nshots, case.N
    Pu = torch.empty((S, r, N), device="cuda")
    Pv = torch.empty((S, r, N), device="cuda")
    d = torch.empty((S, case.nt, G.nrec), device="cuda")
    g = torch.empty(N, device="cuda")
    wp.wp_probe_forward(M.handle, G.c, _t(case.wavelet), _t(Q), r, Tb, Pu, d, ws)
    res = d - _t(d_obs)
    wp.wp_adjoint_image(M.handle, G.c, res.contiguous(), _t(Q), r, Tb, 1.0 / r, Pu, g, Pv, ws)
    out = torch.empty((2 * nh + 1, N), device="cuda")
    wp.wp_offset_image(M.handle, Pu, Pv, r, S, 1.0 / r, nh, out)
    wp.wp_stream_status(ws)
    wp.wp_offset_status()
    vol = out.cpu().numpy()
    # the volume runs on the tensor cores with a bf16 hi/lo split of both operands (16
    # significant bits each), the image in FP32 on CUDA cores: they agree to the split's
    # few parts in 10^6
    assert rel(vol[nh], g.cpu().numpy()) < 1e-5
    ref = _oracle_volume(Pu.cpu().numpy().reshape((S, r) + case.shape),
                         Pv.cpu().numpy().reshape((S, r) + case.shape), nh, 1.0 / r)
    assert rel(vol.reshape(ref.shape), ref) < 1e-5


def test_offset_arguments_rejected(wp):
    M, shape = _model(wp, 2, 20, 1, 5, 4)
    x = torch.zeros(int(np.prod(shape)) * 2, device="cuda")
    for r, S, nh in [(0, 1, 3), (2, 0, 3), (2, 1, -1), (2, 1, 65)]:
        with pytest.raises(wp.WpError):
            wp.wp_offset_image(M.handle, x, x, r, S, 1.0, nh, x)
