"""Multi-shot stack with independent probes per shot (Sec. 3: the noise of the randomized
estimate stacks out).  Two geometries: surface shots and receivers, and a reciprocity-shaped
(ocean-bottom node) one where the 16 sources are nodes on the sea floor, just above the
reflector, recorded along the surface.  For stacks of 1, 4 and 16 shots the error of the
probed stacked gradient against the exact stacked gradient (both from the GPU path, the
exact one checked against the oracle elsewhere) falls: the oracle gives 3.77, 2.82, 1.29
(surface) and 1.42, 1.17, 0.59 (nodes) for these seeds with r = 16."""
import numpy as np
import pytest

from tests.cases import layered_case, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("node_depth", [None, 0.45])
def test_noise_stacks_out_over_shots(node_depth):
    from paper_2201_06914_gb300 import inputs as I
    from paper_2201_06914_gb300 import wp
    case = layered_case(ndim=2, nx=121, nz=61, nbl=8, nt=360, nshots=16, zi=0.5,
                        background="const", seed=3)
    src = case.src.copy()
    if node_depth is not None:
        src[:, 0, 2] = node_depth * (case.nz - 1) * case.h   # nodes on the sea floor
    r, Tb = 16, 32
    Mt = wp.Model(2, case.nx, 1, case.nz, case.nbl, case.h, case.h, case.h, case.dt, case.nt,
                  _t(case.m_true.ravel()), case.damp_v)
    M0 = wp.Model(2, case.nx, 1, case.nz, case.nbl, case.h, case.h, case.h, case.dt, case.nt,
                  _t(case.m0.ravel()), case.damp_v)
    wav = _t(case.wavelet)
    errs = {}
    for S in (1, 4, 16):
        idx = np.linspace(0, 15, S).round().astype(int)
        G = wp.Geometry(src[idx], case.rec[idx])
        N, nrec = case.N, G.nrec
        ws = wp.workspace(max(wp.wp_workspace_bytes(M0.handle, G.c, r, Tb, wp.WP_MODE_PROBED),
                              wp.wp_workspace_bytes(M0.handle, G.c, 0, 1, wp.WP_MODE_EXACT_FULL)))
        nbytes = ws.numel()
        d_obs = torch.empty((S, case.nt, nrec), device="cuda")
        wp.wp_probe_forward(Mt.handle, G.c, wav, None, 0, Tb, None, d_obs, ws)
        g_ex = torch.empty(N, device="cuda")
        wp.wp_exact_gradient(M0.handle, G.c, wav, d_obs, g_ex, None, None, wp.WP_MODE_EXACT_FULL, 1, ws)
        Q = _t(np.stack([I.rademacher(100 + int(k), case.nt, r) for k in idx]))
        Pu = torch.empty((S, r, N), device="cuda")
        d = torch.empty((S, case.nt, nrec), device="cuda")
        g = torch.empty(N, device="cuda")
        wp.wp_probe_forward(M0.handle, G.c, wav, Q, r, Tb, Pu, d, ws)
        res = (d - d_obs).contiguous()
        wp.wp_adjoint_image(M0.handle, G.c, res, Q, r, Tb, 1.0 / r, Pu, g, None, ws)
        wp.wp_stream_status(ws)
        errs[S] = rel(g.cpu().numpy(), g_ex.cpu().numpy())
        assert nbytes > 0
    assert errs[16] < 0.5 * errs[1], errs
    assert errs[16] < errs[4] < 1.2 * errs[1], errs
