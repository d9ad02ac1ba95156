"""Two time steps per launch (temporal blocking of the 2-D isotropic sweeps).

A pair of steps performs the arithmetic of two single-step launches operation for
operation, so every output of the probed forward (P_u, recorded data), the probed adjoint
(gradient, P_v) and the exact gradients (full history and checkpointed) must be bitwise
the same with two-step launches switched on and off.  The tilings are forced small so that
sources and receivers fall into the 8-column tile overlaps, across segment boundaries,
into segments shorter than the 4-plane halo, and into the absorbing layer; nt is odd so
that the last step runs alone.  One configuration is also checked against the FP64 oracle
(the interface is shallow enough for its reflection to reach the receivers within nt).
"""
import os

import numpy as np
import pytest

from tests.cases import close, layered_case, oracle_data, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _case():
    case = layered_case(ndim=2, nx=261, nz=61, nbl=10, nt=151, nshots=3, off_grid=True, zi=0.2,
                        background="const")
    h, nbl = case.h, case.nbl
    # padded grid coordinates -> metres from the first interior point
    at = lambda gx, gz: [(gx - nbl) * h, 0.0, (gz - nbl) * h]
    case.src = np.array([[at(119.5, 12.3)],     # x corners 119/120: the 120-column tile overlap
                         [at(60.2, 25.5)],      # z corners 25/26: a 13-plane segment boundary
                         [at(3.3, 20.6)]])      # inside the absorbing layer
    return case


def _run(case, Q, env, Tb=32, ncheck=23):
    from paper_2201_06914_gb300 import wp
    saved = {k: os.environ.get(k) for k in ("WP_STENCIL2", "WP_STENCIL2_TZ", "WP_STENCIL_TX")}
    os.environ.update(env)
    try:
        M = wp.Model(2, case.nx, 1, case.nz, case.nbl, case.h, case.h, case.h, case.dt, case.nt,
                     _t(case.m0.ravel()), case.damp_v)
        G = wp.Geometry(case.src, case.rec)
        S, N, nt, r = case.nshots, case.N, case.nt, Q.shape[-1]
        ws = wp.workspace(wp.wp_workspace_bytes(M.handle, G.c, r, Tb, wp.WP_MODE_PROBED))
        Pu = torch.full((S, r, N), float("nan"), device="cuda")
        d = torch.full((S, nt, G.nrec), float("nan"), device="cuda")
        wav = _t(case.wavelet)
        wp.wp_probe_forward(M.handle, G.c, wav, _t(Q), r, Tb, Pu, d, ws)
        res = d - _t(case.d_obs)
        g = torch.full((N,), float("nan"), device="cuda")
        Pv = torch.full((S, r, N), float("nan"), device="cuda")
        wp.wp_adjoint_image(M.handle, G.c, res, _t(Q), r, Tb, 1.0 / r, Pu, g, Pv, ws)
        wp.wp_stream_status(ws)
        out = dict(Pu=Pu.cpu().numpy(), d=d.cpu().numpy(), g=g.cpu().numpy(), Pv=Pv.cpu().numpy())
        for name, mode, nck in (("gx", wp.WP_MODE_EXACT_FULL, 1), ("gc", wp.WP_MODE_EXACT_CHECKPOINT, ncheck)):
            wse = wp.workspace(wp.wp_workspace_bytes(M.handle, G.c, 0, nck, mode))
            ge = torch.full((N,), float("nan"), device="cuda")
            de = torch.empty((S, nt, G.nrec), device="cuda")
            wp.wp_exact_gradient(M.handle, G.c, wav, _t(case.d_obs), ge, None, de, mode, nck, wse)
            wp.wp_stream_status(wse)
            out[name] = ge.cpu().numpy()
            out["d_" + name] = de.cpu().numpy()
        M.close()
        return out
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.fixture(scope="module")
def case_and_probes():
    from paper_2201_06914_gb300.inputs import rademacher_shots
    case = _case()
    case.d_obs = oracle_data(case, "true")
    Q = rademacher_shots(2, case.nshots, case.nt, 8)
    return case, Q


@pytest.mark.parametrize("env", [
    {"WP_STENCIL_TX": "128", "WP_STENCIL2_TZ": "13"},   # 3 tiles of 120 core columns, 7 segments
    {"WP_STENCIL_TX": "256", "WP_STENCIL2_TZ": "5"},    # segments shorter than the halo
    {},                                                 # the library's own choice
])
def test_two_step_bitwise_equals_single_steps(case_and_probes, env):
    case, Q = case_and_probes
    one = _run(case, Q, dict(env, WP_STENCIL2="0"))
    two = _run(case, Q, dict(env, WP_STENCIL2="1"))
    for k in one:
        assert np.isfinite(two[k]).all(), k
        np.testing.assert_array_equal(two[k], one[k], err_msg=k)


def test_two_step_matches_oracle(case_and_probes):
    from oracle import oracle as O
    case, Q = case_and_probes
    out = _run(case, Q, {"WP_STENCIL_TX": "128", "WP_STENCIL2_TZ": "13", "WP_STENCIL2": "1"})
    grid = case.oracle_grid()
    r = Q.shape[-1]
    g = 0.0
    for s in range(case.nshots):
        f = O.forward(grid, case.m0.astype(np.float64), case.src[s], case.wavelet, case.rec[s], Q=Q[s])
        a = O.adjoint(grid, case.m0.astype(np.float64), case.rec[s], out["d"][s] - case.d_obs[s], Q=Q[s])
        ok, err = close(out["d"][s], f["d"], 1e-5)
        assert ok, err
        ok, err = close(out["Pu"][s], f["Pu"].reshape(r, -1), 1e-5)
        assert ok, err
        ok, err = close(out["Pv"][s], a["Pv"].reshape(r, -1), 1e-5)
        assert ok, err
        g = g + O.probed_image(f["Pu"], a["Pv"], 1.0 / r)
    ok, err = close(out["g"], np.ravel(g), 1e-4)
    assert ok, err


@pytest.mark.parametrize("nt,Tb,ncheck", [(1, 16, 2), (2, 16, 2), (3, 16, 5), (17, 16, 3), (33, 16, 8), (64, 32, 5)])
def test_two_step_schedules_short_runs_and_block_boundaries(nt, Tb, ncheck):
    """A single step, one pair, odd counts, a run ending one step after a probe block and
    checkpoint intervals too short for a pair: still bitwise equal to single steps."""
    from paper_2201_06914_gb300.inputs import rademacher_shots
    case = layered_case(ndim=2, nx=45, nz=37, nbl=6, nt=nt, nshots=2, off_grid=True, zi=0.2,
                        background="const")
    case.d_obs = oracle_data(case, "true")
    Q = rademacher_shots(4, case.nshots, nt, 4)
    one = _run(case, Q, {"WP_STENCIL2": "0"}, Tb=Tb, ncheck=ncheck)
    two = _run(case, Q, {"WP_STENCIL2": "1", "WP_STENCIL2_TZ": "7"}, Tb=Tb, ncheck=ncheck)
    for k in one:
        assert np.isfinite(two[k]).all(), k
        np.testing.assert_array_equal(two[k], one[k], err_msg=k)
