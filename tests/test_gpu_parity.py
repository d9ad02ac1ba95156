"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same
seeded inputs.  Tolerances (relative L2): wavefield data and probed projections 1e-5, the
randomized gradient 1e-4 against the oracle's randomized gradient with the same Q."""
import numpy as np
import pytest

from tests.cases import close, layered_case, oracle_data, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wp():
    from paper_2201_06914_gb300 import wp as _wp
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return _wp


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


class GpuRun:
    """Runs the C-ABI calls of one case on the GPU."""

    def __init__(self, wp, case, m):
        self.wp, self.case = wp, case
        self.m = _t(m.ravel())
        self.M = wp.Model(case.ndim, case.nx, case.ny, case.nz, case.nbl, case.h, case.h,
                          case.h, case.dt, case.nt, self.m, case.damp_v)
        self.G = wp.Geometry(case.src, case.rec)
        self.wav = _t(case.wavelet)
        self.S, self.N, self.nt = case.nshots, case.N, case.nt

    def forward(self, Q, Tb=32):
        wp = self.wp
        r = Q.shape[-1]
        ws = wp.workspace(wp.wp_workspace_bytes(self.M.handle, self.G.c, r, Tb, wp.WP_MODE_PROBED))
        Pu = torch.full((self.S, r, self.N), float("nan"), device="cuda")
        d = torch.full((self.S, self.nt, self.G.nrec), float("nan"), device="cuda")
        wp.wp_probe_forward(self.M.handle, self.G.c, self.wav, _t(Q), r, Tb, Pu, d, ws)
        wp.wp_stream_status(ws)
        return Pu.cpu().numpy(), d.cpu().numpy()

    def adjoint(self, res, Q, Pu, scale, Tb=32):
        wp = self.wp
        r = Q.shape[-1]
        ws = wp.workspace(wp.wp_workspace_bytes(self.M.handle, self.G.c, r, Tb, wp.WP_MODE_PROBED))
        g = torch.full((self.N,), float("nan"), device="cuda")
        Pv = torch.full((self.S, r, self.N), float("nan"), device="cuda")
        wp.wp_adjoint_image(self.M.handle, self.G.c, _t(res), _t(Q), r, Tb, scale, _t(Pu), g,
                            Pv, ws)
        wp.wp_stream_status(ws)
        return g.cpu().numpy(), Pv.cpu().numpy()

    def exact(self, d_obs, mode=None, ncheck=1):
        wp = self.wp
        mode = wp.WP_MODE_EXACT_FULL if mode is None else mode
        ws = wp.workspace(wp.wp_workspace_bytes(self.M.handle, self.G.c, 0, ncheck, mode))
        g = torch.full((self.N,), float("nan"), device="cuda")
        J = torch.zeros(1, dtype=torch.float64, device="cuda")
        d = torch.empty((self.S, self.nt, self.G.nrec), device="cuda")
        wp.wp_exact_gradient(self.M.handle, self.G.c, self.wav, _t(d_obs), g, J, d, mode,
                             ncheck, ws)
        wp.wp_stream_status(ws)
        return g.cpu().numpy(), float(J.item()), d.cpu().numpy()


def _probes(case, r, seed=0):
    from paper_2201_06914_gb300.inputs import rademacher_shots
    return rademacher_shots(seed, case.nshots, case.nt, r)


def _oracle_probed(case, Q, scale):
    from oracle import oracle as O
    grid = case.oracle_grid()
    d_obs = oracle_data(case, "true")
    out = dict(Pu=[], Pv=[], d=[], res=[], g=0.0, gx=0.0, J=0.0)
    for s in range(case.nshots):
        f = O.forward(grid, case.m0.astype(np.float64), case.src[s], case.wavelet, case.rec[s],
                      Q=Q[s], want_udd=True)
        res = f["d"] - d_obs[s]
        a = O.adjoint(grid, case.m0.astype(np.float64), case.rec[s], res, Q=Q[s], udd=f["udd"])
        out["Pu"].append(f["Pu"].reshape(Q.shape[-1], -1))
        out["Pv"].append(a["Pv"].reshape(Q.shape[-1], -1))
        out["d"].append(f["d"])
        out["res"].append(res)
        out["g"] = out["g"] + O.probed_image(f["Pu"], a["Pv"], scale)
        out["gx"] = out["gx"] + a["g"]
        out["J"] += O.misfit(f["d"], d_obs[s])
    for k in ("Pu", "Pv", "d", "res"):
        out[k] = np.stack(out[k])
    out["d_obs"] = d_obs
    return out


def test_probe_accumulate_matches_definition(wp):
    """The tcgen05 contraction alone: P += scale * A^T Q for Rademacher and orthonormal Q,
    a ragged point count and a block that starts mid-probe-matrix."""
    rng = np.random.default_rng(1)
    for kind, r, S, cnt, npts, nt, t0 in (
            ("rademacher", 8, 2, 100, 1000, 160, 40), ("orthonormal", 40, 2, 100, 1000, 160, 40),
            ("rademacher", 130, 2, 100, 1000, 160, 40),
            # 128-aligned point counts take the pipelined bulk-copy kernel
            ("rademacher", 64, 3, 150, 1024, 200, 16), ("orthonormal", 24, 2, 64, 2048, 64, 0),
            ("orthonormal", 200, 1, 77, 384, 256, 8),
            # above 128 probes: 16-probe epilogue slices; exact bf16 probes stage no lo image
            ("rademacher", 256, 2, 130, 1024, 300, 24), ("orthonormal", 256, 1, 64, 1024, 320, 8),
            # above 256 probes: one accumulator of 512 columns, two MMAs per product (with and
            # without the lo image); unaligned points: the per-tile kernel in 256-probe slices
            ("rademacher", 448, 2, 130, 1024, 300, 24), ("orthonormal", 320, 1, 64, 1024, 384, 0),
            ("orthonormal", 300, 1, 40, 1000, 320, 8)):
        A = rng.standard_normal((S, cnt, npts)).astype(np.float32)
        if kind == "rademacher":
            Q = rng.choice([-1.0, 1.0], size=(S, nt, r)).astype(np.float32)
        else:
            Q = np.stack([np.linalg.qr(rng.standard_normal((nt, r)))[0] for _ in range(S)]).astype(np.float32)
        P0 = rng.standard_normal((S, r, npts)).astype(np.float32)
        P = _t(P0)
        ws = wp.workspace(wp.wp_probe_accumulate_workspace_bytes(S, nt, r))
        wp.wp_probe_accumulate(_t(A), cnt, npts, S, _t(Q), nt, t0, r, 0.5, P, ws)
        wp.wp_stream_status(ws)
        want = P0 + 0.5 * np.einsum("stx,sti->six", A.astype(np.float64),
                                    Q[:, t0:t0 + cnt].astype(np.float64))
        assert rel(P.cpu().numpy() - P0, want - P0) < 1e-5, kind


@pytest.mark.parametrize("off_grid", [False, True])
def test_forward_adjoint_2d_parity(wp, off_grid):
    case = layered_case(ndim=2, nx=83, nz=53, nbl=10, nt=250, nshots=2, off_grid=off_grid)
    r = 12
    Q = _probes(case, r)
    ref = _oracle_probed(case, Q, 1.0 / r)
    run = GpuRun(wp, case, case.m0)
    Pu, d = run.forward(Q, Tb=32)
    ok, err = close(d, ref["d"], 1e-5)
    assert ok, err
    ok, err = close(Pu, ref["Pu"], 1e-5)
    assert ok, err
    g, Pv = run.adjoint(ref["res"], Q, ref["Pu"], 1.0 / r, Tb=32)
    ok, err = close(Pv, ref["Pv"], 1e-5)
    assert ok, err
    ok, err = close(g, ref["g"].ravel(), 1e-4)
    assert ok, err


def test_exact_gradient_2d_parity(wp):
    case = layered_case(ndim=2, nx=75, nz=49, nbl=10, nt=230, nshots=2, off_grid=True, zi=0.3,
                        background="const")
    ref = _oracle_probed(case, _probes(case, 4), 0.25)
    run = GpuRun(wp, case, case.m0)
    g, J, d = run.exact(ref["d_obs"])
    ok, err = close(d, ref["d"], 1e-5)
    assert ok, err
    assert abs(J - ref["J"]) / ref["J"] < 1e-4
    ok, err = close(g, ref["gx"].ravel(), 1e-4)
    assert ok, err
    gc, Jc, _ = run.exact(ref["d_obs"], mode=wp.WP_MODE_EXACT_CHECKPOINT, ncheck=37)
    np.testing.assert_array_equal(gc, g)  # recomputation from checkpoints is bit-identical
    assert Jc == J


def test_forward_adjoint_3d_parity(wp):
    case = layered_case(ndim=3, nx=37, ny=29, nz=41, nbl=6, nt=150, nshots=2, off_grid=True,
                        zi=0.3, background="const")
    r = 8
    Q = _probes(case, r)
    ref = _oracle_probed(case, Q, 1.0 / r)
    run = GpuRun(wp, case, case.m0)
    Pu, d = run.forward(Q, Tb=48)
    ok, err = close(d, ref["d"], 1e-5)
    assert ok, err
    ok, err = close(Pu, ref["Pu"], 1e-5)
    assert ok, err
    g, Pv = run.adjoint(ref["res"], Q, ref["Pu"], 1.0 / r, Tb=48)
    ok, err = close(Pv, ref["Pv"], 1e-5)
    assert ok, err
    ok, err = close(g, ref["g"].ravel(), 1e-4)
    assert ok, err
    gx, J, _ = run.exact(ref["d_obs"])
    ok, err = close(gx, ref["gx"].ravel(), 1e-4)
    assert ok, err


def test_orthonormal_full_basis_recovers_exact_gradient_gpu(wp):
    """Eq. 3 with Q an orthonormal nt x nt basis and scale 1 equals Eq. 2: the GPU probed
    gradient and the GPU exact gradient both match the oracle's exact gradient."""
    case = layered_case(ndim=2, nx=41, nz=37, nbl=8, nt=120, nshots=1, zi=0.3,
                        background="const")
    ref = _oracle_probed(case, _probes(case, 4), 0.25)
    rng = np.random.default_rng(5)
    Q = np.linalg.qr(rng.standard_normal((case.nt, case.nt)))[0][None].astype(np.float32)
    run = GpuRun(wp, case, case.m0)
    Pu, d = run.forward(Q, Tb=32)
    g, _ = run.adjoint(ref["res"], Q, Pu, 1.0, Tb=32)
    gx, _, _ = run.exact(ref["d_obs"])
    ok, err = close(g, ref["gx"].ravel(), 1e-4)
    assert ok, err
    ok, err = close(gx, ref["gx"].ravel(), 1e-4)
    assert ok, err


@pytest.mark.parametrize("r,Tb,nt", [(5, 16, 70), (17, 64, 40), (64, 32, 97)])
def test_ragged_probe_blocks(wp, r, Tb, nt):
    """r not a multiple of 16, nt shorter than one block, nt not a multiple of Tb."""
    case = layered_case(ndim=2, nx=29, nz=23, nbl=5, nt=nt, nshots=3, off_grid=True, zi=0.3,
                        background="const", f0=25.0)
    Q = _probes(case, r, seed=3)
    ref = _oracle_probed(case, Q, 1.0 / r)
    run = GpuRun(wp, case, case.m0)
    Pu, d = run.forward(Q, Tb=Tb)
    ok, err = close(d, ref["d"], 1e-5)
    assert ok, err
    ok, err = close(Pu, ref["Pu"], 1e-5)
    assert ok, err
    g, Pv = run.adjoint(ref["res"], Q, ref["Pu"], 1.0 / r, Tb=Tb)
    ok, err = close(Pv, ref["Pv"], 1e-5)
    assert ok, err
    ok, err = close(g, ref["g"].ravel(), 1e-4)
    assert ok, err


def test_status_codes(wp):
    case = layered_case(ndim=2, nx=21, nz=17, nbl=4, nt=20)
    m = _t(case.m0.ravel())
    with pytest.raises(wp.WpError) as e:
        wp.Model(2, case.nx, 1, case.nz, case.nbl, case.h, case.h, case.h, case.dt * 2.0,
                 case.nt, m)
    assert e.value.status == wp.WP_ERR_UNSTABLE
    bad = m.clone()
    bad[7] = float("nan")
    with pytest.raises(wp.WpError) as e:
        wp.Model(2, case.nx, 1, case.nz, case.nbl, case.h, case.h, case.h, case.dt, case.nt, bad)
    assert e.value.status == wp.WP_ERR_NONFINITE
    run = GpuRun(wp, case, case.m0)
    Q = _probes(case, 4)
    small = wp.workspace(1024)
    with pytest.raises(wp.WpError) as e:
        wp.wp_probe_forward(run.M.handle, run.G.c, run.wav, _t(Q), 4, 16,
                            torch.empty((1, 4, run.N), device="cuda"), None, small)
    assert e.value.status == wp.WP_ERR_OOM
    with pytest.raises(wp.WpError) as e:
        wp.wp_probe_forward(run.M.handle, run.G.c, run.wav, _t(Q), 4, 24,
                            torch.empty((1, 4, run.N), device="cuda"), None, small)
    assert e.value.status == wp.WP_ERR_INVALID
    far = wp.Geometry(np.array([[[1e6, 0.0, 10.0]]]), case.rec)
    ws = wp.workspace(wp.wp_workspace_bytes(run.M.handle, far.c, 4, 16, wp.WP_MODE_PROBED))
    with pytest.raises(wp.WpError) as e:
        wp.wp_probe_forward(run.M.handle, far.c, run.wav, _t(Q), 4, 16,
                            torch.empty((1, 4, run.N), device="cuda"), None, ws)
    assert e.value.status == wp.WP_ERR_INVALID
