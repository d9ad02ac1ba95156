"""Range-finder probes on the device (Sec. 2.1, [Q, ~] = qr(A Z)) against the oracle's
range_finder, which forms A as a dense FP64 matrix and calls LAPACK's QR.

- Data reading, A = D D^T with a random D (well conditioned): Q element by element
  (<= 1e-4, the bf16 hi/lo contraction's 2^-17 relative error times the sketch's condition
  number) and Q^T Q = I (<= 1e-5).
- Wavelet reading, A = (W W^T)^2 with W the causal convolution by a Ricker wavelet, one W
  shared by all shots: the trailing columns of Q are as ill-determined as the sketch's
  small singular values, so the check is the one the factorisation fixes at any
  conditioning: Q_gpu R_oracle reproduces the oracle's sketch Y = A Z (1e-4 relative),
  plus orthonormality.
- A probed gradient with a range-finder Q (the oracle's Q, scale 1) against the oracle's
  probed gradient with the same Q (1e-4), and the device Q giving a gradient error against
  the exact gradient no more than 10 % above the oracle Q's (the trailing columns of an
  ill-conditioned sketch may differ; the estimate must not get worse).
"""
import numpy as np
import pytest
import scipy.linalg as sl

from oracle import oracle as O
from paper_2201_06914_gb300 import inputs as I
from tests.cases import layered_case, rel
from tests.test_gpu_parity import GpuRun, _oracle_probed

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wp():
    from paper_2201_06914_gb300 import wp as _wp
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return _wp


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _device_rf(wp, D, nt, ncols, S, shared, power, Z, r):
    ws = wp.workspace(wp.wp_range_finder_workspace_bytes(nt, ncols, S, shared, r))
    Q = torch.full((S, nt, r), float("nan"), device="cuda")
    wp.wp_range_finder(_t(D), nt, ncols, S, shared, power, _t(Z), r, Q, ws)
    wp.wp_stream_status(ws)
    return Q.cpu().numpy().astype(np.float64)


def _orth_err(Q):
    return float(np.abs(Q.T @ Q - np.eye(Q.shape[1])).max())


@pytest.mark.parametrize("power", [1, 2])
def test_data_range_finder_matches_oracle(wp, power):
    rng = np.random.default_rng(4)
    S, nt, nrec, r = 3, 300, 60, 16
    D = rng.standard_normal((S, nt, nrec))
    Z = I.rademacher_shots(21, S, nt, r)
    Q = _device_rf(wp, D, nt, nrec, S, False, power, Z, r)
    for s in range(S):
        A = np.linalg.matrix_power(D[s] @ D[s].T, power)
        ref = O.range_finder(A, Z[s])
        err = float(np.abs(Q[s] - ref).max())
        print(f"power {power} shot {s}: max |dQ| {err:.2e}, orthogonality {_orth_err(Q[s]):.2e}")
        assert err <= 1e-4
        assert _orth_err(Q[s]) <= 1e-5


def test_wavelet_range_finder_reproduces_oracle_sketch(wp):
    S, nt, r, dt = 2, 400, 24, 2e-3
    w = I.ricker(nt, dt, 15.0)
    W = sl.toeplitz(w, np.zeros(nt))
    Z = I.rademacher_shots(5, S, nt, r)
    Q = _device_rf(wp, W, nt, nt, S, True, 2, Z, r)
    A = np.linalg.matrix_power(W @ W.T, 2)
    for s in range(S):
        Y = A @ Z[s].astype(np.float64)
        Qo, Ro = np.linalg.qr(Y)
        sg = np.sign(np.diag(Ro))
        Ro = Ro * sg[:, None]
        e = np.linalg.norm(Q[s] @ Ro - Y) / np.linalg.norm(Y)
        print(f"shot {s}: |Q R_o - Y| / |Y| {e:.2e}, orthogonality {_orth_err(Q[s]):.2e}, "
              f"cond(Y) {np.linalg.cond(Y):.1e}")
        assert e <= 1e-4
        assert _orth_err(Q[s]) <= 1e-5


def test_probed_gradient_with_range_finder_probes(wp):
    case = layered_case(ndim=2, nx=61, nz=45, nbl=8, nt=220, nshots=2, zi=0.3,
                        background="const", f0=15.0)
    r = 24
    nt = case.nt
    W = sl.toeplitz(case.wavelet, np.zeros(nt))
    A = np.linalg.matrix_power(W @ W.T, 2)
    Z = I.rademacher_shots(13, case.nshots, nt, r)
    Qo = np.stack([O.range_finder(A, Z[s]) for s in range(case.nshots)]).astype(np.float32)
    ref = _oracle_probed(case, Qo, 1.0)
    run = GpuRun(wp, case, case.m0)
    Pu, _ = run.forward(Qo, Tb=32)
    g, _ = run.adjoint(ref["res"], Qo, ref["Pu"], 1.0, Tb=32)
    e = rel(g, ref["g"].ravel())
    print(f"probed gradient with oracle range-finder Q: rel L2 vs oracle {e:.2e}")
    assert e <= 1e-4
    # the device's own range finder gives an estimate as close to the exact gradient
    Qd = _device_rf(wp, W, nt, nt, case.nshots, True, 2, Z, r).astype(np.float32)
    Pd, _ = run.forward(Qd, Tb=32)
    gd, _ = run.adjoint(ref["res"], Qd, Pd, 1.0, Tb=32)
    e_o = rel(ref["g"].ravel(), ref["gx"].ravel())
    e_d = rel(gd, ref["gx"].ravel())
    print(f"error vs exact gradient: oracle Q {e_o:.4f}, device Q {e_d:.4f}")
    assert e_d <= 1.1 * e_o + 1e-3
