"""wp_probe_accumulate_static: the probe contraction for callers that may not allocate
device memory.

Such callers (a plug-in inside an application whose framework owns all GPU memory, or a
service with a fixed memory budget) cannot hand the library a workspace, so this entry
point keeps its scratch in a fixed 16 MiB device array inside libwp.so.  These tests call
it through the C ABI twice in a row, with different inputs each time, and check each
result against the workspace-based wp_probe_accumulate within the parity tolerance of the
other GPU tests (relative L2 1e-5), and against the definition of the contraction
(P += scale * sum_t A[t] Q[t0 + t], an FP64 einsum) within the same 1e-5.  The second call
shows that scratch left over from the first call does not leak into the next result, and
wp_static_status reads the call's error flag from the static array.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_static_scratch_matches_workspace_version_twice():
    from paper_2201_06914_gb300 import wp
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    rng = np.random.default_rng(11)
    cases = [(2, 96, 1500, 200, 16, 24, "rademacher"), (3, 130, 777, 300, 40, 64, "orthonormal")]
    for S, cnt, npts, nt, t0, r, kind in cases:
        A = rng.standard_normal((S, cnt, npts)).astype(np.float32)
        if kind == "rademacher":
            Q = rng.choice([-1.0, 1.0], size=(S, nt, r)).astype(np.float32)
        else:
            Q = np.stack([np.linalg.qr(rng.standard_normal((nt, r)))[0]
                          for _ in range(S)]).astype(np.float32)
        P0 = rng.standard_normal((S, r, npts)).astype(np.float32)
        P_ws = _t(P0)
        ws = wp.workspace(wp.wp_probe_accumulate_workspace_bytes(S, nt, r))
        wp.wp_probe_accumulate(_t(A), cnt, npts, S, _t(Q), nt, t0, r, 0.25, P_ws, ws)
        P_st = _t(P0)
        wp.wp_probe_accumulate_static(_t(A), cnt, npts, S, _t(Q), nt, t0, r, 0.25, P_st)
        wp.wp_static_status(timeout_s=60.0)
        want = P_ws.cpu().numpy() - P0
        got = P_st.cpu().numpy() - P0
        assert _rel(got, want) < 1e-5, kind
        defn = 0.25 * np.einsum("stx,sti->six", A.astype(np.float64),
                                Q[:, t0:t0 + cnt].astype(np.float64))
        assert _rel(got, defn) < 1e-5, kind


def test_static_scratch_rejects_oversized_request():
    from paper_2201_06914_gb300 import wp
    S, nt, r, npts, cnt = 8, 8000, 256, 128, 16
    with pytest.raises(wp.WpError) as e:
        wp.wp_probe_accumulate_static(_t(np.zeros((S, cnt, npts))), cnt, npts, S,
                                      _t(np.zeros((S, nt, r))), nt, 0, r, 1.0,
                                      _t(np.zeros((S, r, npts))))
    assert e.value.status == wp.WP_ERR_OOM
    assert "16 MiB" in wp.wp_last_error()
