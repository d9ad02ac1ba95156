"""Failure path of the device waits: a wait that nothing completes gives up after about one
second, the host reads WP_ERR_TIMEOUT through wp_stream_status, and the CUDA context stays
usable (a probed forward afterwards still matches the oracle).  Nothing faults or traps."""
import time

import numpy as np
import pytest

from tests.cases import layered_case, oracle_shot, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_bounded_wait_gives_up_and_context_survives():
    from paper_2201_06914_gb300 import wp
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    t0 = time.perf_counter()
    wp.wp_check_bounded_wait(ws)
    with pytest.raises(wp.WpError) as e:
        wp.wp_stream_status(ws, timeout_s=60.0)
    waited = time.perf_counter() - t0
    assert e.value.status == wp.WP_ERR_TIMEOUT
    assert 0.1 < waited < 30.0, waited

    # the context is still usable
    case = layered_case(ndim=2, nx=41, nz=33, nbl=6, nt=80, nshots=1)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    M = wp.Model(2, case.nx, 1, case.nz, case.nbl, case.h, case.h, case.h, case.dt, case.nt,
                 t(case.m0.ravel()), case.damp_v)
    G = wp.Geometry(case.src, case.rec)
    ws2 = wp.workspace(wp.wp_workspace_bytes(M.handle, G.c, 0, 16, wp.WP_MODE_PROBED))
    d = torch.empty((1, case.nt, G.nrec), device="cuda")
    wp.wp_probe_forward(M.handle, G.c, t(case.wavelet), None, 0, 16, None, d, ws2)
    wp.wp_stream_status(ws2)
    assert rel(d.cpu().numpy()[0], oracle_shot(case, 0, case.m0)["d"]) < 1e-5
