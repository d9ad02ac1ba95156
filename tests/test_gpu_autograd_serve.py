"""torch.autograd wrapper and continuous-batching server on the GPU.

- WaveMisfit: J(m) and dJ/dm through loss.backward() for the full-history, checkpointed
  and probed variants match the FP64 oracle (1e-4), and <dJ/dm, dm> matches a central
  finite difference of J computed by the same forward kernels (FP32: 2e-2).
- Server: every job's gradient is bit-identical when it runs alone and when it runs
  concurrently with other jobs of different sizes (own stream and workspace per job).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2201_06914_gb300 import inputs as I
from tests.cases import layered_case, oracle_data, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.fixture(scope="module")
def problem_case():
    from paper_2201_06914_gb300.autograd import Problem
    case = layered_case(ndim=2, nx=61, nz=45, nbl=8, nt=200, nshots=2, zi=0.3, background="const")
    d_obs = oracle_data(case, "true")
    Q = I.rademacher_shots(0, case.nshots, case.nt, 16)

    def make(variant):
        return Problem(2, case.nx, 1, case.nz, case.nbl, case.h, case.dt, case.nt, case.src, case.rec,
                       _t(case.wavelet), _t(d_obs), _t(Q), None, 32, variant, 37, case.damp_v)
    grid = case.oracle_grid()
    gx = 0.0
    gp = 0.0
    J = 0.0
    for s in range(case.nshots):
        J_s, g_s, _ = O.exact_gradient(grid, case.m0, case.src[s], case.wavelet, case.rec[s], d_obs[s])
        p = O.probed_gradient(grid, case.m0, case.src[s], case.wavelet, case.rec[s], d_obs[s], Q[s], 1 / 16)
        gx, gp, J = gx + g_s, gp + p["g_hat"], J + J_s
    return case, make, dict(J=J, gx=gx.ravel(), gp=gp.ravel())


@pytest.mark.parametrize("variant", ["full", "checkpoint", "probed"])
def test_autograd_gradient_matches_oracle(problem_case, variant):
    from paper_2201_06914_gb300.autograd import WaveMisfit
    case, make, ref = problem_case
    m = _t(case.m0.ravel()).requires_grad_(True)
    p = make(variant)
    loss = WaveMisfit.apply(m, p)
    loss.backward()
    assert p.last_variant == variant
    assert abs(loss.item() - ref["J"]) / ref["J"] < 1e-4
    want = ref["gp"] if variant == "probed" else ref["gx"]
    assert rel(m.grad.cpu().numpy(), want) < 1e-4


def test_autograd_finite_difference(problem_case):
    from paper_2201_06914_gb300.autograd import WaveMisfit
    case, make, _ = problem_case
    p = make("full")
    m0 = _t(case.m0.ravel())
    m = m0.clone().requires_grad_(True)
    WaveMisfit.apply(m, p).backward()
    dm = _t(np.random.default_rng(0).standard_normal(m0.shape[0]) * case.m0.ravel() * 0.02)
    h = 1.0
    Jp = WaveMisfit.apply(m0 + h * dm, p).item()
    Jm = WaveMisfit.apply(m0 - h * dm, p).item()
    fd = (Jp - Jm) / (2 * h)
    an = float(torch.dot(m.grad.double(), dm.double()))
    assert abs(fd - an) / abs(an) < 2e-2


def _job(name, nx, nz, nt, r, seed, arrival):
    from paper_2201_06914_gb300.serve import ShotJob
    case = layered_case(ndim=2, nx=nx, nz=nz, nbl=6, nt=nt, nshots=1, zi=0.3, background="const", seed=seed)
    d_obs = oracle_data(case, "true")
    Q = I.rademacher_shots(seed, 1, nt, r)
    return ShotJob(name, 2, nx, 1, nz, 6, case.h, case.dt, nt, case.m0, case.src, case.rec,
                   case.wavelet, d_obs, Q, 32, arrival)


def test_server_results_identical_alone_and_in_mix():
    from paper_2201_06914_gb300.serve import GpuBackend, Scheduler
    specs = [("a", 81, 51, 240, 8), ("b", 121, 61, 300, 16), ("c", 61, 41, 180, 32),
             ("d", 101, 71, 260, 8), ("e", 71, 45, 200, 16)]
    jobs = [_job(n, nx, nz, nt, r, k, 0.002 * k) for k, (n, nx, nz, nt, r) in enumerate(specs)]
    backend = GpuBackend()
    alone = {}
    for j in jobs:
        res = Scheduler(backend, mem_budget=40e9, max_active=1).run([j])
        assert res[j.name].ok, res[j.name].error
        alone[j.name] = res[j.name].g
    sched = Scheduler(backend, mem_budget=40e9, max_active=4)
    mix = sched.run(jobs)
    for j in jobs:
        assert mix[j.name].ok, mix[j.name].error
        np.testing.assert_array_equal(mix[j.name].g, alone[j.name])
    st = Scheduler.stats(mix)
    assert st["ok"] == len(jobs) and st["p99_s"] > 0
