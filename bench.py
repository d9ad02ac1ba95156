#!/usr/bin/env python
"""Benchmark of the probed (randomized-trace) adjoint-state gradient on GB300.

Workload (default): the 2-D layered + salt model of 1601 x 401 points at 12.5 m (padded
1681 x 481), 4000 time steps, 15 Hz Ricker, 1601 receivers, 64 shots, r = 64 Rademacher
probes per shot.  One step = the stacked gradient of all shots: probed forward (stencil +
tensor-core probe contraction), residual, probed adjoint with the randomized imaging
condition.  The exact full-history gradient is timed on the same shots for comparison and
its result is the reference for the relative error of the probed gradient.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "shot-gradients/s and Gpt-updates/s (probed vs exact GPU) at rel.err ≤0.1; HBM/shot"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--shots", type=int, default=64)
    p.add_argument("--nt", type=int, default=4000)
    p.add_argument("--r", type=int, default=64)
    p.add_argument("--tb", type=int, default=256)
    p.add_argument("--nx", type=int, default=1601)
    p.add_argument("--nz", type=int, default=401)
    p.add_argument("--no-exact", action="store_true")
    p.add_argument("--probes", default="rademacher", choices=["rademacher", "wavelet", "data"],
                   help="probing matrix: Rademacher, or the range finder qr(A Z) with A from "
                        "the wavelet or the shot's data")
    p.add_argument("--offsets", type=int, default=40,
                   help="half-width of the subsurface-offset volume timed after the step (0: skip)")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-op", action="store_true", help="skip the rel.err <= 0.1 operating point")
    p.add_argument("--no-3d", action="store_true", help="skip the 3-D checkpointed workload")
    p.add_argument("--no-serving", action="store_true", help="skip the short serving run")
    p.add_argument("--no-tti", action="store_true", help="skip the 3-D TTI workload")
    p.add_argument("--serving-jobs", type=int, default=48, help="jobs of the short serving run")
    p.add_argument("--cpu-steps", type=int, default=120, help="oracle sample length (steps)")
    p.add_argument("--workload", default="salt2d", choices=["salt2d", "serving", "salt3d", "tti3d"])
    p.add_argument("--nx3", type=int, default=512)
    p.add_argument("--ny3", type=int, default=512)
    p.add_argument("--nz3", type=int, default=256)
    p.add_argument("--nt3", type=int, default=2500)
    p.add_argument("--r3", type=int, default=32)
    p.add_argument("--tb3", type=int, default=64)
    p.add_argument("--ncheck3", type=int, default=64)
    p.add_argument("--jobs", type=int, default=256, help="serving: number of jobs")
    p.add_argument("--rate", type=float, default=0.0, help="serving: arrivals/s (0: auto)")
    return p.parse_args()


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def workload(args, world=1, rank=0):
    """The rank's slice of a survey of world*shots shots (weak scaling: fixed shots/GPU)."""
    from paper_2201_06914_gb300 import inputs as I
    from paper_2201_06914_gb300.dist import shot_range
    sv = I.config_salt_2d(nx=args.nx, nz=args.nz, nt=args.nt, r=args.r, nshots=args.shots * world)
    sl = shot_range(sv.nshots, rank, world)
    sv.src, sv.rec = sv.src[sl.start:sl.stop], sv.rec[sl.start:sl.stop]
    sv.probe_seed = sl.start
    return sv


# ----------------------------------------------------------------------------------------
# CPU oracle timing (bounded sample of the same workload)
# ----------------------------------------------------------------------------------------
def oracle_sample(sv, r, steps):
    """Time the oracle's probed gradient of one shot over `steps` time steps at the full
    spatial size.  Returns (seconds of the sample that ran, seconds per full shot-gradient
    extrapolated linearly in steps, sample description, cores)."""
    from oracle import oracle as O
    from paper_2201_06914_gb300 import inputs as I
    grid = O.Grid(2, sv.nx, 1, sv.nz, sv.nbl, steps, sv.spacing, sv.spacing, sv.spacing,
                  sv.dt, sv.damp_v)
    O.build()
    m0 = sv.m_padded("background").astype(np.float64)
    w = I.ricker(steps, sv.dt, sv.f0)
    Q = I.rademacher(0, steps, r)
    d_obs = np.zeros((steps, sv.rec.shape[1]))
    t0 = time.perf_counter()
    O.probed_gradient(grid, m0, sv.src[0], w, sv.rec[0], d_obs, Q, 1.0 / r)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = (f"1 shot x {steps} of {sv.nt} steps (forward+adjoint, r={r}) at full "
            f"{sv.nx}x{sv.nz} size, extrapolated linearly in steps")
    return dt, dt * sv.nt / steps, desc, cores


def oracle_two_layer(repeats=5):
    """The oracle's probed gradient of the two-layer workload (201 x 201 at 10 m + 40-cell
    sponge, 1000 steps, r = 8, one shot) run in full: median of `repeats` runs after one
    warm-up; the observed data are modelled once, untimed."""
    from oracle import oracle as O
    from paper_2201_06914_gb300 import inputs as I
    O.build()
    sv = I.config_two_layer()
    grid = O.Grid(2, sv.nx, 1, sv.nz, sv.nbl, sv.nt, sv.spacing, sv.spacing, sv.spacing,
                  sv.dt, sv.damp_v)
    w = sv.wavelet()
    d_obs = O.forward(grid, sv.m_padded("true").astype(np.float64), sv.src[0], w, sv.rec[0])["d"]
    m0 = sv.m_padded("background").astype(np.float64)
    Q = sv.probes()[0]
    times = []
    for k in range(repeats + 1):
        t0 = time.perf_counter()
        O.probed_gradient(grid, m0, sv.src[0], w, sv.rec[0], d_obs, Q, 1.0 / sv.r)
        if k:
            times.append(time.perf_counter() - t0)
    med = float(np.median(times))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": 1.0 / med, "unit": "shot-gradients/s", "cores": cores, "kind": "oracle",
            "sample": f"two-layer 201x201 (+40-cell sponge), 1000 steps, r=8, one shot, in full: "
                      f"median of {repeats} runs after one warm-up",
            "ms_per_shot_gradient": med * 1e3, "runs_ms": [t * 1e3 for t in times]}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    sv = workload(args)
    for _ in range(args.warmup):
        oracle_sample(sv, args.r, max(10, args.cpu_steps // 4))
    ran, per_shot = [], []
    for _ in range(args.steps):
        t, full, desc, cores = oracle_sample(sv, args.r, args.cpu_steps)
        ran.append(t)
        per_shot.append(full)
    val = 1.0 / float(np.mean(per_shot))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "shot-gradients/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            # the time of the sample each step actually ran; the full shot-gradient time is
            # the separate extrapolated field below
            "ms_per_step": float(np.mean(ran)) * 1e3,
            "extrapolated_ms_per_shot_gradient": float(np.mean(per_shot)) * 1e3,
            "sample_steps": args.cpu_steps,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"salt_2d_{sv.nx}x{sv.nz}_nt{sv.nt}_r{args.r}",
                       "note": "FP64 CPU oracle, one shot per step, a sample of "
                               f"{args.cpu_steps} of {sv.nt} steps (value extrapolated)"},
            "cpu_baseline": {"value": val, "unit": "shot-gradients/s", "cores": cores,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": val, "unit": "shot-gradients/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, dev):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        self.lines = []
        if self.p:
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()

    def _read(self):
        for ln in self.p.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM traffic of one launch of the dominant stencil kernel measured by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum, the command in
# profiles/stencil2_salt2d_64shots.md) on the default workload: reported only while the
# kernel's source file still has the hash it was taken on.
STENCIL_TRAFFIC = {
    "stencil2.cu": {"sha256_16": "0e3b6acc5fe58a4d", "shots": 64, "npoints": 1681 * 481,
                    "bytes_per_launch": 517291776 + 573171200},
}


def stencil_traffic(src_name, S, N):
    import hashlib
    t = STENCIL_TRAFFIC.get(src_name)
    if t is None:
        return None
    try:
        src = open(os.path.join(ROOT, "paper_2201_06914_gb300", "csrc", src_name), "rb").read()
    except OSError:
        return None
    if hashlib.sha256(src).hexdigest()[:16] != t["sha256_16"] or S != t["shots"] or N != t["npoints"]:
        return None
    return t["bytes_per_launch"]


def run_ours(args):
    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2201_06914_gb300 import wp
    from paper_2201_06914_gb300 import inputs as I

    sv = workload(args, world, rank)
    S, r, Tb, nt = sv.nshots, args.r, args.tb, sv.nt
    N, nrec = sv.npoints, sv.rec.shape[1]
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    m_true = torch.from_numpy(sv.m_padded("true").ravel()).to(dev)
    m0 = torch.from_numpy(sv.m_padded("background").ravel()).to(dev)
    Mt = wp.Model.from_survey(sv, m_true)
    M0 = wp.Model.from_survey(sv, m0)
    # P_u, P_v in the row-aligned layout the contraction accumulates in (no copy into the
    # dense layout; 16-byte vector loads in the offset volume)
    wp.wp_set_probe_layout(M0.handle, wp.WP_PROBES_ALIGNED)
    _, RS, _ = wp.wp_probe_layout(M0.handle)
    geom = wp.Geometry(sv.src, sv.rec)
    wav = torch.from_numpy(sv.wavelet().astype(np.float32)).to(dev)
    ws_bytes = wp.wp_workspace_bytes(M0.handle, geom.c, r, Tb, wp.WP_MODE_PROBED)
    ws = wp.workspace(ws_bytes, dev)
    Pu = torch.empty((S, r, RS), device=dev)
    dsyn = torch.empty((S, nt, nrec), device=dev)
    dobs = torch.empty((S, nt, nrec), device=dev)
    res = torch.empty((S, nt, nrec), device=dev)
    g = torch.empty(N, device=dev)
    misfit = torch.zeros(1, dtype=torch.float64, device=dev)
    rws = wp.workspace(wp.wp_residual_workspace_bytes(S * nt * nrec), dev)

    # Observed data from the true model (plain modelling, untimed).
    wp.wp_probe_forward(Mt.handle, geom.c, wav, None, 0, Tb, None, dobs, ws, stream)
    wp.wp_stream_status(ws, stream, 600.0)

    # Probing matrices (host, once per shot): Rademacher (scale 1/r) or the range finder
    # [Q, ~] = qr(A Z) of Sec. 2.1 (scale 1) with A from the wavelet or the shot's data.
    from paper_2201_06914_gb300 import probes as PR
    base_seed = sv.probe_seed   # the first shot index of this rank
    probe_setup = None
    if args.probes == "rademacher":
        Qh, scale = PR.rademacher(base_seed, S, nt, r)
    else:
        # the range finder on the device (wp_range_finder): Q = orth((D D^T)^p Z), D the
        # wavelet's causal convolution matrix (one for all shots, p = 2) or each shot's
        # observed data (p = 1), Z the shot's Rademacher matrix; estimator scale 1
        import scipy.linalg as sl
        Z = torch.from_numpy(I.rademacher_shots(base_seed, S, nt, r)).to(dev)
        if args.probes == "wavelet":
            D = torch.from_numpy(sl.toeplitz(sv.wavelet(), np.zeros(nt)).astype(np.float32)).to(dev)
            ncols, shared, power = nt, True, 2
        else:
            D, ncols, shared, power = dobs, nrec, False, 1
        Qd = torch.empty((S, nt, r), device=dev)
        rfws = wp.workspace(wp.wp_range_finder_workspace_bytes(nt, ncols, S, shared, r), dev)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        wp.wp_range_finder(D, nt, ncols, S, shared, power, Z, r, Qd, rfws, stream)
        p1.record(stream)
        wp.wp_stream_status(rfws, stream, 600.0)
        probe_setup = {"kind": args.probes, "power": power, "ms": p0.elapsed_time(p1)}
        Qh, scale = Qd.cpu().numpy(), 1.0
        del rfws, Qd, Z, D
    Q = torch.from_numpy(np.ascontiguousarray(Qh)).to(dev)

    def probed_step():
        wp.wp_probe_forward(M0.handle, geom.c, wav, Q, r, Tb, Pu, dsyn, ws, stream)
        wp.wp_residual(dsyn, dobs, res, S * nt * nrec, misfit, rws, stream)
        wp.wp_adjoint_image(M0.handle, geom.c, res, Q, r, Tb, scale, Pu, g, None, ws, stream)

    for _ in range(args.warmup):
        probed_step()
    wp.wp_stream_status(ws, stream, 600.0)
    barrier()
    clocks = Clocks(dev.index)
    l0 = wp.wp_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        probed_step()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = (wp.wp_kernel_launches() - l0)
    ms = e0.elapsed_time(e1) / args.steps
    wp.wp_stream_status(ws, stream, 60.0)
    from paper_2201_06914_gb300.dist import max_over_ranks
    ms = max_over_ranks(ms, dev)
    shots_per_s = world * S / (ms / 1e3)
    gpt = world * S * nt * 2 * N / (ms / 1e3) / 1e9
    g_probed = g.clone()

    # Kernel roofline: event-timed launches of one more step.
    wp.wp_profile_enable(True, 2 * nt + 64)
    probed_step()
    torch.cuda.synchronize(dev)
    st1_ms, st1_n = wp.wp_profile_read(0)
    gm_ms, gm_n = wp.wp_profile_read(1)
    st2_ms, st2_n = wp.wp_profile_read(3)
    wp.wp_profile_enable(False, 0)
    # Algorithmic bytes of one time step: per shot and point read u^n and the increment,
    # write u^{n+1} and the new increment (16 B); dt^2/m is shared by the shots (4 B per
    # point once).  A two-step launch processes two steps, so its algorithmic bytes are
    # twice that; the bytes it must move itself are fewer: it reads u^n and d^n (8 B) and
    # writes the field the probe contraction needs from the first step (d^{n+1} forward,
    # v^j adjoint) and u^{n+2}, d^{n+2} (12 B), plus dt^2/m once.
    two = st2_n > 0 and st2_ms >= st1_ms
    st_ms, st_n = (st2_ms, st2_n) if two else (st1_ms, st1_n)
    steps_per_launch = 2 if two else 1
    st_bytes = steps_per_launch * (16.0 * S + 4.0) * N
    own_bytes = ((20.0 * S + 4.0) if two else (16.0 * S + 4.0)) * N
    st_avg = st_ms / max(st_n, 1) / 1e3
    # Algorithmic bytes of the probe contractions of one step (forward + adjoint): each
    # block reads its Tb (+1 forward) ring rows of every padded point and writes P (r
    # values per point and shot), reading P too except in the first block of a pass.
    nblk = -(-nt // Tb)
    shp = sv.shape_padded
    Np = int(np.prod(shp[:-1])) * (-(-shp[-1] // 4) * 4)   # ring rows use the row pitch NXp
    gm_bytes = 4.0 * S * (Np * (nt + nblk) + Np * nt + 2 * r * N * (2 * nblk - 1))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = st_bytes / st_avg / 1e9
    gm_gbs = gm_bytes / (gm_ms / 1e3) / 1e9 if gm_ms > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak,
                "traffic": stencil_traffic("stencil2.cu" if two else "stencil.cu", S, N),
                "kernel": ("stencil2_kernel<64> (2-D, 256-column tiles, two time steps per launch; "
                           "forward/adjoint)") if two else
                          "stencil_kernel<64,1> (2-D, 256-column tiles; forward/adjoint time step)",
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "algorithmic_bytes_per_launch": st_bytes,
                "algorithmic_unit": "(16 B per point and shot + 4 B per point) per time step",
                "steps_per_launch": steps_per_launch,
                "kernel_min_bytes_per_launch": own_bytes,
                "frac_of_kernel_min_bytes": own_bytes / st_avg / 1e9 / hbm_peak,
                "avg_launch_us": st_avg * 1e6, "launches_timed": st_n,
                "probe_gemm": {"avg_launch_us": gm_ms / max(gm_n, 1) * 1e3, "launches": gm_n,
                               "algorithmic_bytes_per_step": gm_bytes, "achieved_gbs": gm_gbs,
                               "frac": gm_gbs / hbm_peak if gm_gbs else None},
                "single_step_launches": {"launches": st1_n, "avg_launch_us": st1_ms / max(st1_n, 1) * 1e3},
                "stencil_share": (st1_ms + st2_ms) / max(st1_ms + st2_ms + gm_ms, 1e-9)}

    # Subsurface-offset image volume (Eq. 4) of the stacked shots, 2*nh+1 offsets along
    # x, from P_u and a kept P_v: timed on its own (not part of the gradient step).
    offsets = None
    if args.offsets > 0:
        nh = args.offsets
        Pv = torch.empty((S, r, RS), device=dev)
        wp.wp_adjoint_image(M0.handle, geom.c, res, Q, r, Tb, scale, Pu, g, Pv, ws, stream)
        vol = torch.empty((2 * nh + 1, N), device=dev)
        wp.wp_offset_image(M0.handle, Pu, Pv, r, S, scale, nh, vol, stream)
        o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        o0.record(stream)
        for _ in range(3):
            wp.wp_offset_image(M0.handle, Pu, Pv, r, S, scale, nh, vol, stream)
        o1.record(stream)
        torch.cuda.synchronize(dev)
        o_ms = o0.elapsed_time(o1) / 3
        o_bytes = 4.0 * (2 * S * r * N + (2 * nh + 1) * N)   # read P_u, P_v once; write the volume
        offsets = {"nh": nh, "offsets": 2 * nh + 1, "ms": o_ms,
                   "algorithmic_bytes": o_bytes, "achieved_gbs": o_bytes / (o_ms / 1e3) / 1e9,
                   "fma_per_s": S * r * N * (2 * nh + 1) / (o_ms / 1e3),
                   "offset0_equals_image_rel": float(torch.linalg.norm(vol[nh] - g) / torch.linalg.norm(g))}
        del Pv, vol

    # End to end through the C ABI with host buffers: inputs from pinned host memory,
    # the stacked gradient back to the host, every step.
    h_m0 = torch.from_numpy(sv.m_padded("background").ravel()).pin_memory()
    h_dobs = dobs.cpu().pin_memory()
    h_wav = wav.cpu().pin_memory()
    h_Q = torch.from_numpy(Qh).pin_memory()
    h_g = torch.empty(N).pin_memory()
    # Uploads on a second stream, overlapping the previous step's kernels: the model into one
    # of two buffers (the other may still be read by the step before), waited for by the
    # host because wp_model validates it; the observed data (1.6 GB), needed only by the
    # residual, while the forward sweep runs, after the previous residual has read them.
    d_ms = [torch.empty_like(m0), torch.empty_like(m0)]
    side = torch.cuda.Stream(dev)
    m_free = [torch.cuda.Event(), torch.cuda.Event()]
    m_ready, dobs_ready, res_done = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()
    for ev in (*m_free, res_done):
        ev.record(stream)
    nstep = [0]

    def e2e_step():
        i = nstep[0] & 1
        nstep[0] += 1
        d_m = d_ms[i]
        with torch.cuda.stream(side):
            side.wait_event(m_free[i])
            d_m.copy_(h_m0, non_blocking=True)
            m_ready.record(side)
            side.wait_event(res_done)
            dobs.copy_(h_dobs, non_blocking=True)
            dobs_ready.record(side)
        wav.copy_(h_wav, non_blocking=True)
        Q.copy_(h_Q, non_blocking=True)
        m_ready.synchronize()   # the model must be on the device before wp_model validates it
        Me = wp.Model.from_survey(sv, d_m)
        wp.wp_set_probe_layout(Me.handle, wp.WP_PROBES_ALIGNED)
        wp.wp_probe_forward(Me.handle, geom.c, wav, Q, r, Tb, Pu, dsyn, ws, stream)
        stream.wait_event(dobs_ready)
        wp.wp_residual(dsyn, dobs, res, S * nt * nrec, misfit, rws, stream)
        res_done.record(stream)
        wp.wp_adjoint_image(Me.handle, geom.c, res, Q, r, Tb, scale, Pu, g, None, ws, stream)
        h_g.copy_(g, non_blocking=True)
        m_free[i].record(stream)
        Me.close()

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.steps
    h2d = (h_m0.numel() + h_dobs.numel() + h_wav.numel() + h_Q.numel()) * 4
    e2e = {"value": world * S / e2e_s, "unit": "shot-gradients/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": N * 4, "ms_per_step": e2e_s * 1e3}

    hbm_probed = (wp.wp_workspace_bytes(M0.handle, wp.Geometry(sv.src[:1], sv.rec[:1]).c, r,
                                        Tb, wp.WP_MODE_PROBED) + r * RS * 4) / 1e9
    g1 = wp.Geometry(sv.src[:1], sv.rec[:1])
    hbm_exact = wp.wp_workspace_bytes(M0.handle, g1.c, 0, 1, wp.WP_MODE_EXACT_FULL) / 1e9

    # Exact full-history gradient on the same shots (batched to fit HBM).
    exact = None
    rel_err = None
    if not args.no_exact:
        del ws, Pu, dsyn, res
        torch.cuda.empty_cache()
        free, _ = torch.cuda.mem_get_info(dev)
        bs = S
        while bs > 1:
            gb = wp.Geometry(sv.src[:bs], sv.rec[:bs])
            if wp.wp_workspace_bytes(M0.handle, gb.c, 0, 1, wp.WP_MODE_EXACT_FULL) < 0.85 * free:
                break
            bs = (bs + 1) // 2
        batches = [(s, min(S, s + bs)) for s in range(0, S, bs)]
        geoms = [wp.Geometry(sv.src[a:b], sv.rec[a:b]) for a, b in batches]
        wse = wp.workspace(wp.wp_workspace_bytes(M0.handle, geoms[0].c, 0, 1,
                                                 wp.WP_MODE_EXACT_FULL), dev)
        gb_out = torch.empty(N, device=dev)
        g_exact = torch.zeros(N, device=dev)
        Je = torch.zeros(1, dtype=torch.float64, device=dev)

        def exact_step(acc):
            for (a, b), gg in zip(batches, geoms):
                wp.wp_exact_gradient(M0.handle, gg.c, wav, dobs[a:b], gb_out, Je, None,
                                     wp.WP_MODE_EXACT_FULL, 1, wse, stream)
                if acc is not None:
                    acc += gb_out
        exact_step(g_exact)  # warm-up and reference gradient
        wp.wp_stream_status(wse, stream, 600.0)
        barrier()
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        x0.record(stream)
        exact_step(None)
        x1.record(stream)
        barrier()
        ex_ms = x0.elapsed_time(x1)
        ex_val = world * S / (ex_ms / 1e3)
        exact = {"value": ex_val, "unit": "shot-gradients/s", "mode": "full history",
                 "batch_shots": bs, "ms_per_step": ex_ms,
                 "gpt_updates_per_s": world * S * nt * 2 * N / (ex_ms / 1e3) / 1e9}
        rel_err = float(torch.linalg.vector_norm((g_probed - g_exact).double()) /
                        torch.linalg.vector_norm(g_exact.double()))
        # Exact-path kernels, event-timed over one more exact step: the adjoint stencil with
        # the imaging condition of Eq. 2 fused (two steps per launch on this 2-D grid, a
        # single step where a pair does not fit) and the forward pairs.  The imaging adjoint
        # moves, per point, shot and step, u/d in and out (16 B), two history rows (8 B) and
        # the image read-modify-write (8 B), plus dt^2/m once.
        wp.wp_profile_enable(True, 2 * nt * len(batches) + 64)
        exact_step(None)
        torch.cuda.synchronize(dev)
        img1_ms, img1_n = wp.wp_profile_read(0)
        fwd_ms, fwd_n = wp.wp_profile_read(3)
        img2_ms, img2_n = wp.wp_profile_read(4)
        wp.wp_profile_enable(False, 0)
        pair_img = img2_n > 0
        img_ms, img_n = (img2_ms, img2_n) if pair_img else (img1_ms, img1_n)
        img_steps = 2 if pair_img else 1
        img_avg = img_ms / max(img_n, 1) / 1e3
        img_bytes = img_steps * (32.0 * bs + 4.0) * N
        fwd_avg = fwd_ms / max(fwd_n, 1) / 1e3
        fwd_bytes = 2 * (16.0 * bs + 4.0) * N
        exact["roofline"] = {
            "kernel": ("stencil2_kernel<64,IMG> (exact adjoint, two steps per launch with g += u_tt v of both fused)"
                       if pair_img else "stencil_kernel<64,1,IMG> (exact adjoint step with g += u_tt v fused)"),
            "bound": "hbm", "avg_launch_us": img_avg * 1e6, "launches": img_n, "steps_per_launch": img_steps,
            "single_step_launches": img1_n if pair_img else 0,
            "algorithmic_bytes_per_launch": img_bytes,
            "algorithmic_unit": "32 B per point and shot + 4 B per point (dt^2/m) per step",
            "achieved": img_bytes / img_avg / 1e9 if img_n else None, "peak": hbm_peak,
            "frac": (img_bytes / img_avg / 1e9 / hbm_peak) if img_n else None,
            "forward_pairs": {"kernel": "stencil2_kernel<64> (history-writing forward, two steps)",
                              "avg_launch_us": fwd_avg * 1e6, "launches": fwd_n,
                              "algorithmic_bytes_per_launch": fwd_bytes,
                              "frac": (fwd_bytes / fwd_avg / 1e9 / hbm_peak) if fwd_n else None}}
        del wse

    # The metric's operating point: the smallest r whose stacked gradient is within 0.1 of
    # the exact gradient (Eq. 1: the error falls as r^-1/2, so r is predicted from the error
    # at the default r and then checked), timed on the same shots in batches that fit HBM.
    op = None
    if exact is not None and not args.no_op and rel_err is not None:
        exact["hbm_per_shot_gb"] = hbm_exact
        op = operating_point(args, sv, M0, geom, wav, dobs, g_exact, exact, r, rel_err, dev, stream)

    salt3d = None
    if not args.no_3d and world == 1:
        del g_exact
        torch.cuda.empty_cache()
        a3 = argparse.Namespace(**vars(args))
        a3.steps, a3.warmup = 1, 1
        salt3d = measure_volume(a3, "salt3d")
        salt3d = {k: salt3d.get(k) for k in ("value", "unit", "ms_per_step", "config", "gpt_updates_per_s",
                                                "hbm_probed_gb", "exact", "speedup_vs_exact", "operating_point",
                                                "roofline", "clocks")}

    # The 3-D pseudo-acoustic TTI workload (400 x 400 x 300 at 12.5 m, 3000 steps, r = 32),
    # probed against the checkpointed exact gradient, one shot.
    tti3d = None
    if not args.no_3d and not args.no_tti and world == 1:
        torch.cuda.empty_cache()
        a4 = argparse.Namespace(**vars(args))
        a4.steps, a4.warmup = 1, 1
        a4.nx3, a4.ny3, a4.nz3, a4.nt3, a4.r3 = 400, 400, 300, 3000, 32
        tti3d = measure_volume(a4, "tti3d")
        tti3d = {k: tti3d.get(k) for k in ("value", "unit", "ms_per_step", "config", "gpt_updates_per_s",
                                              "hbm_probed_gb", "exact", "speedup_vs_exact", "roofline", "clocks")}

    # Serving, driver-observed: a shortened run of the serving mix (Poisson arrivals at
    # 1.2 jobs/s, 2-D and 3-D, isotropic and TTI) with its p50/p99 latency.
    serving = None
    if not args.no_serving and world == 1:
        torch.cuda.empty_cache()
        a5 = argparse.Namespace(**vars(args))
        a5.jobs, a5.rate = args.serving_jobs, 0.0
        sl = measure_serving(a5)
        serving = {k: sl.get(k) for k in ("value", "unit", "latency_p50_s", "latency_p99_s",
                                            "latency_by_kind", "jobs_ok", "config",
                                            "gpt_updates_per_s", "peak_admitted_bytes", "clocks")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        _, per_shot, desc, cores = oracle_sample(sv, r, args.cpu_steps)
        cpu = {"value": 1.0 / per_shot, "unit": "shot-gradients/s", "cores": cores,
               "kind": "oracle", "sample": desc,
               "two_layer_full": oracle_two_layer()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": shots_per_s, "unit": "shot-gradients/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 stencil, bf16 hi/lo split probe contraction with f32 accumulation",
            "data": "synthetic",
            "config": {"workload": f"salt_2d_{sv.nx}x{sv.nz}_pad{sv.nbl}_nt{nt}_shots{S}_r{r}",
                       "grid_padded": [sv.shape_padded[1], sv.shape_padded[0]], "nt": nt,
                       "shots_per_gpu": S, "r": r, "Tb": Tb, "probes": args.probes,
                       "probe_setup": probe_setup,
                       "parallelism": f"shots sharded, {world} GPU(s), no collective",
                       "l2": "per-step working set (~50 GB) far exceeds L2; no flush needed"},
            "gpt_updates_per_s": gpt,
            "exact": exact,
            "offset_image": offsets,
            "speedup_vs_exact": (shots_per_s / exact["value"]) if exact else None,
            "rel_err_vs_exact": rel_err,
            "operating_point": op,
            "salt3d_checkpointed": salt3d,
            "tti3d_checkpointed": tti3d,
            "serving": serving,
            "hbm_per_shot_gb": {"probed": hbm_probed, "exact_full_history": hbm_exact},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def operating_point(args, sv, M0, geom, wav, dobs, g_exact, exact, r0, err0, dev, stream):
    """Probed gradient at the smallest r (a multiple of 16, at most 512) whose stacked error
    against the exact gradient is <= 0.1: the first guess scales r0 by (err0 / 0.1)^2 (the
    estimator's r^-1/2 law), later guesses by the measured error.  At that r the probe
    blocks are also timed at Tb = 512 (half the P traffic per step, in more shot batches if
    memory requires) and the faster block length is reported.  Returns the timing, the
    error, the HBM per shot and the speed-up over the exact path at that r."""
    import torch
    from paper_2201_06914_gb300 import inputs as I
    from paper_2201_06914_gb300 import wp
    S, nt, N, nrec = sv.nshots, sv.nt, sv.npoints, sv.rec.shape[1]
    _, RS, _ = wp.wp_probe_layout(M0.handle)   # floats per probe row of P_u

    def trial(r_op, Tb):
        free, _ = torch.cuda.mem_get_info(dev)
        bs = S
        while bs > 1:
            gb = wp.Geometry(sv.src[:bs], sv.rec[:bs])
            need = wp.wp_workspace_bytes(M0.handle, gb.c, r_op, Tb, wp.WP_MODE_PROBED) + \
                bs * (r_op * RS + 2 * nt * nrec) * 4
            if need < 0.85 * free:
                break
            bs = (bs + 1) // 2
        batches = [(a, min(S, a + bs)) for a in range(0, S, bs)]
        geoms = [wp.Geometry(sv.src[a:b], sv.rec[a:b]) for a, b in batches]
        ws = wp.workspace(wp.wp_workspace_bytes(M0.handle, geoms[0].c, r_op, Tb, wp.WP_MODE_PROBED), dev)
        Q = torch.from_numpy(I.rademacher_shots(sv.probe_seed, S, nt, r_op)).to(dev)
        Pu = torch.empty((bs, r_op, RS), device=dev)
        dsyn = torch.empty((bs, nt, nrec), device=dev)
        res = torch.empty((bs, nt, nrec), device=dev)
        gb_out = torch.empty(N, device=dev)
        g = torch.zeros(N, device=dev)

        def step(acc):
            for (a, b), gg in zip(batches, geoms):
                n = b - a
                wp.wp_probe_forward(M0.handle, gg.c, wav, Q[a:b], r_op, Tb, Pu[:n], dsyn[:n], ws, stream)
                wp.wp_residual(dsyn[:n], dobs[a:b], res[:n], n * nt * nrec, None, None, stream)
                wp.wp_adjoint_image(M0.handle, gg.c, res[:n], Q[a:b], r_op, Tb, 1.0 / r_op, Pu[:n],
                                    gb_out, None, ws, stream)
                if acc is not None:
                    acc += gb_out
        step(g)
        wp.wp_stream_status(ws, stream, 600.0)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(None)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        err = float(torch.linalg.vector_norm((g - g_exact).double()) / torch.linalg.vector_norm(g_exact.double()))
        g1 = wp.Geometry(sv.src[:1], sv.rec[:1])
        hbm = (wp.wp_workspace_bytes(M0.handle, g1.c, r_op, Tb, wp.WP_MODE_PROBED) + r_op * RS * 4) / 1e9
        del ws, Q, Pu, dsyn, res, gb_out, g
        torch.cuda.empty_cache()
        return {"r": r_op, "tb": Tb, "rel_err_vs_exact": err, "value": S / (ms / 1e3), "ms_per_step": ms,
                "batch_shots": bs, "hbm_per_shot_gb": hbm}

    tried = []
    r_op = r0 if err0 <= 0.1 else min(512, -(-int(np.ceil(r0 * (err0 / 0.1) ** 2)) // 16) * 16)
    for _ in range(3):
        tried.append(trial(r_op, args.tb))
        err = tried[-1]["rel_err_vs_exact"]
        if err <= 0.1 or r_op >= 512:
            break
        r_op = min(512, -(-int(np.ceil(r_op * (err / 0.1) ** 2)) // 16) * 16 + 16)
    best = tried[-1]
    if best["rel_err_vs_exact"] <= 0.1 and args.tb < 512 and nt >= 1024:
        t = trial(best["r"], 512)
        tried.append(t)
        if t["rel_err_vs_exact"] <= 0.1 and t["value"] > best["value"]:
            best = t
    return {"r": best["r"], "tb": best["tb"], "value": best["value"], "unit": "shot-gradients/s",
            "rel_err_vs_exact": best["rel_err_vs_exact"], "meets_0.1": best["rel_err_vs_exact"] <= 0.1,
            "batch_shots": best["batch_shots"], "hbm_per_shot_gb": best["hbm_per_shot_gb"],
            "hbm_per_shot_exact_gb": None if exact is None else exact.get("hbm_per_shot_gb"),
            "speedup_vs_exact": best["value"] / exact["value"], "tried": tried,
            "note": "same shots, Rademacher probes; Tb the headline's or 512, whichever is faster; "
                    "error against the exact full-history gradient of the stack"}


def _serving_jobs(args, rng):
    """The serving mix: 2-D salt grids 401x401 .. 1601x401 (12.5 m) and 3-D layered + salt
    grids 128^3 .. 256^3 (10 m isotropic, 12.5 m TTI, 20-cell sponge, receiver carpet every
    4 cells), isotropic acoustic or pseudo-acoustic TTI (eps <= 0.25), 1000-4000 steps,
    r in {8, 16, 32}, Poisson arrivals.  Models and Thomsen fields are built once per
    dimension and equation (3-D ones are crops of one 256^3 model) and shared by the jobs."""
    from paper_2201_06914_gb300 import inputs as I
    from paper_2201_06914_gb300.serve import ShotJob
    kinds = [("2d", (401, 1, 401)), ("2d", (801, 1, 401)), ("2d", (1601, 1, 401)),
             ("3d", (128, 128, 128)), ("3d", (192, 192, 192)), ("3d", (256, 256, 256))]
    cache = {}

    def survey(dim, tti):
        key = (dim, tti)
        if key not in cache:
            if dim == "2d":
                sv = I.config_salt_2d(nx=1601, nz=401, nt=1000, r=8, nshots=1)
                if tti:   # the anisotropic operator is faster by sqrt(1 + 2 eps_max)
                    sv.dt /= np.sqrt(1.5)
            else:
                sv = I.config_salt_3d(nx=256, ny=256, nz=256, nt=1000, nbl=20, r=8, nshots=1,
                                      rec_stride=4, dx=12.5 if tti else 10.0,
                                      eps_max=0.25 if tti else 0.0)
            th = I.tti_fields(sv.v_true.shape, sv.spacing) if tti else None
            cache[key] = (sv, th)
        return cache[key]

    crops = {}

    def crop(dim, size, tti):
        key = (dim, size, tti)
        if key not in crops:
            sv, th = survey(dim, tti)
            nx, ny, nz = size
            sl = (slice(0, nz), slice(0, nx)) if dim == "2d" else (slice(0, nz), slice(0, ny), slice(0, nx))
            m0 = I.pad_edge(I.slowness_squared(sv.v_background[sl]), sv.nbl).astype(np.float32)
            thp = None
            if th is not None:
                thp = tuple(I.pad_edge(f[sl], sv.nbl).astype(np.float32) for f in th)
            if dim == "2d":
                x = np.arange(nx) * sv.spacing
                rec = np.stack([x, np.zeros(nx), np.full(nx, 12.5)], axis=1)[None]
            else:
                gx, gy = np.meshgrid(np.arange(0, nx, 4) * sv.spacing, np.arange(0, ny, 4) * sv.spacing)
                rec = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 20.0)], axis=1)[None]
            crops[key] = (sv, m0, thp, rec, float(sv.v_true.max()))
        return crops[key]

    zeros = {}
    jobs, t = [], 0.0
    rate = args.rate if args.rate > 0 else 1.2
    for k in range(args.jobs):
        dim, size = kinds[rng.integers(len(kinds))]
        tti = bool(rng.integers(2))
        nt = int(rng.choice([1000, 2000, 4000]))
        r = int(rng.choice([8, 16, 32]))
        sv, m0, thp, rec, vmax = crop(dim, size, tti)
        nx, ny, nz = size
        h = sv.spacing
        src = np.array([[rng.uniform(0.1, 0.9) * (nx - 1) * h,
                         (rng.uniform(0.1, 0.9) * (ny - 1) * h) if dim == "3d" else 0.0,
                         20.0 if dim == "3d" else 12.5]])
        zk = (nt, rec.shape[1])
        if zk not in zeros:   # imaging the direct arrivals
            zeros[zk] = np.zeros((1, nt, rec.shape[1]), np.float32)
        jobs.append(ShotJob(f"job{k}", 2 if dim == "2d" else 3, nx, ny, nz, sv.nbl, h, sv.dt, nt, m0,
                            src[:, None, :], rec, I.ricker(nt, sv.dt, sv.f0), zeros[zk],
                            I.rademacher_shots(k, 1, nt, r), 64, t, thomsen=thp, damp_v=vmax))
        t += rng.exponential(1.0 / rate)
    return jobs, rate


def run_serving(args):
    rank, world, local = dist_info()
    if rank != 0:
        return 0
    print(json.dumps(measure_serving(args)), flush=True)
    return 0


def measure_serving(args):
    """Serving workload: Poisson-arriving shot-gradient jobs mixing 2-D and 3-D grids,
    isotropic and TTI equations, 1000-4000 steps and r in {8, 16, 32} under continuous
    batching (admission by device footprint, one stream per job).  Latency runs from
    arrival to the gradient on the host."""
    import torch
    from paper_2201_06914_gb300.serve import GpuBackend, Scheduler
    t_build = time.perf_counter()
    jobs, rate = _serving_jobs(args, np.random.default_rng(7))
    t_build = time.perf_counter() - t_build
    backend = GpuBackend()
    for j in jobs:
        backend.footprint(j)
    warm = sorted(jobs, key=lambda j: np.prod(j.m.shape))[:2]
    Scheduler(backend, 200e9, max_active=8).run([dataclasses.replace(j, name="w" + j.name, arrival=0.0)
                                                 for j in warm])
    torch.cuda.synchronize()
    clocks = Clocks(0)
    sched = Scheduler(backend, mem_budget=200e9, max_active=8)
    t0 = time.perf_counter()
    res = sched.run(jobs)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    st = Scheduler.stats(res, wall)
    by = {}
    for j in jobs:
        k = f"{j.ndim}d_{'tti' if j.thomsen is not None else 'iso'}"
        if res[j.name].ok:
            by.setdefault(k, []).append(res[j.name].latency)
    mix = {k: {"jobs": len(v), "p50_s": float(np.percentile(v, 50)), "p99_s": float(np.percentile(v, 99))}
           for k, v in sorted(by.items())}
    pts = sum(2 * j.nt * j.fields * int(np.prod(j.m.shape)) for j in jobs if res[j.name].ok)
    line = {"metric": METRIC + " (serving)", "value": st.get("jobs_per_s"), "unit": "jobs/s",
            "n_gpus": 1, "steps": len(jobs), "warmup": 2, "ms_per_step": wall * 1e3 / len(jobs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 stencil, bf16 hi/lo split probe contraction with f32 accumulation",
            "data": "synthetic",
            "config": {"workload": "serving: Poisson arrivals, 2-D salt grids 401x401..1601x401 and "
                                   "3-D layered+salt grids 128^3..256^3, isotropic and TTI, "
                                   "1000-4000 steps, r in {8,16,32}, probed gradients",
                       "jobs": len(jobs), "arrival_rate_per_s": rate, "max_active": 8,
                       "mem_budget_bytes": 200e9},
            "latency_p50_s": st.get("p50_s"), "latency_p99_s": st.get("p99_s"),
            "latency_by_kind": mix, "jobs_ok": st["ok"], "peak_admitted_bytes": sched.peak_used,
            "gpt_updates_per_s": pts / wall / 1e9, "host_setup_s": t_build, "clocks": clk}
    return line


def run_volume(args):
    print(json.dumps(measure_volume(args, args.workload)), flush=True)
    return 0


def measure_volume(args, workload):
    """3-D workloads on one GPU, one shot (the paper's 3-D configurations): the isotropic
    layered + salt model (512 x 512 x 256 at 10 m, r = 32) or the pseudo-acoustic TTI model
    (400 x 400 x 300 at 12.5 m, r = 32).  Times the probed gradient and, unless --no-exact,
    the exact gradient with two-level checkpointing (the full history would not fit), and
    reports the stencil roofline from CUDA events on the launching stream."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    from paper_2201_06914_gb300 import inputs as I
    from paper_2201_06914_gb300 import wp
    tti = workload == "tti3d"
    nx, ny, nz = (args.nx3, args.ny3, args.nz3)
    if tti:   # config: 12.5 m, eps up to 0.25 (the CFL step shrinks by sqrt(1.5))
        sv = I.config_salt_3d(nx=nx, ny=ny, nz=nz, nt=args.nt3, r=args.r3, nshots=1, dx=12.5,
                              f0=12.0, eps_max=0.25)
    else:
        sv = I.config_salt_3d(nx=nx, ny=ny, nz=nz, nt=args.nt3, r=args.r3, nshots=1)
    S, r, Tb, nt = 1, args.r3, args.tb3, sv.nt
    N, nrec = sv.npoints, sv.rec.shape[1]
    stream = torch.cuda.current_stream(dev)
    th = None
    if tti:
        fields = I.tti_fields((nz, ny, nx), sv.spacing)
        th = [torch.from_numpy(I.pad_edge(f, sv.nbl).astype(np.float32).ravel()).to(dev) for f in fields]

    def model(which):
        m = torch.from_numpy(sv.m_padded(which).ravel()).to(dev)
        kw = dict(eps=th[0], delta=th[1], theta=th[2], phi=th[3]) if tti else {}
        return wp.Model(3, nx, ny, nz, sv.nbl, sv.spacing, sv.spacing, sv.spacing, sv.dt, nt, m,
                        sv.damp_v, **kw)
    Mt, M0 = model("true"), model("background")
    wp.wp_set_probe_layout(M0.handle, wp.WP_PROBES_ALIGNED)   # no copy of P into the dense layout
    _, RS, _ = wp.wp_probe_layout(M0.handle)
    geom = wp.Geometry(sv.src, sv.rec)
    wav = torch.from_numpy(sv.wavelet().astype(np.float32)).to(dev)
    Q = torch.from_numpy(I.rademacher_shots(0, S, nt, r)).to(dev)
    F = 2 if tti else 1                                   # fields per shot
    ws = wp.workspace(wp.wp_workspace_bytes(M0.handle, geom.c, r, Tb, wp.WP_MODE_PROBED), dev)
    Pu = torch.empty((S * F, r, RS), device=dev)
    dsyn = torch.empty((S, nt, nrec), device=dev)
    dobs = torch.empty((S, nt, nrec), device=dev)
    res = torch.empty_like(dobs)
    g = torch.empty(N, device=dev)
    J = torch.zeros(1, dtype=torch.float64, device=dev)
    rws = wp.workspace(wp.wp_residual_workspace_bytes(S * nt * nrec), dev)
    wp.wp_probe_forward(Mt.handle, geom.c, wav, None, 0, Tb, None, dobs, ws, stream)

    def probed_step():
        wp.wp_probe_forward(M0.handle, geom.c, wav, Q, r, Tb, Pu, dsyn, ws, stream)
        wp.wp_residual(dsyn, dobs, res, S * nt * nrec, J, rws, stream)
        wp.wp_adjoint_image(M0.handle, geom.c, res, Q, r, Tb, 1.0 / r, Pu, g, None, ws, stream)

    for _ in range(max(1, args.warmup)):
        probed_step()
    wp.wp_stream_status(ws, stream, 600.0)
    torch.cuda.synchronize(dev)
    clocks = Clocks(0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        probed_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    wp.wp_profile_enable(True, 2 * nt + 64)
    probed_step()
    torch.cuda.synchronize(dev)
    st_ms, st_n = wp.wp_profile_read(0)
    gm_ms, gm_n = wp.wp_profile_read(1)
    wp.wp_profile_enable(False, 0)
    g_probed = g.clone()
    del Pu, ws
    torch.cuda.empty_cache()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    # algorithmic bytes of one time step: iso 16 B per point and shot + 4 B (dt^2/m);
    # TTI: pass 1 reads both fields and writes D_r of both (16 B), pass 2 reads D_r, both
    # fields and both increments and writes both fields and increments (40 B), plus the six
    # parameter fields E, sqrt(1+2 delta), a_x, a_y, a_z, dt^2/m (24 B)
    st_bytes = ((56.0 * S + 24.0) if tti else (16.0 * S + 4.0)) * N
    st_avg = st_ms / max(st_n, 1) / 1e3
    achieved = st_bytes / st_avg / 1e9
    exact = None
    if not args.no_exact:
        nck = args.ncheck3
        wse = wp.workspace(wp.wp_workspace_bytes(M0.handle, geom.c, 0, nck, wp.WP_MODE_EXACT_CHECKPOINT), dev)
        ge = torch.empty(N, device=dev)
        wp.wp_exact_gradient(M0.handle, geom.c, wav, dobs, ge, None, None, wp.WP_MODE_EXACT_CHECKPOINT, nck, wse, stream)
        torch.cuda.synchronize(dev)
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        x0.record(stream)
        wp.wp_exact_gradient(M0.handle, geom.c, wav, dobs, ge, None, None, wp.WP_MODE_EXACT_CHECKPOINT, nck, wse, stream)
        x1.record(stream)
        torch.cuda.synchronize(dev)
        ems = x0.elapsed_time(x1)
        exact = {"value": S / (ems / 1e3), "unit": "shot-gradients/s", "mode": f"checkpoint every {nck} steps",
                 "ms_per_step": ems, "hbm_gb": wse.numel() / 1e9,
                 "full_history_gb": 4.0 * F * N * (nt + 1) / 1e9}
        exact["rel_err_probed"] = float(torch.linalg.norm(g_probed - ge) / torch.linalg.norm(ge))
        del wse
    op = None
    if exact is not None and not tti and not args.no_op:
        torch.cuda.empty_cache()
        try:
            op = volume_operating_point(args, sv, M0, geom, wav, dobs, dsyn, res, ge, exact, r,
                                        exact["rel_err_probed"], RS, dev, stream)
        except (RuntimeError, wp.WpError) as e:   # e.g. memory taken by the caller's buffers
            op = {"meets_0.1": False, "note": f"search stopped: {str(e).splitlines()[0][:200]}"}
        torch.cuda.empty_cache()
    line = {"metric": METRIC + (" (3-D TTI)" if tti else " (3-D)"), "value": S / (ms / 1e3),
            "unit": "shot-gradients/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 stencil, bf16 hi/lo split probe contraction with f32 accumulation",
            "data": "synthetic",
            "config": {"workload": f"{workload}_{nx}x{ny}x{nz}_pad{sv.nbl}_nt{nt}_r{r}_Tb{Tb}",
                       "grid_padded": list(sv.shape_padded), "shots": S},
            "gpt_updates_per_s": S * F * nt * 2 * N / (ms / 1e3) / 1e9,
            "hbm_probed_gb": 4.0 * F * N * (r * 2 + Tb + 4) / 1e9,
            "exact": exact, "speedup_vs_exact": (exact["ms_per_step"] / ms) if exact else None,
            "operating_point": op,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "algorithmic_bytes_per_step": st_bytes,
                         "kernel": "tti pass1+pass2+injection" if tti else "stencil_kernel<16,8> (3-D)",
                         "avg_step_us": st_avg * 1e6, "steps_timed": st_n,
                         "probe_gemm_avg_us": gm_ms / max(gm_n, 1) * 1e3,
                         "stencil_share": st_ms / max(st_ms + gm_ms, 1e-9)},
            "clocks": clk, "gpu_launches": None}
    return line


def volume_operating_point(args, sv, M0, geom, wav, dobs, dsyn, res, g_exact, exact, r0, err0,
                           RS, dev, stream):
    """The 3-D isotropic workload's probed gradient at the smallest r (a multiple of 16)
    whose error against the checkpointed exact gradient is <= 0.1, predicted from the error
    at r0 by the estimator's r^-1/2 law and then checked; timed at the workload's Tb and at
    twice it where that fits, the faster reported.  P_u and P_v grow as 8 r B per point, so
    r is bounded by the device memory: a guess that does not fit ends the search."""
    import torch
    from paper_2201_06914_gb300 import inputs as I
    from paper_2201_06914_gb300 import wp
    S, nt, N, nrec = 1, sv.nt, sv.npoints, sv.rec.shape[1]

    def need_bytes(r_op, Tb):
        return wp.wp_workspace_bytes(M0.handle, geom.c, r_op, Tb, wp.WP_MODE_PROBED) + 4 * S * r_op * RS

    def trial(r_op, Tb):
        ws = wp.workspace(wp.wp_workspace_bytes(M0.handle, geom.c, r_op, Tb, wp.WP_MODE_PROBED), dev)
        Q = torch.from_numpy(I.rademacher_shots(0, S, nt, r_op)).to(dev)
        Pu = torch.empty((S, r_op, RS), device=dev)
        g = torch.empty(N, device=dev)

        def step():
            wp.wp_probe_forward(M0.handle, geom.c, wav, Q, r_op, Tb, Pu, dsyn, ws, stream)
            wp.wp_residual(dsyn, dobs, res, S * nt * nrec, None, None, stream)
            wp.wp_adjoint_image(M0.handle, geom.c, res, Q, r_op, Tb, 1.0 / r_op, Pu, g, None, ws, stream)
        step()
        wp.wp_stream_status(ws, stream, 600.0)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        err = float(torch.linalg.vector_norm((g - g_exact).double()) / torch.linalg.vector_norm(g_exact.double()))
        out = {"r": r_op, "tb": Tb, "rel_err_vs_exact": err, "value": S / (ms / 1e3), "ms_per_step": ms,
               "hbm_per_shot_gb": need_bytes(r_op, Tb) / 1e9}
        del ws, Q, Pu, g
        torch.cuda.empty_cache()
        return out

    def fits(r_op, Tb):
        free, _ = torch.cuda.mem_get_info(dev)
        return need_bytes(r_op, Tb) < 0.9 * free

    Tb = args.tb3
    tried, note = [], None
    r_op = r0 if err0 <= 0.1 else min(512, -(-int(np.ceil(r0 * (err0 / 0.1) ** 2)) // 16) * 16)
    for _ in range(3):
        if not fits(r_op, Tb):
            note = f"r = {r_op} does not fit in device memory at Tb = {Tb}"
            break
        tried.append(trial(r_op, Tb))
        err = tried[-1]["rel_err_vs_exact"]
        if err <= 0.1 or r_op >= 512:
            break
        r_op = min(512, -(-int(np.ceil(r_op * (err / 0.1) ** 2)) // 16) * 16 + 16)
    ok = [t for t in tried if t["rel_err_vs_exact"] <= 0.1]
    if not ok:
        return {"meets_0.1": False, "tried": tried, "note": note}
    best = ok[-1]
    if fits(best["r"], 2 * Tb):
        t = trial(best["r"], 2 * Tb)
        tried.append(t)
        if t["rel_err_vs_exact"] <= 0.1 and t["value"] > best["value"]:
            best = t
    return {"r": best["r"], "tb": best["tb"], "value": best["value"], "unit": "shot-gradients/s",
            "rel_err_vs_exact": best["rel_err_vs_exact"], "meets_0.1": True,
            "hbm_per_shot_gb": best["hbm_per_shot_gb"], "hbm_exact_checkpointed_gb": exact["hbm_gb"],
            "speedup_vs_exact": best["value"] / exact["value"], "tried": tried,
            "note": "one shot, Rademacher probes; error against the checkpointed exact gradient"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload in ("salt3d", "tti3d"):
        return run_volume(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
