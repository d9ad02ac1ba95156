"""Continuous batching of shot-gradient jobs on one GPU.

Jobs (one probed gradient each: forward with probing, residual, adjoint with the
randomized imaging condition, Eq. 3) arrive over time with different grids (2-D or 3-D),
equations (isotropic acoustic or pseudo-acoustic TTI), step counts and probe counts.  The scheduler admits a job as soon as an execution slot is free and
its device footprint (the workspace of the method plus inputs and outputs, i.e. the
quantity the method shrinks) fits in the memory budget; each admitted job gets its own
CUDA stream, so the work of admitted jobs overlaps on the device while later jobs keep
arriving.  Completion is detected by polling CUDA events from the host with a deadline
(no device-side waits).  Latency is measured from arrival to completion.

The scheduler (`Scheduler`) is plain host logic over a backend interface, so it is tested
on the CPU with a fake backend; `GpuBackend` runs the jobs through libwp.so.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque
from typing import Any, Callable

import numpy as np


@dataclasses.dataclass
class ShotJob:
    """One shot-gradient request."""
    name: str
    ndim: int
    nx: int
    ny: int
    nz: int
    nbl: int
    h: float
    dt: float
    nt: int
    m: np.ndarray             # padded squared slowness (float32)
    src: np.ndarray           # (1, nsrc, 3) metres
    rec: np.ndarray           # (1, nrec, 3)
    wavelet: np.ndarray       # (nt,)
    d_obs: np.ndarray         # (1, nt, nrec)
    Q: np.ndarray             # (1, nt, r) probing matrix
    Tb: int = 64
    arrival: float = 0.0      # seconds after the start of the run
    deadline: float = 600.0   # seconds allowed on the device
    thomsen: tuple | None = None   # (eps, delta, theta, phi) padded float32: pseudo-acoustic TTI
    damp_v: float = 0.0       # sponge velocity (0: the model's maximum)

    @property
    def fields(self) -> int:
        return 2 if self.thomsen is not None else 1


@dataclasses.dataclass
class JobResult:
    name: str
    ok: bool
    error: str = ""
    g: Any = None
    arrival: float = 0.0
    admitted: float = 0.0
    finished: float = 0.0

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Scheduler:
    """Admission by footprint, bounded concurrency, FIFO with first-fit bypass."""

    def __init__(self, backend, mem_budget: float, max_active: int = 8,
                 clock: Callable[[], float] = time.perf_counter, bypass: int = 4):
        self.backend = backend
        self.mem_budget = float(mem_budget)
        self.max_active = int(max_active)
        self.clock = clock
        self.bypass = bypass
        self.used = 0.0
        self.peak_used = 0.0
        self.pending: deque = deque()
        self.active: list = []
        self.results: dict[str, JobResult] = {}
        self.cancelled: set = set()
        self.zombies: list = []   # (handle, need): timed-out jobs still running on the device

    def cancel(self, name: str):
        """Cancel a job: a pending job is dropped; an active job's work finishes on the
        device (kernels are never interrupted) and its result is discarded."""
        self.cancelled.add(name)
        for j in list(self.pending):
            if j.name == name:
                self.pending.remove(j)
                self.results[name] = JobResult(name, False, "cancelled", arrival=j.arrival)

    def _admit(self, now, t0):
        progressed = True
        while progressed and self.pending and len(self.active) < self.max_active:
            progressed = False
            for k, job in enumerate(list(self.pending)[: self.bypass + 1]):
                need = self.backend.footprint(job)
                if need > self.mem_budget:
                    self.pending.remove(job)
                    self.results[job.name] = JobResult(job.name, False, "footprint exceeds the budget",
                                                       arrival=job.arrival)
                    progressed = True
                    break
                if self.used + need <= self.mem_budget:
                    self.pending.remove(job)
                    try:
                        handle = self.backend.start(job)
                    except Exception as e:  # allocation or launch failure: job fails alone
                        self.results[job.name] = JobResult(job.name, False, f"start failed: {e}",
                                                           arrival=job.arrival)
                        progressed = True
                        break
                    self.used += need
                    self.peak_used = max(self.peak_used, self.used)
                    self.active.append((job, handle, need, now - t0))
                    progressed = True
                    break

    def _reap(self, now, t0):
        alive = []
        for handle, need in self.zombies:
            if self.backend.poll(handle) == "running":
                alive.append((handle, need))
            else:
                self.backend.release(handle)
                self.used -= need
        self.zombies = alive
        still = []
        for job, handle, need, adm in self.active:
            state = self.backend.poll(handle)
            elapsed = now - t0 - adm
            if state == "running" and elapsed <= job.deadline:
                still.append((job, handle, need, adm))
                continue
            if state == "running":
                res = JobResult(job.name, False, "deadline exceeded", arrival=job.arrival,
                                admitted=adm, finished=now - t0)
                # the device work is left to finish; its memory stays counted until it does
                self.zombies.append((handle, need))
                self.results[job.name] = res
                continue
            elif state == "error":
                res = JobResult(job.name, False, self.backend.error(handle), arrival=job.arrival,
                                admitted=adm, finished=now - t0)
                self.backend.release(handle)
            else:
                g = None if job.name in self.cancelled else self.backend.result(handle)
                res = JobResult(job.name, job.name not in self.cancelled,
                                "cancelled" if job.name in self.cancelled else "", g,
                                job.arrival, adm, now - t0)
                self.backend.release(handle)
            self.used -= need
            self.results[job.name] = res
        self.active = still

    def run(self, jobs, poll_sleep: float = 2e-4):
        """Serve `jobs` (arrival times relative to the start); returns the results."""
        order = sorted(jobs, key=lambda j: j.arrival)
        t0 = self.clock()
        i = 0
        while i < len(order) or self.pending or self.active or self.zombies:
            now = self.clock()
            while i < len(order) and order[i].arrival <= now - t0:
                if order[i].name in self.cancelled:
                    self.results[order[i].name] = JobResult(order[i].name, False, "cancelled",
                                                            arrival=order[i].arrival)
                else:
                    self.pending.append(order[i])
                i += 1
            self._reap(now, t0)
            self._admit(self.clock(), t0)
            if not self.active and not self.pending and i < len(order):
                time.sleep(max(0.0, min(order[i].arrival - (self.clock() - t0), 0.01)))
            elif self.active:
                time.sleep(poll_sleep)
        return self.results

    @staticmethod
    def stats(results: dict, wall: float | None = None):
        lat = np.array([r.latency for r in results.values() if r.ok])
        out = {"jobs": len(results), "ok": int(sum(r.ok for r in results.values()))}
        if lat.size:
            out.update(p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                       mean_s=float(lat.mean()))
            span = wall if wall is not None else max(r.finished for r in results.values() if r.ok)
            out["jobs_per_s"] = float(lat.size / span) if span > 0 else None
        return out


class GpuBackend:
    """Runs a job through libwp.so on its own stream: H2D of the inputs, probed forward,
    residual, probed adjoint + imaging, D2H of the gradient, then an event.

    The host work of a start (the model upload, its validation, which synchronises the
    job's stream once, and the enqueueing of every launch of the job) runs on a pool of
    submit threads, so the scheduler thread keeps polling and admitting while a long job
    is being enqueued; `poll` reports "running" until the submit has finished and the
    job's final event has completed."""

    def __init__(self, device="cuda", allocator=None, submit_threads: int = 4):
        import concurrent.futures as cf

        import torch
        from . import wp
        self.torch, self.wp = torch, wp
        self.device = torch.device(device)
        if self.device.index is None:   # submit threads start on device 0: pin the index
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.alloc = allocator or (lambda nbytes: torch.empty(nbytes, dtype=torch.uint8,
                                                              device=self.device))
        self.pool = cf.ThreadPoolExecutor(max_workers=submit_threads,
                                          thread_name_prefix="wp-submit")

    def _geom(self, job):
        return self.wp.Geometry(job.src, job.rec)

    def _model(self, job, m, th=None):
        kw = {}
        if th is not None:
            kw = dict(eps=th[0], delta=th[1], theta=th[2], phi=th[3])
        return self.wp.Model(job.ndim, job.nx, job.ny, job.nz, job.nbl, job.h, job.h, job.h,
                             job.dt, job.nt, m, job.damp_v, **kw)

    def footprint(self, job) -> int:
        wp = self.wp
        N = int(np.prod(job.m.shape))
        r = job.Q.shape[-1]
        # ws needs a model handle; estimate it from the layout sizes exactly by creating
        # a handle on the first call per grid shape.
        F = job.fields
        key = (job.ndim, job.nx, job.ny, job.nz, job.nbl, job.nt, r, job.Tb, job.rec.shape[1], F)
        if not hasattr(self, "_fp"):
            self._fp = {}
        if key not in self._fp:
            m = self.torch.from_numpy(np.ascontiguousarray(job.m.ravel())).to(self.device)
            th = None
            if job.thomsen is not None:   # zero fields: only the layout matters here
                th = [self.torch.zeros(N, device=self.device) for _ in range(4)]
            M = self._model(job, m, th)
            ws = wp.wp_workspace_bytes(M.handle, self._geom(job).c, r, job.Tb, wp.WP_MODE_PROBED)
            RS = M.use_aligned_probes()
            M.close()
            io = 4 * (N * (1 + (4 if F == 2 else 0)) + F * r * RS + N + 3 * job.nt * job.rec.shape[1]
                      + job.nt * (r + 1))
            self._fp[key] = ws + io
        return self._fp[key]

    def start(self, job):
        """Queue the job's host work on a submit thread; returns its handle at once."""
        return {"job": job, "future": self.pool.submit(self._submit, job)}

    def _submit(self, job):
        torch, wp = self.torch, self.wp
        dev = self.device
        torch.cuda.set_device(dev)
        st = torch.cuda.Stream(device=dev)
        h = {"job": job, "stream": st}
        r = job.Q.shape[-1]
        with torch.cuda.stream(st):
            m = torch.from_numpy(np.ascontiguousarray(job.m.ravel(), dtype=np.float32)).pin_memory().to(dev, non_blocking=True)
            wav = torch.from_numpy(job.wavelet.astype(np.float32)).to(dev, non_blocking=True)
            Q = torch.from_numpy(np.ascontiguousarray(job.Q, dtype=np.float32)).to(dev, non_blocking=True)
            dobs = torch.from_numpy(np.ascontiguousarray(job.d_obs, dtype=np.float32)).pin_memory().to(dev, non_blocking=True)
            th = None
            if job.thomsen is not None:
                th = [torch.from_numpy(np.ascontiguousarray(f.ravel(), dtype=np.float32)).pin_memory()
                      .to(dev, non_blocking=True) for f in job.thomsen]
            st.synchronize()   # the model must be on the device before it is validated
            M = self._model(job, m, th)
            G = self._geom(job)
            N = M.N
            RS = M.use_aligned_probes()   # P_u stays internal: kept in the contraction's layout
            ws = self.alloc(wp.wp_workspace_bytes(M.handle, G.c, r, job.Tb, wp.WP_MODE_PROBED))
            Pu = torch.empty((job.fields, r, RS), device=dev)
            dsyn = torch.empty_like(dobs)
            res = torch.empty_like(dobs)
            J = torch.zeros(1, dtype=torch.float64, device=dev)
            rws = wp.workspace(wp.wp_residual_workspace_bytes(dsyn.numel()), dev)
            g = torch.empty(N, device=dev)
            wp.wp_probe_forward(M.handle, G.c, wav, Q, r, job.Tb, Pu, dsyn, ws, st)
            wp.wp_residual(dsyn, dobs, res, dsyn.numel(), J, rws, st)
            wp.wp_adjoint_image(M.handle, G.c, res, Q, r, job.Tb, 1.0 / r, Pu, g, None, ws, st)
            host = torch.empty(N, pin_memory=True)
            host.copy_(g, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        h.update(M=M, G=G, keep=(m, wav, Q, dobs, ws, Pu, dsyn, res, J, rws, g, th), host=host, event=ev)
        return h

    def _started(self, h):
        """The submit's result once it has finished (None while it runs)."""
        if "run" not in h:
            f = h["future"]
            if not f.done():
                return None
            h["run"] = f.result()   # re-raises a failure of the submit
        return h["run"]

    def poll(self, h) -> str:
        try:
            run = self._started(h)
            if run is None:
                return "running"
            return "done" if run["event"].query() else "running"
        except Exception as e:  # the submit failed, or a CUDA error surfaced on the stream
            h["err"] = str(e)
            return "error"

    def error(self, h) -> str:
        return h.get("err", "unknown error")

    def result(self, h):
        return h["run"]["host"].numpy().copy()

    def release(self, h):
        f = h.get("future")
        if f is not None:
            try:
                run = f.result()   # a timed-out job is released only after its submit ended
                run["event"].synchronize()
                run["M"].close()
            except Exception:
                pass
        h.clear()

