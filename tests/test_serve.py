"""Host logic of the continuous-batching scheduler, with a fake backend (no GPU):
admission by footprint, bounded concurrency, memory budget never exceeded, and host-side
fault injection (allocation failure, cancellation, deadline) that leaves the other jobs'
results unchanged."""
import time

import numpy as np
import pytest

from paper_2201_06914_gb300.serve import JobResult, Scheduler


class Job:
    def __init__(self, name, size, duration, arrival=0.0, deadline=60.0):
        self.name, self.size, self.duration = name, size, duration
        self.arrival, self.deadline = arrival, deadline


class FakeBackend:
    """Jobs 'run' for job.duration seconds; the result is a value derived from the name."""

    def __init__(self, fail_start=()):
        self.fail_start = set(fail_start)
        self.live = 0
        self.max_live = 0
        self.released = []

    def footprint(self, job):
        return job.size

    def start(self, job):
        if job.name in self.fail_start:
            raise MemoryError("injected allocation failure")
        self.live += 1
        self.max_live = max(self.max_live, self.live)
        return {"job": job, "end": time.perf_counter() + job.duration}

    def poll(self, h):
        return "done" if time.perf_counter() >= h["end"] else "running"

    def error(self, h):
        return "error"

    def result(self, h):
        return np.full(3, float(hash(h["job"].name) % 1000))

    def release(self, h):
        self.live -= 1
        self.released.append(h["job"].name)


def test_budget_and_concurrency():
    be = FakeBackend()
    rng = np.random.default_rng(0)
    jobs = [Job(f"j{i}", int(rng.integers(1, 5)), 0.01 + 0.02 * rng.random(), 0.003 * i)
            for i in range(30)]
    sched = Scheduler(be, mem_budget=8, max_active=3)
    res = sched.run(jobs)
    assert len(res) == 30 and all(r.ok for r in res.values())
    assert sched.peak_used <= 8
    assert be.max_live <= 3
    st = Scheduler.stats(res)
    assert st["ok"] == 30 and st["p99_s"] >= st["p50_s"] > 0


def test_oversized_job_rejected_others_served():
    be = FakeBackend()
    jobs = [Job("big", 100, 0.01), Job("a", 2, 0.01), Job("b", 2, 0.01)]
    res = Scheduler(be, mem_budget=10).run(jobs)
    assert not res["big"].ok and "budget" in res["big"].error
    assert res["a"].ok and res["b"].ok


def test_injected_allocation_failure_isolated():
    be = FakeBackend(fail_start={"bad"})
    jobs = [Job("a", 2, 0.01), Job("bad", 2, 0.01, 0.001), Job("c", 2, 0.01, 0.002)]
    res = Scheduler(be, mem_budget=10).run(jobs)
    assert not res["bad"].ok and "injected" in res["bad"].error
    base = Scheduler(FakeBackend(), mem_budget=10).run([Job("a", 2, 0.01), Job("c", 2, 0.01)])
    for n in ("a", "c"):
        assert res[n].ok and np.array_equal(res[n].g, base[n].g)


def test_cancel_pending_and_deadline():
    be = FakeBackend()
    sched = Scheduler(be, mem_budget=4, max_active=1)
    sched.cancel("later")
    jobs = [Job("slow", 1, 0.2, deadline=0.02), Job("later", 1, 0.01, 0.001), Job("ok", 1, 0.01, 0.002)]
    res = sched.run(jobs)
    assert res["later"].error == "cancelled" and not res["later"].ok
    assert res["slow"].error == "deadline exceeded"
    assert res["ok"].ok
    assert sched.used == 0 and "slow" in be.released   # timed-out work released once done


def test_stats_percentiles():
    res = {f"j{i}": JobResult(f"j{i}", True, finished=float(i + 1), arrival=0.0) for i in range(100)}
    st = Scheduler.stats(res, wall=100.0)
    assert st["p50_s"] == pytest.approx(50.5)
    assert st["p99_s"] == pytest.approx(99.01)
    assert st["jobs_per_s"] == pytest.approx(1.0)
