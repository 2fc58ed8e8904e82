"""Host logic of the serving loop (admission by device-memory budget, FIFO order,
the resident-handle cache and its LRU eviction, failures), driven by a fake engine
on the CPU: no GPU and no library call."""
import threading
import time
from dataclasses import dataclass

import numpy as np
import pytest

from paper_2601_12941_gb300.serve import AdmissionError, Server
from synth import workloads as WL


@dataclass
class FakeJob:
    id: int
    bytes: int
    dur: float = 0.02
    key: object = None
    fail: bool = False


class FakeEngine:
    """Tracks the bytes its live handles hold and how many jobs run at once."""

    def __init__(self, budget):
        self.budget = budget
        self.lock = threading.Lock()
        self.live = 0
        self.max_live = 0
        self.running = 0
        self.max_running = 0
        self.opened = 0
        self.closed = 0
        self.over_budget = []
        self.start_order = []

    def worker_init(self):
        pass

    def make_stream(self):
        return type("S", (), {"cuda_stream": 0})()

    def estimate(self, job):
        if job.bytes < 0:
            raise ValueError("bad job")
        return job.bytes

    def estimate_reuse(self, handle, job):
        return max(handle["bytes"], job.bytes)

    def cache_key(self, job):
        return job.key

    def _grow(self, delta):
        with self.lock:
            self.live += delta
            self.max_live = max(self.max_live, self.live)
            if self.live > self.budget:
                self.over_budget.append(self.live)

    def open(self, job):
        self._grow(job.bytes)
        with self.lock:
            self.opened += 1
        return {"bytes": job.bytes}

    def reuse(self, handle, job):
        new = max(handle["bytes"], job.bytes)
        self._grow(new - handle["bytes"])
        handle["bytes"] = new

    def run(self, handle, job, stream):
        with self.lock:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
            self.start_order.append(job.id)
        time.sleep(job.dur)
        with self.lock:
            self.running -= 1
        if job.fail:
            raise RuntimeError("job %d failed" % job.id)
        return dict(fields={"u": np.array([float(job.id)])}, n_points=1, nx=1, ny=1, n_accepted=1, n_waves=1)

    def bytes(self, handle):
        return handle["bytes"]

    def close(self, handle):
        self._grow(-handle["bytes"])
        with self.lock:
            self.closed += 1

    @staticmethod
    def reusable_after(exc):
        return False


def test_results_reach_their_jobs():
    eng = FakeEngine(1000)
    with Server(workers=4, hbm_budget=1000, engine=eng) as srv:
        futs = [srv.submit(FakeJob(i, 10, dur=0.001 * (i % 5))) for i in range(40)]
        res = [f.result(timeout=30) for f in futs]
    assert [r.fields["u"][0] for r in res] == [float(i) for i in range(40)]
    st = srv.stats()
    assert st["completed"] == 40 and st["submitted"] == 40
    assert eng.live == 0 and eng.opened == eng.closed == 40


def test_budget_bounds_concurrency_and_fifo_order():
    eng = FakeEngine(100)
    with Server(workers=4, hbm_budget=100, engine=eng) as srv:
        futs = [srv.submit(FakeJob(i, 40, dur=0.03)) for i in range(8)]
        res = [f.result(timeout=30) for f in futs]
    assert not eng.over_budget
    assert eng.max_running <= 2            # two 40-byte jobs fit in 100, three do not
    assert srv.stats()["peak_bytes"] <= 100
    admits = [r.t_admit for r in res]
    assert admits == sorted(admits)        # admitted in submission order
    assert srv.stats()["memory_waits"] >= 1


def test_oversized_job_is_rejected_and_serving_continues():
    eng = FakeEngine(100)
    with Server(workers=2, hbm_budget=100, engine=eng) as srv:
        big = srv.submit(FakeJob(0, 101))
        ok = [srv.submit(FakeJob(i, 30)) for i in range(1, 5)]
        with pytest.raises(AdmissionError):
            big.result(timeout=30)
        assert all(f.result(timeout=30).fields["u"][0] == i + 1 for i, f in enumerate(ok))
    assert srv.stats()["rejected"] == 1


def test_invalid_and_failing_jobs_fail_their_futures_only():
    eng = FakeEngine(100)
    with Server(workers=2, hbm_budget=100, engine=eng) as srv:
        bad = srv.submit(FakeJob(0, -1))
        boom = srv.submit(FakeJob(1, 10, fail=True))
        good = srv.submit(FakeJob(2, 10))
        with pytest.raises(ValueError):
            bad.result(timeout=30)
        with pytest.raises(RuntimeError, match="job 1 failed"):
            boom.result(timeout=30)
        assert good.result(timeout=30).fields["u"][0] == 2.0
    st = srv.stats()
    assert st["failed"] == 1 and st["invalid"] == 1 and st["completed"] == 1
    assert eng.live == 0


def test_cache_hits_and_lru_eviction():
    eng = FakeEngine(100)
    with Server(workers=1, hbm_budget=100, engine=eng) as srv:
        order = ["A", "B", "C", "B", "A"]
        res = [srv.submit(FakeJob(i, 40, dur=0.001, key=k)).result(timeout=30) for i, k in enumerate(order)]
        st = srv.stats()
    # A, B cached (80); C needs 40: evict A (LRU); B hits; A misses and evicts C (LRU after B's reuse)
    assert [r.cache_hit for r in res] == [False, False, False, True, False]
    assert st["cache_hits"] == 1 and st["cache_misses"] == 4 and st["evictions"] == 2
    assert st["cached_handles"] == 2 and st["cached_bytes"] == 80
    assert not eng.over_budget
    assert eng.live == 0                   # close() frees the cached handles


def test_max_cached_bounds_idle_handles():
    eng = FakeEngine(1000)
    with Server(workers=1, hbm_budget=1000, engine=eng, max_cached=1) as srv:
        for i, k in enumerate(["A", "B", "A"]):
            srv.submit(FakeJob(i, 10, dur=0.001, key=k)).result(timeout=30)
        st = srv.stats()
    assert st["cached_handles"] == 1 and st["cache_hits"] == 0 and st["evictions"] == 2


def test_close_drains_pending_jobs():
    eng = FakeEngine(100)
    srv = Server(workers=1, hbm_budget=100, engine=eng)
    futs = [srv.submit(FakeJob(i, 10, dur=0.005)) for i in range(10)]
    srv.close()
    assert all(f.done() and f.exception() is None for f in futs)
    with pytest.raises(RuntimeError):
        srv.submit(FakeJob(99, 10))


def test_serving_stream_recipe():
    jobs = WL.serving_stream(n_jobs=50)
    assert [j.index for j in jobs] == list(range(50))
    assert all(b.arrival_s > a.arrival_s for a, b in zip(jobs, jobs[1:]))
    for j in jobs:
        w = j.workload
        assert 15 <= w.subset_size <= 61 and w.subset_size % 2 == 1 and 1 <= w.subset_step <= 10
        assert 512 <= w.width <= 16384 and w.width == w.height and w.dtype in ("u8", "u16")


def test_engine_cache_key_separates_what_the_resident_reference_depends_on():
    # the resident reference plane differs with the interpolant and the precision, so
    # jobs that differ there must not share a cached handle; seeds, subsets and the
    # other parameters do not enter the key (no GPU call: the key is host logic)
    pytest.importorskip("torch")
    from paper_2601_12941_gb300.serve import Job, LibdicEngine

    eng = LibdicEngine()
    ref = np.zeros((64, 80), np.uint8)
    base = dict(ref=ref, deformed=ref, seeds=[(40, 32)], ref_key="r0")
    k = eng.cache_key(Job(**base))
    assert k == eng.cache_key(Job(**base, subset_size=31, subset_step=2, shape="quadratic",
                                  params=dict(cost="nssd", optimizer="lm", init="fft")))
    assert k != eng.cache_key(Job(**base, interp="bicubic"))
    assert k != eng.cache_key(Job(**base, params=dict(precision="fp64")))
    assert k != eng.cache_key(Job(**dict(base, ref=ref.astype(np.uint16))))
    assert eng.cache_key(Job(**dict(base, ref_key=None))) is None
