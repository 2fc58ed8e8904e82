"""Continuous-batching server over libdic handles.

Jobs (one reference/deformed pair each, with their own subset settings) queue in
arrival order. A dispatcher admits the oldest job as soon as a worker is free and
the job's device footprint fits the memory budget; idle cached handles are evicted,
least recently used first, to make room, and a job that cannot fit even on an
empty device fails with AdmissionError. Each worker is a host thread with its own
CUDA stream, so the wave launches of several jobs interleave on the GPU and small
jobs fill the SMs that a large job's narrow frontier leaves idle.

Handles stay resident per reference image (the job's ``ref_key``): a later job on
the same reference re-grids the cached handle (dic_set_subsets) and replaces only
the deformed image, so the reference is neither uploaded nor prefiltered again.

The paper has no serving layer; this is infrastructure around the correlation,
whose every step runs in libdic's kernels. PyTorch is used here for streams and
for the device-to-host copy of the requested result fields.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field
from typing import Any, Hashable

import numpy as np

from . import binding as B


class AdmissionError(RuntimeError):
    """The job's device footprint exceeds the whole memory budget."""


@dataclass
class Job:
    """One correlation request. ``ref``/``deformed``: 2-D numpy arrays (copied by the
    library) or CUDA tensors (borrowed until the job completes; a cached handle keeps
    its reference tensor alive). Jobs that pass the same ``ref_key`` promise the same
    reference image."""
    ref: Any
    deformed: Any
    seeds: Any
    subset_size: int = 21
    subset_step: int = 5
    shape: str = "affine"
    interp: str = "bspline3"
    roi: Any = None
    params: dict = field(default_factory=dict)
    ref_key: Hashable = None
    fields: tuple = ("u", "v", "zncc", "status")


@dataclass
class JobResult:
    fields: dict
    n_points: int
    nx: int
    ny: int
    n_accepted: int
    n_waves: int
    cache_hit: bool
    device_bytes: int
    worker: int
    t_submit: float
    t_admit: float
    t_start: float
    t_end: float

    @property
    def latency_s(self) -> float:
        return self.t_end - self.t_submit

    @property
    def queue_s(self) -> float:
        return self.t_admit - self.t_submit


class LibdicEngine:
    """Runs jobs through libdic on one device."""

    def __init__(self, device: int = 0):
        import torch

        self.torch = torch
        self.device = device
        B.load()

    def worker_init(self):
        self.torch.cuda.set_device(self.device)

    def make_stream(self):
        return self.torch.cuda.Stream(device=self.device)

    @staticmethod
    def _shape(job):
        return B.SHAPES[job.shape] if isinstance(job.shape, str) else job.shape

    @staticmethod
    def _params(job):
        return B.params(**job.params)

    @staticmethod
    def _n_seeds(job):
        return int(np.asarray(job.seeds).reshape(-1, 2).shape[0])

    @staticmethod
    def _on_device(a):
        return not isinstance(a, np.ndarray)

    def estimate(self, job) -> int:
        h, w = job.ref.shape
        ref = B.image_desc(w, h, B.image_dtype_code(job.ref), self._on_device(job.ref))
        dfm = B.image_desc(w, h, B.image_dtype_code(job.deformed), self._on_device(job.deformed))
        return B.dic_estimate_device_bytes(ref, dfm, job.roi is not None, job.subset_size, job.subset_step,
                                           self._shape(job), self._params(job), self._n_seeds(job))

    def estimate_reuse(self, handle, job) -> int:
        h, w = job.ref.shape
        dfm = B.image_desc(w, h, B.image_dtype_code(job.deformed), self._on_device(job.deformed))
        return B.dic_estimate_regrid_bytes(handle["h"], dfm, job.roi is not None, job.subset_size, job.subset_step,
                                           self._shape(job), self._params(job), self._n_seeds(job))

    def cache_key(self, job):
        if job.ref_key is None:
            return None
        h, w = job.ref.shape
        # the resident reference plane depends on the interpolant and the precision
        return (job.ref_key, w, h, B.image_dtype_code(job.ref), self._on_device(job.ref),
                self._params(job).precision, job.interp)

    def open(self, job):
        h, keep = B.dic_create(job.ref, job.deformed, job.roi, job.subset_size, job.subset_step, self._shape(job),
                               B.INTERPS[job.interp])
        # a borrowed reference must outlive the handle
        return {"h": h, "ref": keep[0] if self._on_device(job.ref) else None}

    def reuse(self, handle, job):
        B.dic_set_subsets(handle["h"], job.roi, job.subset_size, job.subset_step, self._shape(job))
        B.dic_set_deformed(handle["h"], job.deformed)

    def run(self, handle, job, stream) -> dict:
        torch = self.torch
        h = handle["h"]
        B.dic_set_params(h, self._params(job))
        B.dic_correlate(h, job.seeds, stream.cuda_stream)
        r = B.dic_get_results(h, on_device=True)
        host = {}
        with torch.cuda.stream(stream):
            for name in job.fields:
                t = r[name]
                host[name] = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                host[name].copy_(t, non_blocking=True)
        stream.synchronize()
        return dict(fields={k: v.numpy() for k, v in host.items()}, n_points=r["n_points"], nx=r["nx"],
                    ny=r["ny"], n_accepted=r["n_accepted"], n_waves=r["n_waves"])

    def bytes(self, handle) -> int:
        return B.dic_get_device_bytes(handle["h"])

    def close(self, handle):
        B.dic_destroy(handle["h"])

    @staticmethod
    def reusable_after(exc) -> bool:
        # a job that ended with no accepted point leaves a valid handle
        return isinstance(exc, B.DicError) and exc.code == B.DIC_ENOSEED


_COUNTS = ("submitted", "completed", "failed", "invalid", "rejected", "cache_hits", "cache_misses",
           "evictions", "memory_waits", "close_errors")


@dataclass
class _Entry:
    key: Any
    handle: Any
    bytes: int


@dataclass
class _Item:
    job: Any
    future: Future
    est: int
    t_submit: float
    waited_for_memory: bool = False


class Server:
    """``submit(job) -> Future[JobResult]``; see the module docstring.

    workers     : host threads (each with its own stream).
    hbm_budget  : device bytes for handles; default 90% of the free memory at start.
    engine      : the job runner (LibdicEngine on ``device`` by default).
    max_cached  : upper bound on idle cached handles (None: the budget alone)."""

    def __init__(self, workers: int = 4, hbm_budget: int | None = None, engine=None, device: int = 0,
                 max_cached: int | None = None):
        if workers < 1:
            raise ValueError("at least one worker")
        self.engine = engine if engine is not None else LibdicEngine(device)
        if hbm_budget is None:
            import torch

            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget = int(0.9 * free)
        self.budget = int(hbm_budget)
        self.max_cached = max_cached
        self._cv = threading.Condition()
        self._pending: collections.deque[_Item] = collections.deque()
        self._idle: collections.OrderedDict[int, _Entry] = collections.OrderedDict()  # LRU order
        self._idle_seq = 0
        self._reserved = 0
        self._cached = 0
        self._free_workers = workers
        self._closing = False
        self._work: collections.deque = collections.deque()
        self.counts = collections.Counter()
        self.peak_bytes = 0
        self.peak_busy = 0
        self._dispatcher = threading.Thread(target=self._dispatch, name="dic-dispatch", daemon=True)
        self._workers = [threading.Thread(target=self._work_loop, args=(i,), name="dic-worker-%d" % i, daemon=True)
                         for i in range(workers)]
        self._n_workers = workers
        for t in self._workers:
            t.start()
        self._dispatcher.start()

    # ---- client side -----------------------------------------------------
    def submit(self, job) -> Future:
        fut: Future = Future()
        t = time.perf_counter()
        try:
            est = int(self.engine.estimate(job))
        except Exception as e:  # invalid job: fail its future, keep serving
            fut.set_exception(e)
            with self._cv:
                self.counts["invalid"] += 1
            return fut
        with self._cv:
            if self._closing:
                raise RuntimeError("server is closed")
            self._pending.append(_Item(job, fut, est, t))
            self.counts["submitted"] += 1
            self._cv.notify_all()
        return fut

    def stats(self) -> dict:
        with self._cv:
            counts = {k: self.counts[k] for k in _COUNTS}
            counts.update(self.counts)
            return dict(counts, budget_bytes=self.budget, peak_bytes=self.peak_bytes,
                        reserved_bytes=self._reserved, cached_bytes=self._cached, cached_handles=len(self._idle),
                        peak_busy_workers=self.peak_busy, pending=len(self._pending))

    def close(self, wait: bool = True):
        with self._cv:
            self._closing = True
            self._cv.notify_all()
        if wait:
            self._dispatcher.join()
            for t in self._workers:
                t.join()
            with self._cv:
                idle = list(self._idle.values())
                self._idle.clear()
                self._cached = 0
            for e in idle:
                self._close_quietly(e.handle)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- dispatcher --------------------------------------------------------
    def _used(self) -> int:
        return self._reserved + self._cached

    def _take_idle(self, key):
        if key is None:
            return None
        for seq in reversed(self._idle):  # most recently used first
            e = self._idle[seq]
            if e.key == key:
                del self._idle[seq]
                self._cached -= e.bytes
                return e
        return None

    def _put_idle(self, e: _Entry):
        self._idle_seq += 1
        self._idle[self._idle_seq] = e
        self._cached += e.bytes

    def _close_quietly(self, handle):
        try:
            self.engine.close(handle)
        except Exception:
            with self._cv:
                self.counts["close_errors"] += 1

    def _reuse_bytes(self, entry, item) -> int:
        try:
            return int(self.engine.estimate_reuse(entry.handle, item.job))
        except Exception:
            return entry.bytes + item.est  # an upper bound

    def _dispatch(self):
        while True:
            victims = []
            admitted = False
            with self._cv:
                while not self._pending or self._free_workers == 0:
                    if self._closing and not self._pending:
                        for _ in range(self._n_workers):
                            self._work.append(None)
                        self._cv.notify_all()
                        return
                    self._cv.wait()
                item = self._pending[0]
                key = self.engine.cache_key(item.job)
                entry = self._take_idle(key)
                need = item.est if entry is None else self._reuse_bytes(entry, item)
                if need > self.budget and entry is not None:
                    victims.append(entry)  # a cached handle too large to reuse
                    entry, need = None, item.est
                if need > self.budget:
                    self._pending.popleft()
                    self.counts["rejected"] += 1
                    item.future.set_exception(AdmissionError(
                        "job needs %d device bytes, the budget is %d" % (need, self.budget)))
                elif self._reserved + need <= self.budget:
                    # fits once enough idle handles are evicted, least recently used first
                    while self._used() + need > self.budget:
                        _, v = self._idle.popitem(last=False)
                        self._cached -= v.bytes
                        victims.append(v)
                    self._pending.popleft()
                    self._reserved += need
                    self._free_workers -= 1
                    self.peak_busy = max(self.peak_busy, self._n_workers - self._free_workers)
                    self.counts["cache_hits" if entry is not None else "cache_misses"] += 1
                    if item.waited_for_memory:
                        self.counts["memory_waits"] += 1
                    admitted = True
                else:
                    # running jobs hold the memory: wait for one to finish
                    if entry is not None:
                        self._put_idle(entry)
                    item.waited_for_memory = True
                    self._cv.wait(timeout=0.05)
            # evicted handles are freed before the job that needed the room starts
            for v in victims:
                self._close_quietly(v.handle)
            with self._cv:
                self.counts["evictions"] += len(victims)
                if admitted:
                    self.peak_bytes = max(self.peak_bytes, self._used())
                    self._work.append((item, entry, need, time.perf_counter()))
                    self._cv.notify_all()

    # ---- workers -----------------------------------------------------------
    def _work_loop(self, wid: int):
        self.engine.worker_init()
        stream = self.engine.make_stream()
        while True:
            with self._cv:
                while not self._work:
                    self._cv.wait()
                task = self._work.popleft()
            if task is None:
                return
            item, entry, need, t_admit = task
            job = item.job
            t_start = time.perf_counter()
            handle, out, exc, keep = None, None, None, False
            try:
                if entry is not None:
                    handle = entry.handle
                    self.engine.reuse(handle, job)
                else:
                    handle = self.engine.open(job)
                out = self.engine.run(handle, job, stream)
                keep = True
            except Exception as e:  # reported through the future
                exc = e
                keep = handle is not None and self.engine.reusable_after(e)
            key = self.engine.cache_key(job)
            cache = keep and key is not None and (self.max_cached is None or self.max_cached > 0)
            nbytes = self.engine.bytes(handle) if handle is not None and keep else 0
            if handle is not None and not cache:
                self._close_quietly(handle)  # freed before the reservation is released
            t_end = time.perf_counter()
            evict = []
            with self._cv:
                self._reserved -= need
                self._free_workers += 1
                if cache:
                    self._put_idle(_Entry(key, handle, nbytes))
                    while self.max_cached is not None and len(self._idle) > self.max_cached:
                        _, v = self._idle.popitem(last=False)
                        self._cached -= v.bytes
                        evict.append(v)
                self.peak_bytes = max(self.peak_bytes, self._used())
                self.counts["failed" if exc is not None else "completed"] += 1
                self._cv.notify_all()
            for v in evict:
                self._close_quietly(v.handle)
            if evict:
                with self._cv:
                    self.counts["evictions"] += len(evict)
            if exc is not None:
                item.future.set_exception(exc)
            else:
                item.future.set_result(JobResult(
                    fields=out["fields"], n_points=out["n_points"], nx=out["nx"], ny=out["ny"],
                    n_accepted=out["n_accepted"], n_waves=out["n_waves"], cache_hit=entry is not None,
                    device_bytes=nbytes, worker=wid, t_submit=item.t_submit, t_admit=t_admit,
                    t_start=t_start, t_end=t_end))
