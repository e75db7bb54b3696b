"""Continuous-batching imaging server.

Imaging requests (visibilities + imaging parameters) arrive at any time.  The
server keeps a pool of resident *slots*.  Each slot is an ``Imager``:
  - a plan with its cuFFT plan, taper table and kernel fits;
  - a binning workspace and the w-planes;
  - device input buffers and a pinned host output buffer;
  - its own CUDA stream.

A scheduler thread admits queued requests as soon as a compatible slot is idle,
or HBM budget can be freed for a new one.  It enqueues each request's whole
path (host->device copy, bin, grid, FFT, w-correct, device->host copy) on the
slot's stream, and completes the request when the stream's event fires.  Work of
requests admitted while others run overlaps on the device.  With
``merge_small`` small requests admitted together (at most BATCH_MAX_VIS
visibilities each, same support and tile, FP32, fused transform) are gridded by
one launch over all their (request, plane, tile) work items
(rick_grid_sparse_batch) on the server's batch stream, between their binnings
and their transforms on their slots' streams.  It is off by default: on the
serving trace it made the saturated throughput a few percent lower (the merged
launch waits for every binning of its group, and every transform of the group
waits for it), while the requests' own launches already overlap on their
streams.

Admission is by HBM footprint: a request needs a slot with the same grid size,
tile and precision, and visibility and plane capacities at least its own; the
slot's plan is re-targeted to the request's plane count, field of view, w
range, image crop and gridding kernel (rick_plan_set_planes,
rick_plan_set_geometry, rick_plan_set_image_n, rick_plan_set_kernel), so the
plan and the buffers are reused.  If no idle slot fits, a new one is created
when budget - used >= its footprint, after evicting idle slots
least-recently-used first.  A request larger than the whole budget is rejected
with an error, and only that request fails.

``run_plain`` is the per-request baseline: a fresh plan and fresh allocations
for every request, run to completion before the next.
"""
from __future__ import annotations

import collections
import itertools
import math
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from . import rick as R
from .imager import IMAGE_FLAGS, Imager, grid_sparse_batch

MIN_CAPACITY = 1 << 20  # smaller requests share slots of this capacity
MIN_PLANES = 16         # plane capacity of a slot (more if a request needs more)
BATCH_MAX_VIS = 1 << 21  # requests up to this size are gridded in merged launches


def capacity_class(n_vis: int) -> int:
    """Visibility capacity of the slot serving n_vis (powers of two)."""
    c = MIN_CAPACITY
    while c < n_vis:
        c <<= 1
    return c


def plane_class(n_w: int) -> int:
    """Plane capacity of the slot serving n_w planes."""
    return max(int(n_w), MIN_PLANES)


def capacities(job) -> tuple:
    """(visibilities, planes) a slot must hold for the job."""
    return capacity_class(job.n_vis), plane_class(job.n_w)


@dataclass
class ImagingJob:
    """One imaging request.  uvw [n,3] f64, vis [n] c64, weight [n] f32 (or
    None) are host tensors (pinned memory lets the copies run asynchronously)."""
    uvw: object
    vis: object
    weight: object
    n: int
    n_w: int
    fov: float
    kernel: str = "kb"
    support: int = 7
    tile: int = 64
    precision: str = "fp32"
    w_range: tuple | None = None
    flags: int = IMAGE_FLAGS
    job_id: int = -1
    arrival: float = field(default_factory=time.perf_counter)
    image_n: int | None = None  # central crop of the n-cell grid (None: n)

    @property
    def n_vis(self) -> int:
        return int(self.uvw.shape[0])

    @property
    def side(self) -> int:
        """Side of the returned image."""
        return int(self.image_n) if self.image_n else self.n

    def key(self):
        """What a slot must share with the request (its capacities may be larger)."""
        return (self.n, self.tile, self.precision)


@dataclass
class JobResult:
    job_id: int
    image: np.ndarray
    latency_s: float
    queued_s: float
    slot: int


class AdmissionError(RuntimeError):
    """The request can never fit the server's HBM budget."""


class Admission:
    """Footprint accounting of resident slots (host-only logic)."""

    def __init__(self, budget_bytes: int, max_slots: int | None = None):
        self.budget = int(budget_bytes)
        self.max_slots = max_slots  # resident slots at most (None: budget only)
        self.slots = {}  # id -> dict(key, bytes, busy, last)
        self._ids = itertools.count()

    def used(self) -> int:
        return sum(s["bytes"] for s in self.slots.values())

    def plan(self, key, bytes_needed: int, cap=0):
        """('reuse', id) | ('new', [ids to evict]) | None (wait).  An idle slot
        of the same key with capacity >= cap (a number, or a tuple compared
        element by element) is reused (the smallest such, then the least
        recently used).  Raises AdmissionError if bytes_needed exceeds the
        whole budget."""
        if bytes_needed > self.budget:
            raise AdmissionError(f"request needs {bytes_needed} B, budget is {self.budget} B")

        def holds(c):
            if isinstance(cap, tuple):
                return all(a >= b for a, b in zip(c, cap))
            return c >= cap

        idle_same = [i for i, s in self.slots.items()
                     if s["key"] == key and not s["busy"] and holds(s["cap"])]
        if idle_same:
            return ("reuse", min(idle_same, key=lambda i: (self.slots[i]["cap"],
                                                          self.slots[i]["last"])))
        free = self.budget - self.used()
        count = len(self.slots)
        evict = []
        for i in sorted((i for i, s in self.slots.items() if not s["busy"]),
                        key=lambda i: self.slots[i]["last"]):
            if free >= bytes_needed and (self.max_slots is None or count < self.max_slots):
                break
            evict.append(i)
            free += self.slots[i]["bytes"]
            count -= 1
        fits = free >= bytes_needed and (self.max_slots is None or count < self.max_slots)
        return ("new", evict) if fits else None

    def add(self, key, nbytes: int, now: float, cap=0) -> int:
        i = next(self._ids)
        self.slots[i] = dict(key=key, bytes=int(nbytes), busy=True, last=now,
                             cap=cap if isinstance(cap, tuple) else int(cap))
        assert self.used() <= self.budget
        return i

    def acquire(self, i: int, now: float):
        self.slots[i]["busy"] = True
        self.slots[i]["last"] = now

    def release(self, i: int, now: float):
        self.slots[i]["busy"] = False
        self.slots[i]["last"] = now

    def remove(self, i: int):
        del self.slots[i]


def slot_footprint(job: ImagingJob) -> int:
    """Device bytes of a slot for job's key (without creating it)."""
    from . import rick as R
    from .imager import KERNELS, PRECISIONS
    cap, planes_cap = capacities(job)
    p = R.make_params(job.n, planes_cap, job.fov, KERNELS[job.kernel], job.support, tile=job.tile,
                      precision=PRECISIONS[job.precision], image_n=job.image_n or 0)
    ws, planes = R.rick_workspace_bytes(p, cap)
    # planes + workspace + cuFFT area (bounded by the planes' size for in-place
    # C2C) + the fused transform's work buffer + image + resident input buffers
    # (uvw, vis, weight)
    return ws + 2 * planes + R.rick_fused_work_bytes(p) + job.n * job.n * 4 + cap * (24 + 8 + 4)


class _Slot:
    def __init__(self, job: ImagingJob, device, out_host):
        import torch
        self.key = job.key()
        cap, planes_cap = capacities(job)
        self.imager = Imager(job.n, planes_cap, job.fov, kernel=job.kernel, support=job.support,
                             tile=job.tile, precision=job.precision, max_vis=cap,
                             device=device, image_n=job.image_n)
        self.kernel = (job.kernel, job.support)
        self.stream = torch.cuda.Stream(device=device)
        self.out = out_host  # pinned image buffer, from the server's pool
        self.event = None
        self.job = None
        self.future = None
        self.t_start = 0.0


class _PinnedPool:
    """Pinned host image buffers by image side, reused across slots
    (pinning host memory is slow; a new slot should not pay for it)."""

    def __init__(self):
        self.free = collections.defaultdict(list)
        self.lock = threading.Lock()

    def get(self, n: int):
        import torch
        with self.lock:
            if self.free[n]:
                return self.free[n].pop()
        return torch.empty((n, n), dtype=torch.float32).pin_memory()

    def put(self, buf):
        with self.lock:
            self.free[buf.shape[0]].append(buf)


class Server:
    """Continuous-batching server on one device (see the module docstring)."""

    def __init__(self, device="cuda:0", budget_bytes: int | None = None, max_running: int = 8,
                 max_slots: int | None = None, merge_small: bool = False):
        """merge_small: grid small requests admitted together in one merged
        launch (by default every request runs its own launches)."""
        import torch
        from concurrent.futures import ThreadPoolExecutor
        self.device = torch.device(device)
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget_bytes = int(0.8 * free)
        # resident slots beyond the running ones are kept for reuse; past the
        # cap the least recently used idle slot gives its memory back first
        self.admission = Admission(budget_bytes, max_slots or 2 * max_running)
        self.max_running = max_running
        self.merge_small = bool(merge_small)
        self.counters = dict(new_slots=0, reused=0, evicted=0, host_create_s=0.0,
                             host_launch_s=0.0, batches=0, batched=0)
        self._batch_stream = torch.cuda.Stream(device=self.device)
        # finished images leave the pinned buffers on worker threads, so the
        # scheduler never waits on a host copy
        self._copier = ThreadPoolExecutor(max_workers=4, thread_name_prefix="rick-copy")
        self._pending = collections.deque()
        self._slots = {}  # admission id -> _Slot
        self._pinned = _PinnedPool()
        self._cv = threading.Condition()
        self._stop = False
        self.peak_used = 0
        self._thread = threading.Thread(target=self._loop, name="rick-server", daemon=True)
        self._thread.start()

    # ---------------------------------------------------------------- API
    def submit(self, job: ImagingJob) -> Future:
        fut = Future()
        with self._cv:
            if self._stop:
                raise RuntimeError("server is closed")
            self._pending.append((job, fut))
            self._cv.notify()
        return fut

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify()
        self._thread.join()
        self._copier.shutdown(wait=True)
        for sid in list(self._slots):
            self._evict(sid)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------- scheduler
    def _running(self):
        return [i for i, s in self._slots.items() if s.job is not None]

    def _admit(self) -> bool:
        """Admit pending jobs in arrival order; a job that must wait for memory
        does not hold back later jobs that fit now."""
        progressed = False
        waiting = collections.deque()
        started = []  # (sid, slot, job, future) admitted in this pass, not yet enqueued
        while self._pending and len(self._running()) < self.max_running:
            job, fut = self._pending.popleft()
            try:
                need = slot_footprint(job)
                decision = self.admission.plan(job.key(), need, capacities(job))
            except Exception as e:  # invalid request or larger than the budget
                fut.set_exception(e)
                progressed = True
                continue
            if decision is None:
                waiting.append((job, fut))
                continue
            now = time.perf_counter()
            try:
                if decision[0] == "reuse":
                    sid = decision[1]
                    self.admission.acquire(sid, now)
                    slot = self._slots[sid]
                    self.counters["reused"] += 1
                else:
                    for sid in decision[1]:
                        self._evict(sid)
                    slot = _Slot(job, self.device, self._pinned.get(job.side))
                    sid = self.admission.add(job.key(), need, now, capacities(job))
                    self._slots[sid] = slot
                    self.peak_used = max(self.peak_used, self.admission.used())
                    self.counters["new_slots"] += 1
                    self.counters["host_create_s"] += time.perf_counter() - now
                self._prepare(slot, job, fut)
                started.append((sid, slot, job, fut))
            except Exception as e:
                fut.set_exception(e)
                if decision[0] == "reuse":
                    self.admission.release(decision[1], time.perf_counter())
            progressed = True
        self._pending.extendleft(reversed(waiting))
        if started:
            t0 = time.perf_counter()
            self._launch_group(started)
            self.counters["host_launch_s"] += time.perf_counter() - t0
        return progressed

    def _evict(self, sid):
        slot = self._slots.pop(sid)
        slot.stream.synchronize()  # idle already; the plan's work is complete
        slot.imager.close()
        if slot.out is not None:
            self._pinned.put(slot.out)
        self.admission.remove(sid)
        self.counters["evicted"] += 1

    def _prepare(self, slot, job, fut):
        """Claim the slot for the job and re-target its plan (host side; the slot
        is idle, so none of its work is in flight)."""
        slot.job, slot.future, slot.t_start = job, fut, time.perf_counter()
        if slot.out is None or slot.out.shape[0] != job.side:
            if slot.out is not None:
                self._pinned.put(slot.out)
            slot.out = self._pinned.get(job.side)
        if slot.kernel != (job.kernel, job.support):  # the slot is idle: its work is done
            slot.imager.set_kernel(job.kernel, job.support)
            slot.kernel = (job.kernel, job.support)
        if slot.imager.m != job.side:
            slot.imager.set_image_n(job.image_n)
        if slot.imager.n_w != job.n_w:
            slot.imager.set_planes(job.n_w)

    def _launch(self, slot, job):
        import torch
        with torch.cuda.stream(slot.stream):
            slot.imager.set_geometry(job.fov, job.w_range)
            slot.imager.image_from_host(job.uvw, job.vis, job.weight, slot.out, job.flags)
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)

    def _batchable(self, slot, job) -> bool:
        return (self.merge_small and job.n_vis <= BATCH_MAX_VIS and job.precision == "fp32"
                and slot.imager.fused
                and not slot.imager.params.options & R.RICK_OPT_DETERMINISTIC)

    def _launch_group(self, started):
        """Enqueue the jobs admitted in one pass: small compatible ones with one
        merged gridding launch per group, the others each on its own.  A launch
        that fails fails only its own request (or its merged group)."""
        groups = collections.defaultdict(list)
        for sid, slot, job, fut in started:
            key = (job.support, job.tile) if self._batchable(slot, job) else None
            groups[key].append((sid, slot))
        parts = []
        for key, members in groups.items():
            if key is None:
                parts += [[m] for m in members]
            else:
                parts += [members[i:i + R.RICK_GRID_BATCH_MAX]
                          for i in range(0, len(members), R.RICK_GRID_BATCH_MAX)]
        for part in parts:
            try:
                if len(part) == 1:
                    self._launch(part[0][1], part[0][1].job)
                else:
                    self._launch_batch([slot for _, slot in part])
            except Exception as e:
                for sid, slot in part:
                    self._fail(sid, slot, e)

    def _fail(self, sid, slot, err):
        """The request on this slot failed at launch: its future gets the error
        and the slot is idle again once the work enqueued on its stream is done."""
        fut = slot.future
        slot.stream.synchronize()
        slot.job = slot.future = slot.event = None
        self.admission.release(sid, time.perf_counter())
        if fut is not None and not fut.done():
            fut.set_exception(err)

    def _launch_batch(self, slots):
        import torch
        binned = []
        for slot in slots:
            job = slot.job
            with torch.cuda.stream(slot.stream):
                slot.imager.set_geometry(job.fov, job.w_range)
                slot.imager.bin_from_host(job.uvw, job.vis, job.weight)
                ev = torch.cuda.Event()
                ev.record(slot.stream)
                binned.append(ev)
        bs = self._batch_stream
        with torch.cuda.stream(bs):
            for ev in binned:
                bs.wait_event(ev)
            grid_sparse_batch([slot.imager for slot in slots])
            gridded = torch.cuda.Event()
            gridded.record(bs)
        for slot in slots:
            with torch.cuda.stream(slot.stream):
                slot.stream.wait_event(gridded)
                slot.imager.transform_to_host(slot.out, slot.job.flags)
                slot.event = torch.cuda.Event()
                slot.event.record(slot.stream)
        self.counters["batches"] += 1
        self.counters["batched"] += len(slots)

    def _complete(self) -> bool:
        progressed = False
        for sid in self._running():
            slot = self._slots[sid]
            if not slot.event.query():
                continue
            job, fut, buf = slot.job, slot.future, slot.out
            slot.job = slot.future = slot.event = None
            slot.out = None  # the next job on this slot takes another pooled buffer
            self.admission.release(sid, time.perf_counter())
            self._copier.submit(self._deliver, job, fut, buf, slot.t_start, sid)
            progressed = True
        return progressed

    def _deliver(self, job, fut, buf, t_start, sid):
        img = buf.numpy().copy()
        self._pinned.put(buf)
        now = time.perf_counter()
        fut.set_result(JobResult(job.job_id, img, now - job.arrival, t_start - job.arrival, sid))

    def _loop(self):
        import torch
        torch.cuda.set_device(self.device)
        while True:
            with self._cv:
                if self._stop and not self._pending and not self._running():
                    return
                if not self._pending and not self._running():
                    self._cv.wait(timeout=0.05)
            try:
                busy = self._complete()
                with self._cv:
                    busy = self._admit() or busy
            except Exception as e:  # fail every outstanding request, keep serving
                for sid in self._running():
                    s = self._slots[sid]
                    if s.future and not s.future.done():
                        s.future.set_exception(e)
                    s.job = s.future = s.event = None
                    self.admission.release(sid, time.perf_counter())
                busy = True
            if not busy:
                time.sleep(50e-6)


def run_plain(job: ImagingJob, device="cuda:0") -> np.ndarray:
    """The per-request baseline: fresh plan and allocations, run, tear down."""
    import torch
    with torch.cuda.device(device):
        im = Imager(job.n, job.n_w, job.fov, kernel=job.kernel, support=job.support,
                    tile=job.tile, precision=job.precision, w_range=job.w_range,
                    max_vis=max(job.n_vis, 1), device=device, image_n=job.image_n)
        out = torch.empty((job.side, job.side), dtype=torch.float32).pin_memory()
        im.image_from_host(job.uvw, job.vis, job.weight, out, job.flags)
        torch.cuda.current_stream().synchronize()
        img = out.numpy().copy()
        im.close()
        del im
    return img


def fov_for(n: int, support: int, uv_max: float) -> float:
    """Field of view whose uv cell keeps every footprint of |u|,|v| <= uv_max on
    an n-cell grid: (n/2 - W - 1) / uv_max."""
    return (n / 2 - support - 1) / uv_max


def poisson_arrivals(n_jobs: int, rate: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n_jobs))


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if len(xs) else math.nan
