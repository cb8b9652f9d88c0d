"""Serving loop: continuous batching of hull requests under a memory budget.

Requests (an (n, 3) int32 point array each) arrive at any time through
HullServer.submit(), which returns a Future resolved with the canonical face
array.  One scheduler thread
  * admits requests in arrival order while their device footprint (input
    12 n bytes + output 12 (2n - 4) bytes) fits in what the budget leaves
    after the resident buffers; a request that can never fit is rejected
    with HULL3D_ERR_BUDGET;
  * gathers admitted small clouds (at most `small_max` points) into batches
    for the persistent batched kernel, double-buffered on two streams: a
    batch launches as soon as a batch slot is free, so requests that arrive
    while others run join the next batch (continuous batching);
  * gathers admitted large clouds the same way into batches for resident
    large-cloud slots, each batch hulled together level by level (one launch
    sequence per merge level for all its clouds), a batch taking requests
    while their aligned rank blocks fit the slot's rank space;
  * polls completion events, copies results back, resolves futures and
    returns their bytes to the budget.
All device buffers (plans, staging rings) are allocated once at start and
stay resident.  The GPU work is done by a backend object; `CudaBackend`
drives the C ABI, and tests substitute a fake.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

ERR_BUDGET = 6


class ServeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(msg)
        self.code = code


def footprint(n: int) -> int:
    """Device bytes a request holds while in flight (its input and output rows)."""
    return 12 * n + 12 * max(2 * n - 4, 1)


def rank_block(n: int) -> int:
    """Ranks a cloud takes in a large-cloud batch: its aligned block, the
    smallest power of two >= n."""
    return 1 << max(0, int(n) - 1).bit_length()


@dataclass
class Request:
    points: np.ndarray
    arrival: float
    future: Future
    rid: int
    done: float = 0.0

    @property
    def n(self) -> int:
        return int(self.points.shape[0])


@dataclass
class Stats:
    latencies: list = field(default_factory=list)
    completed: int = 0
    rejected: int = 0
    batches: int = 0
    large: int = 0
    max_inflight_bytes: int = 0
    t_first: float = 0.0
    t_last: float = 0.0

    def summary(self) -> dict:
        lat = np.array(self.latencies) * 1e3 if self.latencies else np.zeros(1)
        span = max(self.t_last - self.t_first, 1e-9)
        return {"completed": self.completed, "rejected": self.rejected, "batches": self.batches,
                "large_runs": self.large, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                "hulls_per_s": self.completed / span, "max_inflight_bytes": self.max_inflight_bytes}


class CudaBackend:
    """GPU work through the C ABI: double-buffered batch slots for small
    clouds (the one-CTA batch kernel) and for large clouds (hulled together,
    level by level), each slot with its own plan, stream and resident
    device and pinned host buffers."""

    def __init__(self, small_max: int = 4096, batch_points: int = 1 << 21, batch_clouds: int = 8192,
                 large_slots: int = 2, large_max: int = 1 << 18, large_rank_space: int = 1 << 21,
                 large_clouds: int = 1024, device: str = "cuda", tuned: bool = True):
        import torch

        from paper_1205_1171_gb300 import hull3d

        self.torch, self.H = torch, hull3d
        self.small_max, self.batch_points, self.batch_clouds = small_max, batch_points, batch_clouds
        self.large_max, self.large_rank_space, self.large_clouds = large_max, large_rank_space, large_clouds
        if rank_block(large_max) > large_rank_space:
            raise ValueError("the largest request must fit a large slot's rank space")
        dev = torch.device(device)

        def plan(max_n, clouds, kind):  # the autotuner's knobs for this kind of work, if any
            if tuned:
                return hull3d.Hull3D.tuned(max_n, max_clouds=clouds, kind=kind)
            return hull3d.Hull3D(max_n, max_clouds=clouds)

        def slot(max_n, points, clouds, kind):
            return {"plan": plan(max_n, clouds, kind),
                    "stream": torch.cuda.Stream(dev),
                    "xyz": torch.empty((points, 3), dtype=torch.int32, device=dev),
                    "faces": torch.empty((2 * points, 3), dtype=torch.int32, device=dev),
                    "nf": torch.zeros(clouds, dtype=torch.int64, device=dev),
                    "st": torch.zeros(clouds, dtype=torch.int32, device=dev),
                    "h_xyz": torch.empty((points, 3), dtype=torch.int32).pin_memory(),
                    "h_faces": torch.empty((2 * points, 3), dtype=torch.int32).pin_memory(),
                    "h_nf": torch.zeros(clouds, dtype=torch.int64).pin_memory(),
                    "h_st": torch.zeros(clouds, dtype=torch.int32).pin_memory(),
                    "busy": None}

        self.batch_slots = [slot(small_max, batch_points, batch_clouds, "batch") for _ in range(2)]
        # a large batch holds at most large_rank_space points (their blocks fill that many ranks)
        self.large_slots = [slot(large_rank_space, large_rank_space, large_clouds, "multi") for _ in range(large_slots)]
        self.knobs = {"batch": getattr(self.batch_slots[0]["plan"], "tuned_knobs", {}),
                      "multi": getattr(self.large_slots[0]["plan"], "tuned_knobs", {}) if self.large_slots else {}}

    def resident_bytes(self) -> int:
        b = 0
        for s in self.batch_slots + self.large_slots:
            b += s["plan"].scratch_bytes + s["xyz"].numel() * 4 + s["faces"].numel() * 4
        return b

    def _launch(self, slot, reqs: list):
        torch = self.torch
        sizes = np.array([r.n for r in reqs], np.int64)
        off = np.zeros(len(reqs) + 1, np.int64)
        off[1:] = np.cumsum(sizes)
        caps = np.where(sizes >= 3, 2 * sizes - 4, 0)
        foff = np.zeros(len(reqs) + 1, np.int64)
        foff[1:] = np.cumsum(caps)
        h = slot["h_xyz"].numpy()
        for r, o in zip(reqs, off[:-1]):
            h[o: o + r.n] = r.points
        N = int(off[-1])
        with torch.cuda.stream(slot["stream"]):
            slot["xyz"][:N].copy_(slot["h_xyz"][:N], non_blocking=True)
            slot["plan"].batch_async(slot["xyz"], off, slot["faces"], foff, slot["nf"], slot["st"], slot["stream"])
            # results to pinned host memory on the same stream: completion
            # then needs no device call from the scheduler thread
            F = int(foff[-1])
            if F:
                slot["h_faces"][:F].copy_(slot["faces"][:F], non_blocking=True)
            B = len(reqs)
            slot["h_nf"][:B].copy_(slot["nf"][:B], non_blocking=True)
            slot["h_st"][:B].copy_(slot["st"][:B], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(slot["stream"])
        slot["busy"] = (ev, reqs, foff)

    # -- large clouds -------------------------------------------------------
    def free_large(self):
        return [s for s in self.large_slots if s["busy"] is None]

    def launch_large(self, slot, reqs: list):
        self._launch(slot, reqs)

    # -- small clouds ---------------------------------------------------------
    def free_batch(self):
        return [s for s in self.batch_slots if s["busy"] is None]

    def launch_batch(self, slot, reqs: list):
        self._launch(slot, reqs)

    # -- completion -----------------------------------------------------------
    def poll(self):
        """Completed work as (request, faces or exception) pairs; frees the slots."""
        out = []
        for slot in self.batch_slots + self.large_slots:
            if slot["busy"] is not None and slot["busy"][0].query():
                _, reqs, foff = slot["busy"]
                B = len(reqs)
                nf = slot["h_nf"][:B].numpy()
                st = slot["h_st"][:B].numpy()
                hf = slot["h_faces"].numpy()
                for b, r in enumerate(reqs):
                    if st[b]:
                        out.append((r, self.H.Hull3DError(int(st[b]), "serve")))
                    else:
                        out.append((r, hf[foff[b]: foff[b] + nf[b]].copy()))
                slot["busy"] = None
        return out

    def idle(self) -> bool:
        return all(s["busy"] is None for s in self.batch_slots + self.large_slots)


class HullServer:
    def __init__(self, backend=None, budget_bytes: int = 8 << 30, small_max: int = 4096, max_batch_clouds: int = 8192,
                 max_batch_points: int = 1 << 21):
        self.backend = backend if backend is not None else CudaBackend(small_max, max_batch_points,
                                                                      max_batch_clouds)
        self.small_max = small_max
        self.max_batch_clouds = max_batch_clouds
        self.max_batch_points = max_batch_points
        self.resident = self.backend.resident_bytes()
        if self.resident > budget_bytes:
            raise ServeError(ERR_BUDGET, "resident buffers exceed the memory budget")
        self.budget = budget_bytes
        self.inflight = 0
        self.stats = Stats()
        self._incoming = collections.deque()
        self._small = collections.deque()
        self._large = collections.deque()
        self._cv = threading.Condition()
        self._stop = False
        self._next_id = 0
        self._thread = threading.Thread(target=self._run, name="hull-server", daemon=True)
        self._thread.start()

    # -- API --------------------------------------------------------------
    def submit(self, points) -> Future:
        pts = np.ascontiguousarray(points, dtype=np.int32)
        if pts.ndim != 2 or pts.shape[1] != 3:
            raise ValueError("points must be (n, 3)")
        fut: Future = Future()
        with self._cv:
            req = Request(pts, time.perf_counter(), fut, self._next_id)
            self._next_id += 1
            self._incoming.append(req)
            self._cv.notify()
        return fut

    def close(self, timeout: float = 60.0):
        with self._cv:
            self._stop = True
            self._cv.notify()
        self._thread.join(timeout)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- scheduler ---------------------------------------------------------
    def _admit(self):
        with self._cv:
            while self._incoming:
                r = self._incoming.popleft()
                if self.stats.t_first == 0.0:
                    self.stats.t_first = r.arrival
                if footprint(r.n) > self.budget - self.resident or r.n > getattr(self.backend, "large_max", 1 << 62):
                    self.stats.rejected += 1
                    r.future.set_exception(ServeError(ERR_BUDGET, "request above the memory budget"))
                    continue
                (self._small if r.n <= self.small_max else self._large).append(r)

    def _complete(self):
        for req, res in self.backend.poll():
            self.inflight -= footprint(req.n)
            req.done = time.perf_counter()
            self.stats.t_last = req.done
            if isinstance(res, Exception):
                req.future.set_exception(res)
            else:
                self.stats.completed += 1
                self.stats.latencies.append(req.done - req.arrival)
                req.future.set_result(res)

    def _fits(self, n: int) -> bool:
        return self.inflight + footprint(n) <= self.budget - self.resident

    def _dispatch(self):
        # large clouds: a free large slot takes everything pending, in arrival
        # order, while memory allows and their rank blocks fit its rank space
        space_cap = getattr(self.backend, "large_rank_space", 1 << 62)
        count_cap = getattr(self.backend, "large_clouds", 1 << 30)
        for slot in self.backend.free_large():
            batch, space = [], 0
            while (self._large and len(batch) < count_cap and space + rank_block(self._large[0].n) <= space_cap
                   and self._fits(self._large[0].n)):
                r = self._large.popleft()
                self.inflight += footprint(r.n)
                space += rank_block(r.n)
                batch.append(r)
            if not batch:
                break
            self.backend.launch_large(slot, batch)
            self.stats.large += 1
        # small clouds: a free batch slot takes everything pending that fits
        free = self.backend.free_batch()
        if free and self._small:
            batch, pts = [], 0
            while (self._small and len(batch) < self.max_batch_clouds and pts + self._small[0].n <= self.max_batch_points
                   and self._fits(self._small[0].n)):
                r = self._small.popleft()
                self.inflight += footprint(r.n)
                pts += r.n
                batch.append(r)
            if batch:
                self.backend.launch_batch(free[0], batch)
                self.stats.batches += 1
        self.stats.max_inflight_bytes = max(self.stats.max_inflight_bytes, self.inflight)

    def _run(self):
        while True:
            self._admit()
            self._complete()
            self._dispatch()
            with self._cv:
                if self._stop and not self._incoming and not self._small and not self._large and self.backend.idle():
                    break
                if not self._incoming and self.backend.idle() and not self._small and not self._large:
                    self._cv.wait(0.01)
            if not self.backend.idle():
                time.sleep(20e-6)


def poisson_arrivals(rate: float, duration: float, rng: np.random.Generator) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    gaps = rng.exponential(1.0 / rate, size=int(rate * duration * 1.5) + 16)
    t = np.cumsum(gaps)
    return t[t < duration]


def request_pool(count: int, seed: int, lo_exp: float = 6.0, hi_exp: float = 18.0):
    """A pool of distinct clouds, sizes round(2^U(lo, hi)), mixed distributions;
    requests sample from it (independent work, shared point sets)."""
    from paper_1205_1171_gb300 import inputs

    rng = np.random.default_rng(seed)
    sizes = inputs.batch_sizes(count, lo_exp, hi_exp, rng)
    kinds = rng.integers(0, len(inputs.DISTS), size=count)
    return [inputs.cloud_seeded(inputs.DISTS[k], int(n), seed * 7919 + i) for i, (n, k) in
            enumerate(zip(sizes, kinds))]


def replay(server_submit, arrivals: np.ndarray, pool: list, picks):
    """Submits pool[picks[i]] at arrival time arrivals[i] (open loop); returns
    the futures.  picks may be a numpy Generator, which then draws them."""
    futs = []
    if isinstance(picks, np.random.Generator):
        picks = picks.integers(0, len(pool), size=len(arrivals))
    t0 = time.perf_counter()
    for t, k in zip(arrivals, picks):
        while True:
            dt = t0 + t - time.perf_counter()
            if dt <= 0:
                break
            time.sleep(min(dt, 0.001))
        futs.append(server_submit(pool[k]))
    return futs
