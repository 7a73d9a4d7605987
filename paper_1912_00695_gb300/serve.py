"""Continuous-batching shot server on top of the batch C-ABI.

Requests (a shot: interior size, space order, storage, model, source,
number of steps) arrive over time. Each (space order, storage) class owns one
batch (``fd_batch_*``) on its own CUDA stream, so the classes' launches overlap
on the GPU. A request is admitted as soon as it has arrived and its device
state (``fd_shot_device_bytes``) fits in the memory budget; it then joins its
class batch between two chunks of steps, its wavefields stay resident in HBM,
and when it has taken its steps its final wavefield is read back, its slot and
memory are freed and waiting requests are admitted. A shot's result does not
depend on which other shots shared its launches (the batch kernel's per-point
arithmetic is that of the single-shot kernel).

The scheduling loop is host logic (this module); every step of every shot runs
in the library's kernels.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import Batch, FD_STORAGE_BF16, FD_STORAGE_F16, FD_STORAGE_F32, fd_shot_device_bytes

_STORAGE_ID = {"f32": FD_STORAGE_F32, "bf16": FD_STORAGE_BF16, "f16": FD_STORAGE_F16}


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the start of the run
    interior: tuple
    nbl: int
    space_order: int
    storage: str
    dt: float
    m: np.ndarray             # squared slowness over the computational domain (float32)
    source: tuple             # interior node
    wavelet: np.ndarray       # float32 samples
    nt: int
    result: np.ndarray | None = field(default=None, repr=False)
    admitted: float = -1.0
    completed: float = -1.0
    visible: float = 0.0      # when the server could first see it (latency is measured from here)

    @property
    def points(self) -> int:
        return int(np.prod([n + 2 * self.nbl for n in self.interior]))

    @property
    def device_bytes(self) -> int:
        nx, ny, nz = self.interior
        return fd_shot_device_bytes(nx, ny, nz, self.nbl, _STORAGE_ID[self.storage])


class Server:
    """Admits requests by memory budget and advances every resident shot in
    chunks of at most `chunk` steps (a chunk never overshoots a shot's end)."""

    def __init__(self, h: float, budget_bytes: int, chunk: int = 50, keep_results: bool = True,
                 batch_factory=None, bytes_fn=None):
        self.h = float(h)
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.keep_results = keep_results
        self.classes: dict[tuple, Batch] = {}
        # the batch constructor and the per-request byte count are injectable so
        # that the scheduling policy can be exercised without a GPU
        self.batch_factory = batch_factory or (lambda k, h, storage: Batch(k, h, storage=storage))
        self.bytes_fn = bytes_fn or (lambda req: req.device_bytes)
        self.used = 0
        self.peak_used = 0
        self.active: dict[int, tuple] = {}  # rid -> (class key, slot, remaining, request)
        self.log: list[tuple] = []

    def _batch(self, key) -> Batch:
        b = self.classes.get(key)
        if b is None:
            k, storage = key
            b = self.batch_factory(k, self.h, storage)
            self.classes[key] = b
        return b

    def admit(self, req: Request, now: float) -> bool:
        need = self.bytes_fn(req)
        if self.used + need > self.budget:
            return False
        key = (req.space_order, req.storage)
        b = self._batch(key)
        slot = b.add(req.interior, req.nbl, req.dt, req.m)
        b.inject(slot, *req.source, req.wavelet)
        self.used += need
        self.peak_used = max(self.peak_used, self.used)
        req.admitted = now
        self.active[req.rid] = (key, slot, req.nt, req)
        return True

    def step(self, now_fn) -> list[Request]:
        """One chunk on every class with resident shots; returns the requests
        that completed."""
        if not self.active:
            return []
        by_class: dict[tuple, list] = {}
        for rid, (key, slot, remaining, req) in self.active.items():
            by_class.setdefault(key, []).append((rid, slot, remaining, req))
        advanced = {}
        for key, entries in by_class.items():
            n = min(self.chunk, min(e[2] for e in entries))
            self.classes[key].forward(n)  # asynchronous; classes overlap on their streams
            advanced[key] = n
        for key in by_class:
            self.classes[key].synchronize()
        done = []
        for key, entries in by_class.items():
            n = advanced[key]
            b = self.classes[key]
            for rid, slot, remaining, req in entries:
                left = remaining - n
                if left > 0:
                    self.active[rid] = (key, slot, left, req)
                    continue
                out = b.wavefield(slot)
                req.result = out if self.keep_results else None
                b.remove(slot)
                self.used -= self.bytes_fn(req)
                req.completed = now_fn()
                del self.active[rid]
                done.append(req)
        return done

    def run(self, requests: list[Request], realtime: bool = True) -> dict:
        """Serve a trace. With realtime, requests become visible at their arrival
        times on the wall clock; otherwise all are visible at once (offline) and
        latencies count from the start of the run."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting: deque[Request] = deque()
        finished: list[Request] = []
        t0 = time.perf_counter()
        now_fn = (lambda: time.perf_counter() - t0)
        while pending or waiting or self.active:
            now = now_fn()
            while pending and (not realtime or pending[0].arrival <= now):
                r = pending.popleft()
                r.visible = r.arrival if realtime else 0.0
                waiting.append(r)
            while waiting and self.admit(waiting[0], now):
                waiting.popleft()
            if waiting and not self.active:
                raise RuntimeError(f"request {waiting[0].rid} needs {self.bytes_fn(waiting[0])} bytes, "
                                   f"more than the budget {self.budget}")
            if not self.active:
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                continue
            finished += self.step(now_fn)
        makespan = now_fn()
        return summarize(finished, makespan)

    def close(self):
        for b in self.classes.values():
            b.close()
        self.classes.clear()


def summarize(finished: list[Request], makespan: float) -> dict:
    lat = np.array([r.completed - r.visible for r in finished]) if finished else np.zeros(1)
    pts = sum(r.points * r.nt for r in finished)
    return {"requests": len(finished), "makespan_s": makespan,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "gpts": pts / max(makespan, 1e-9) / 1e9,
            "point_steps": pts}
