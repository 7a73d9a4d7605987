"""Continuous-batching shot server on top of the batch C-ABI.

Requests (a shot: interior size, space order, storage, model, source,
number of steps) arrive over time. Each (space order, storage) class owns one
batch (``fd_batch_*``) on its own CUDA stream, so the classes' launches overlap
on the GPU. A request is admitted as soon as it has arrived and its device
state (``fd_shot_device_bytes``) fits in the memory budget; it then joins its
class batch between two chunks of steps, its wavefields stay resident in HBM,
and when it has taken its steps its final wavefield is copied out, its slot is
freed and waiting requests are admitted. A shot's result does not depend on
which other shots shared its launches (the batch kernel's per-point arithmetic
is that of the single-shot kernel).

The loop never waits for the GPU while it has work to queue: each class keeps
up to ``depth`` chunks queued on its stream; a shot that finishes within a
chunk is read out (stream-ordered copy to pinned host memory) and removed
right behind that chunk, so the next chunk can be queued at once. Model
uploads and checks of newly admitted shots run on the shots' own streams.
The host only blocks when every class has ``depth`` chunks in flight and
nothing has completed. The scheduling loop is host logic (this module); every
step of every shot runs in the library's kernels.
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
    m: np.ndarray | None      # squared slowness over the computational domain (float32)
    source: tuple             # interior node
    wavelet: np.ndarray       # float32 samples
    nt: int
    result: np.ndarray | None = field(default=None, repr=False)
    admitted: float = -1.0
    completed: float = -1.0
    visible: float = 0.0      # when the server could first see it (latency is measured from here)
    # the model may instead come from a callable, asked for it at admission (a
    # client that streams its model in, or a generator bounded in host memory)
    m_fn: object = field(default=None, repr=False)

    def model(self) -> np.ndarray:
        return self.m if self.m is not None or self.m_fn is None else self.m_fn()

    @property
    def points(self) -> int:
        return int(np.prod([n + 2 * self.nbl for n in self.interior]))

    @property
    def device_bytes(self) -> int:
        nx, ny, nz = self.interior
        return fd_shot_device_bytes(nx, ny, nz, self.nbl, _STORAGE_ID[self.storage])


def _default_batch(k, h, storage):
    import torch
    # per-step launches pinned: a server's batches change as shots arrive and leave,
    # and the schedule probes would block the loop once per batch
    return Batch(k, h, storage=storage, stream=torch.cuda.Stream(), kernel="tma")


class Server:
    """Admits requests by memory budget and advances every resident shot in
    chunks of at most `chunk` steps (a chunk never overshoots a shot's end),
    keeping up to `depth` chunks queued per class.

    The batch factory (and the per-request byte count) are injectable so that
    the scheduling policy can be exercised without a GPU; a batch offers
    add/inject/forward/remove/close, ``read_async(slot)`` (an object with
    ``ready()`` and ``result()``) and ``mark()`` (an object with ``ready()``
    and ``wait()``)."""

    def __init__(self, h: float, budget_bytes: int, chunk: int = 50, keep_results: bool = True,
                 batch_factory=None, bytes_fn=None, depth: int = 2):
        self.h = float(h)
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.depth = max(1, int(depth))
        self.keep_results = keep_results
        self.classes: dict[tuple, Batch] = {}
        self.batch_factory = batch_factory or _default_batch
        self.bytes_fn = bytes_fn or (lambda req: req.device_bytes)
        self.used = 0
        self.peak_used = 0
        self.active: dict[int, list] = {}       # rid -> [class key, slot, steps not yet queued, request]
        self.inflight: dict[tuple, deque] = {}  # class key -> marks of queued chunks
        self.reads: list[tuple] = []            # (request, pending read, bytes)
        # kernels queued: a step per chunk step, the model set-up of an admission
        # (validation, default damping, factored coefficients, scale reset) and the
        # read-out's unpack
        self.launches = 0

    def _batch(self, key) -> Batch:
        b = self.classes.get(key)
        if b is None:
            k, storage = key
            b = self.batch_factory(k, self.h, storage)
            self.classes[key] = b
            self.inflight[key] = deque()
        return b

    def admit(self, req: Request, now: float) -> bool:
        need = self.bytes_fn(req)
        if self.used + need > self.budget:
            return False
        key = (req.space_order, req.storage)
        b = self._batch(key)
        slot = b.add(req.interior, req.nbl, req.dt, req.model())
        b.inject(slot, *req.source, req.wavelet)
        self.used += need
        self.launches += 4
        self.peak_used = max(self.peak_used, self.used)
        req.admitted = now
        self.active[req.rid] = [key, slot, req.nt, req]
        return True

    def _queue_chunk(self, key) -> bool:
        """Queue one chunk on class `key` (False if it has nothing to run)."""
        entries = [e for e in self.active.values() if e[0] == key]
        if not entries:
            return False
        b = self.classes[key]
        n = min(self.chunk, min(e[2] for e in entries))
        b.forward(n)
        self.launches += n
        for e in entries:
            e[2] -= n
            if e[2] == 0:
                _, slot, _, req = e
                # stream-ordered behind this chunk: the copy-out, then the slot's release
                self.reads.append((req, b.read_async(slot), self.bytes_fn(req)))
                self.launches += 1
                b.remove(slot)
                del self.active[req.rid]
        self.inflight[key].append(b.mark())
        return True

    def _progress(self, now_fn) -> list[Request]:
        """Retire completed chunk marks and reads; returns the finished requests."""
        for q in self.inflight.values():
            while q and q[0].ready():
                q.popleft()
        done, keep = [], []
        for req, pending, nbytes in self.reads:
            if pending.ready():
                out = pending.result()
                req.result = out if self.keep_results else None
                req.completed = now_fn()
                self.used -= nbytes
                done.append(req)
            else:
                keep.append((req, pending, nbytes))
        self.reads = keep
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
        while pending or waiting or self.active or self.reads:
            now = now_fn()
            while pending and (not realtime or pending[0].arrival <= now):
                r = pending.popleft()
                r.visible = r.arrival if realtime else 0.0
                waiting.append(r)
            while waiting and self.admit(waiting[0], now):
                waiting.popleft()
            if waiting and not self.active and not self.reads:
                raise RuntimeError(f"request {waiting[0].rid} needs {self.bytes_fn(waiting[0])} bytes, "
                                   f"more than the budget {self.budget}")
            queued = False
            for key in list(self.classes):
                if len(self.inflight[key]) < self.depth:
                    queued |= self._queue_chunk(key)
            done = self._progress(now_fn)
            finished += done
            if queued or done:
                continue
            # nothing to queue and nothing completed: wait a little (for a chunk, a
            # read-out or the next arrival)
            if self.reads or any(self.inflight.values()):
                time.sleep(0.0002)
            elif pending:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
        makespan = now_fn()
        out = summarize(finished, makespan)
        out["gpu_launches"] = self.launches
        return out

    def close(self):
        for b in self.classes.values():
            b.close()
        self.classes.clear()
        self.inflight.clear()


def summarize(finished: list[Request], makespan: float) -> dict:
    lat = np.array([r.completed - r.visible for r in finished]) if finished else np.zeros(1)
    pts = sum(r.points * r.nt for r in finished)
    return {"requests": len(finished), "makespan_s": makespan,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "gpts": pts / max(makespan, 1e-9) / 1e9,
            "point_steps": pts}
