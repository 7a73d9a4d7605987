"""One shot split into slabs along x, with an r-plane halo exchange per step.

The paper's OPS backend partitions a block across distributed-memory
processes (Sec. 3, Devito-OPS integration, item (vii): ``ops_partition``) and
Devito exchanges halos between the subdomains, overlapping the exchange with
computation (Sec. 5). Here a shot's planes along x (the slowest axis) are cut
into contiguous slabs; each slab is a library handle (``fd_slab_create``) that
owns its planes plus r = k/2 ghost planes per neighbour. Every time step runs,
per slab:

1. the boundary part (``fd_slab_step(FD_SLAB_BOUNDARY)``): the own planes
   within r of a neighbour, which are the planes the neighbours need;
2. the exchange: each slab's first / last r new planes go to the lower /
   upper neighbour's ghost planes of the same level;
3. the interior part, concurrently with the exchange;

and the next step's boundary part starts only after the ghost planes it reads
have arrived. Every point then gets the same arithmetic on the same inputs as
in the undivided shot, so the slabs' planes equal ``fd_forward`` bit for bit.

This module is host logic only: the partition, the exchange plan and the
ordering. The steps run in the library's kernels; the exchange is a device
copy (``fd_slab_exchange``, a peer copy between devices) when one process
drives every slab (:class:`SlabGroup`), or point-to-point messages of
``torch.distributed`` when each rank owns one slab (:class:`HaloDriver`, with
:class:`GpuSlab` as the rank's slab: NCCL between GPUs).
"""
from __future__ import annotations

import contextlib
from dataclasses import dataclass

import numpy as np

from ._abi import (FD_SLAB_BOUNDARY, FD_SLAB_INTERIOR, fd_default_damping, fd_destroy, fd_get_dims,
                   fd_get_step, fd_inject, fd_read_wavefield, fd_reset, fd_set_model, fd_set_stream,
                   fd_slab_create, fd_slab_exchange, fd_slab_exchange_ptrs, fd_slab_info, fd_slab_step,
                   fd_synchronize)


def partition(n_planes: int, parts: int, radius: int) -> list[tuple[int, int]]:
    """Split planes [0, n_planes) into `parts` contiguous ranges as even as
    possible (the first n_planes % parts get one plane more). Every range must
    hold at least `radius` planes, so that a slab's ghost planes all come from
    its immediate neighbour."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    if parts == 1:
        return [(0, n_planes)]  # one slab has no neighbour to take ghosts from
    base, extra = divmod(n_planes, parts)
    if base < max(radius, 1):
        raise ValueError(f"{n_planes} planes cannot be split into {parts} slabs of at least {radius} planes")
    out, x = [], 0
    for i in range(parts):
        n = base + (1 if i < extra else 0)
        out.append((x, x + n))
        x += n
    return out


@dataclass(frozen=True)
class Transfer:
    """One halo message of a step: r planes of slab `src` to slab `dst`.
    direction "up": src's last r own planes -> dst's low ghost planes (dst is
    the next slab); "down": src's first r own planes -> dst's high ghost planes."""
    src: int
    dst: int
    direction: str


def exchange_plan(ranges: list[tuple[int, int]]) -> list[Transfer]:
    """The transfers of every step, for slabs with the given plane ranges
    (contiguous and ordered along x)."""
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        if a1 != b0:
            raise ValueError("slab ranges must be contiguous and ordered")
    plan = []
    for i in range(len(ranges) - 1):
        plan.append(Transfer(i, i + 1, "up"))
        plan.append(Transfer(i + 1, i, "down"))
    return plan


def ghost_planes(ranges, index: int, radius: int, n_planes: int) -> tuple[int, int]:
    """(ghosts below, ghosts above) of slab `index`: radius where it has a neighbour."""
    x0, x1 = ranges[index]
    return (radius if x0 > 0 else 0), (radius if x1 < n_planes else 0)


def slab_window(ranges, index: int, radius: int, n_planes: int) -> tuple[int, int]:
    """Domain planes [w0, w1) that slab `index` holds: its own planes and its ghosts."""
    x0, x1 = ranges[index]
    lo, hi = ghost_planes(ranges, index, radius, n_planes)
    return x0 - lo, x1 + hi


def _options(**opts):
    from . import options
    return options(**opts)


class SlabGroup:
    """A shot split into `parts` slabs along x, every slab driven from this
    process (on one device, or on `devices[i]` each: the exchange is then a
    peer copy). Same calls as a shot: set_model, inject, forward, wavefield.

    Each slab computes on its own stream and sends on a second one, so that
    the exchange of a step overlaps its interior part."""

    def __init__(self, interior, space_order, h, dt, nbl, parts, devices=None, **opts):
        import torch
        self.interior = tuple(int(n) for n in interior)
        self.nbl = int(nbl)
        self.k = int(space_order)
        self.r = self.k // 2
        self.h = float(h)
        self.shape = tuple(n + 2 * self.nbl for n in self.interior)
        self.ranges = partition(self.shape[0], parts, self.r)
        self.plan = exchange_plan(self.ranges)
        self.devices = list(devices) if devices is not None else [torch.cuda.current_device()] * parts
        if len(self.devices) != parts:
            raise ValueError("one device per slab")
        opt = _options(**opts)
        self.handles, self.compute, self.send, self.windows = [], [], [], []
        try:
            for i, (x0, x1) in enumerate(self.ranges):
                with torch.cuda.device(self.devices[i]):
                    hd = fd_slab_create(*self.interior, self.k, self.h, dt, self.nbl, x0, x1, opt)
                    self.handles.append(hd)
                    cs, xs = torch.cuda.Stream(), torch.cuda.Stream()
                    fd_set_stream(hd, cs.cuda_stream)
                    self.compute.append(cs)
                    self.send.append(xs)
                    self.windows.append(slab_window(self.ranges, i, self.r, self.shape[0]))
                    assert fd_slab_info(hd)[:2] == (x0, x1)
        except Exception:
            self.close()
            raise
        self._sent = [None] * parts  # event after each slab's sends of the last step

    def set_model(self, m, eta=None):
        """Global host arrays over the whole domain; eta None: the default profile
        of the whole model (the library's host helper)."""
        m = np.ascontiguousarray(m, dtype=np.float32)
        if eta is None:
            eta = fd_default_damping(m, self.nbl, self.h)
        eta = np.ascontiguousarray(eta, dtype=np.float32)
        for hd, (w0, w1) in zip(self.handles, self.windows):
            fd_set_model(hd, m[w0:w1], eta[w0:w1])

    def inject(self, ix, iy, iz, wavelet):
        """A point source at interior node (ix, iy, iz); the slab owning its plane takes it."""
        for hd in self.handles:
            fd_inject(hd, ix, iy, iz, wavelet)

    def reset(self):
        for hd in self.handles:
            fd_reset(hd)
        self._sent = [None] * len(self.handles)

    def _step(self):
        import torch
        n = len(self.handles)
        # the ghost planes this step reads arrived with the last step's transfers, and
        # the buffer it writes was last read by this slab's own sends of the step before
        for i in range(n):
            for t in self.plan:
                if t.dst == i and self._sent[t.src] is not None:
                    self.compute[i].wait_event(self._sent[t.src])
            if self._sent[i] is not None:
                self.compute[i].wait_event(self._sent[i])
        done_b = []
        for i, hd in enumerate(self.handles):
            fd_slab_step(hd, FD_SLAB_BOUNDARY)
            ev = torch.cuda.Event()
            ev.record(self.compute[i])
            done_b.append(ev)
        for t in self.plan:
            xs = self.send[t.src]
            xs.wait_event(done_b[t.src])
            fd_slab_exchange(self.handles[t.src], self.handles[t.dst], 1, xs.cuda_stream)
        for i, hd in enumerate(self.handles):
            ev = torch.cuda.Event()
            ev.record(self.send[i])
            self._sent[i] = ev
            fd_slab_step(hd, FD_SLAB_INTERIOR)

    def forward(self, nt: int):
        for _ in range(int(nt)):
            self._step()

    @property
    def step(self) -> int:
        return fd_get_step(self.handles[0])

    def synchronize(self):
        for i, hd in enumerate(self.handles):
            fd_synchronize(hd)
            self.send[i].synchronize()

    def wavefield(self, level: int = 0) -> np.ndarray:
        """The whole domain's level (0: u^n, 1: u^{n-1}) assembled from the slabs' own planes."""
        self.synchronize()
        out = np.empty(self.shape, dtype=np.float32)
        for hd, (x0, x1), (w0, _) in zip(self.handles, self.ranges, self.windows):
            buf = np.empty(fd_get_dims(hd), dtype=np.float32)
            fd_read_wavefield(hd, buf, level)
            out[x0:x1] = buf[x0 - w0:x1 - w0]
        return out

    def close(self):
        for hd in getattr(self, "handles", []):
            if hd:
                fd_destroy(hd)
        self.handles = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class _DeviceView:
    """A device buffer described by __cuda_array_interface__ (so that
    torch.as_tensor views it without a copy)."""

    def __init__(self, ptr: int, shape, device: int):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4", "data": (int(ptr), False),
                                         "version": 3, "strides": None}
        self.device = device


class GpuSlab:
    """This rank's slab as a :class:`HaloDriver` stepper: a library slab on the
    current CUDA device whose kernels run on a torch stream of its own; the
    driver makes that stream current around each step, so that
    torch.distributed's point-to-point operations (and host staging copies)
    order with the slab's kernels."""

    def __init__(self, interior, space_order, h, dt, nbl, ranges, index, **opts):
        import torch
        self.interior_dims = tuple(int(n) for n in interior)
        self.nbl, self.k, self.r, self.h = int(nbl), int(space_order), int(space_order) // 2, float(h)
        self.shape = tuple(n + 2 * self.nbl for n in self.interior_dims)
        self.ranges, self.index = ranges, index
        x0, x1 = ranges[index]
        self.window = slab_window(ranges, index, self.r, self.shape[0])
        self.handle = fd_slab_create(*self.interior_dims, self.k, self.h, dt, self.nbl, x0, x1, _options(**opts))
        self.device = torch.cuda.current_device()
        # a stream object of its own: the library reads a null stream handle as "the
        # handle's own stream", which would not order with torch's default stream
        self.stream = torch.cuda.Stream()
        fd_set_stream(self.handle, self.stream.cuda_stream)
        self.dims = fd_get_dims(self.handle)

    def stream_context(self):
        import torch
        return torch.cuda.stream(self.stream)

    def set_model(self, m, eta):
        w0, w1 = self.window
        fd_set_model(self.handle, np.ascontiguousarray(m[w0:w1], dtype=np.float32),
                     np.ascontiguousarray(eta[w0:w1], dtype=np.float32))

    def inject(self, ix, iy, iz, wavelet):
        fd_inject(self.handle, ix, iy, iz, wavelet)

    def boundary(self):
        fd_slab_step(self.handle, FD_SLAB_BOUNDARY)

    def interior(self):
        fd_slab_step(self.handle, FD_SLAB_INTERIOR)

    def views(self, level: int):
        """(send_lo, send_hi, recv_lo, recv_hi) as torch tensors viewing the slab's
        planes at `level` (None where there is no neighbour)."""
        import torch
        *ptrs, nbytes = fd_slab_exchange_ptrs(self.handle, level)
        planes = nbytes // (4 * self.r) if self.r else 0
        shape = (self.r, planes)
        return tuple(None if p is None else
                     torch.as_tensor(_DeviceView(p, shape, self.device), device=f"cuda:{self.device}")
                     for p in ptrs)

    def own_planes(self, level: int = 0) -> np.ndarray:
        self.stream.synchronize()
        buf = np.empty(self.dims, dtype=np.float32)
        fd_read_wavefield(self.handle, buf, level)
        x0, x1 = self.ranges[self.index]
        return buf[x0 - self.window[0]:x1 - self.window[0]]

    def close(self):
        if self.handle:
            fd_destroy(self.handle)
            self.handle = None


class HaloDriver:
    """The per-rank schedule of a slab-decomposed shot over a torch.distributed
    process group (rank i owns slab i): per step, the boundary part, the halo
    sends and receives posted (isend/irecv to the ranks i - 1 and i + 1), the
    interior part while they are in flight, and the receives completed before
    the next step, all with the stepper's stream current (stream_context(), if
    it has one). `stepper` provides boundary(), interior() and views(level)
    (send_lo, send_hi, recv_lo, recv_hi: tensors the transport accepts, or
    None at the domain's ends); `stage` (optional) maps a view to the tensor
    actually sent or received and back (host staging for a CPU-only
    transport)."""

    def __init__(self, stepper, group=None, stage=None):
        import torch.distributed as dist
        self.dist = dist
        self.stepper = stepper
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.stage = stage
        self.steps = 0

    def step(self):
        ctx = getattr(self.stepper, "stream_context", None)
        with (ctx() if ctx else contextlib.nullcontext()):
            self._step()

    def _step(self):
        d, st = self.dist, self.stepper
        st.boundary()
        s_lo, s_hi, r_lo, r_hi = st.views(1)  # the level this step writes
        ops, back = [], []
        for peer, send, recv in ((self.rank - 1, s_lo, r_lo), (self.rank + 1, s_hi, r_hi)):
            if 0 <= peer < self.world and send is not None and recv is not None:
                if self.stage is not None:
                    send_t, recv_t = self.stage.out(send), self.stage.buffer(recv)
                    back.append((recv_t, recv))
                else:
                    send_t, recv_t = send, recv
                ops.append(d.P2POp(d.isend, send_t, peer, self.group))
                ops.append(d.P2POp(d.irecv, recv_t, peer, self.group))
        reqs = d.batch_isend_irecv(ops) if ops else []
        st.interior()
        for q in reqs:
            q.wait()
        for staged, view in back:
            self.stage.into(staged, view)
        self.steps += 1

    def forward(self, nt: int):
        for _ in range(int(nt)):
            self.step()


class HostStage:
    """Host staging for a transport that carries CPU tensors only (gloo):
    device views are copied to host tensors before sending and received
    tensors copied back."""

    def out(self, view):
        return view.cpu()

    def buffer(self, view):
        import torch
        return torch.empty(view.shape, dtype=view.dtype)

    def into(self, staged, view):
        view.copy_(staged)
