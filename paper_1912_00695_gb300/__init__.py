"""GB300 (sm_103a) library for the explicit time step of the 3D acoustic
isotropic wave equation with absorbing-layer damping and point-source
injection (arXiv 1912.00695, Sec. 2.1 Eq. 1 and Listing 2).

The compute path is the C-ABI shared library built from ``csrc/`` (declared in
include/fd_acoustic.h); this package only marshals arguments into it through
ctypes (:mod:`._abi`, same names as the C functions) and offers :class:`Shot`,
a small owner object around one solver handle. PyTorch, where used, provides
device memory and streams only.
"""
from __future__ import annotations

import numpy as np

from ._abi import (fd_batch_add, fd_batch_create, fd_batch_destroy, fd_batch_forward, fd_batch_forward_flow,  # noqa: F401
                   fd_batch_get_config, fd_batch_schedule,
                   fd_batch_inject, fd_batch_read, fd_batch_read_device, fd_batch_remove, fd_batch_reset,
                   fd_batch_set_stream, fd_batch_shot_status, fd_batch_shot_step, fd_batch_size,
                   fd_batch_synchronize, fd_shot_device_bytes)
from ._abi import (FD_BOUNDARY_PERIODIC, FD_BOUNDARY_ZERO, FD_EFULL, FD_EINVAL, FD_ENOMEM, FD_ENONFINITE, FD_ENOTSUP, FD_EUNSTABLE,  # noqa: F401
                   FD_ERANGE, FD_ESTATE, FD_ETIMEOUT, FD_FORM_EXPANDED, FD_FORM_FACTORED,
                   FD_KERNEL_AUTO, FD_KERNEL_NAIVE, FD_KERNEL_STREAM, FD_KERNEL_TMA, FD_OK, FD_STORAGE_BF16,
                   FD_STORAGE_F16, FD_STORAGE_F32, FdError, fd_acoustic_create,
                   fd_acoustic_create_ex, fd_clear_sources, fd_default_damping, fd_destroy, fd_dt_max, fd_fd_weights,
                   fd_forward, fd_forward_flow, fd_forward_two_step, fd_get_config, fd_get_dims, fd_get_schedule, fd_get_step, fd_inject, fd_inject_at,
                   fd_load_state, fd_read_traces, fd_set_receivers, fd_fwi_gradient,
                   fd_kernel_launches, fd_selftest_waits, fd_last_error, fd_last_forward_ms, fd_options, fd_options_default,
                   fd_read_wavefield, fd_read_wavefield_device, fd_reset, fd_set_model,
                   fd_set_model_device, fd_set_stream, fd_status, fd_synchronize, fd_version)

STORAGE = {"f32": FD_STORAGE_F32, "bf16": FD_STORAGE_BF16, "f16": FD_STORAGE_F16}
FORMS = {"factored": FD_FORM_FACTORED, "expanded": FD_FORM_EXPANDED}
KERNELS = {"auto": FD_KERNEL_AUTO, "stream": FD_KERNEL_STREAM, "naive": FD_KERNEL_NAIVE,
           "tma": FD_KERNEL_TMA}
BOUNDARIES = {"zero": FD_BOUNDARY_ZERO, "periodic": FD_BOUNDARY_PERIODIC}


def options(storage="f32", form="factored", kernel="auto", tile_z=0, tile_y=0, x_block=0,
            check_finite=True, boundary="zero", rows=0) -> fd_options:
    o = fd_options_default()
    o.storage = STORAGE[storage]
    o.form = FORMS[form]
    o.kernel = KERNELS[kernel]
    o.tile_z = int(tile_z)
    o.tile_y = int(tile_y)
    o.x_block = int(x_block)
    o.check_finite = int(bool(check_finite))
    o.boundary = BOUNDARIES[boundary]
    o.rows = int(rows)
    return o


class PendingRead:
    """A shot's wavefield on its way to pinned host memory (stream-ordered after
    the launches queued before it); ``ready()`` polls, ``result()`` waits."""

    def __init__(self, host, event, keep):
        self._host = host
        self._event = event
        self._keep = keep  # device staging, alive until the copy ran

    def ready(self) -> bool:
        return self._event.query()

    def result(self) -> np.ndarray:
        self._event.synchronize()
        self._keep = None
        return self._host.numpy()


class Batch:
    """A batch of uneven shots advanced together (owns its device state).

    With ``stream`` (a ``torch.cuda.Stream``) every launch, upload and read of
    the batch is queued on that stream; ``read_async`` and ``mark`` then give
    stream-ordered completion handles, so a host loop can keep several chunks
    queued per batch without synchronising."""

    def __init__(self, space_order, h, storage="f32", form="factored", tile_z=0, tile_y=0,
                 x_block=0, stream=None, kernel="auto"):
        # kernel="tma" pins one launch per step; "auto" lets an FP32 batch time the
        # persistent launch against it
        self.space_order = int(space_order)
        self.h = float(h)
        self.handle = fd_batch_create(space_order, h, options(storage=storage, form=form,
                                                              tile_z=tile_z, tile_y=tile_y,
                                                              x_block=x_block, kernel=kernel))
        self.shapes = {}
        self.stream = stream
        if stream is not None:
            fd_batch_set_stream(self.handle, stream.cuda_stream)

    def add(self, interior, nbl, dt, m, eta=None) -> int:
        nx, ny, nz = interior
        slot = fd_batch_add(self.handle, nx, ny, nz, nbl, dt, m, eta)
        self.shapes[slot] = tuple(n + 2 * nbl for n in interior)
        return slot

    def inject(self, slot, ix, iy, iz, wavelet):
        fd_batch_inject(self.handle, slot, ix, iy, iz, wavelet)

    def remove(self, slot):
        fd_batch_remove(self.handle, slot)
        self.shapes.pop(slot, None)

    def forward(self, nt):
        fd_batch_forward(self.handle, nt)

    def forward_flow(self, nt):
        """nt steps of every shot in one persistent launch (FP32): same bits as forward."""
        fd_batch_forward_flow(self.handle, nt)

    def schedule(self):
        """1 when forward runs one persistent launch per call (autotuned), else 0."""
        return fd_batch_schedule(self.handle)

    def wavefield(self, slot, level=0, out=None) -> np.ndarray:
        if out is None:
            out = np.empty(self.shapes[slot], dtype=np.float32)
        return fd_batch_read(self.handle, slot, out, level)

    def read_async(self, slot, level=0) -> PendingRead:
        """Start copying the shot's wavefield (dense FP32) to pinned host memory
        without waiting; the shot may be removed right after this call."""
        import torch
        if self.stream is None:
            raise RuntimeError("read_async needs a batch created with a torch stream")
        shape = self.shapes[slot]
        with torch.cuda.stream(self.stream):
            dev = torch.empty(shape, dtype=torch.float32, device="cuda")
            fd_batch_read_device(self.handle, slot, dev.data_ptr(), level)
            host = torch.empty(shape, dtype=torch.float32, pin_memory=True)
            host.copy_(dev, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        dev.record_stream(self.stream)
        return PendingRead(host, ev, dev)

    def mark(self):
        """An event recorded after the work queued so far (``ready()``/``wait()``)."""
        import torch
        if self.stream is None:
            raise RuntimeError("mark needs a batch created with a torch stream")
        ev = torch.cuda.Event()
        ev.record(self.stream)
        return _Mark(ev)

    def step(self, slot) -> int:
        return fd_batch_shot_step(self.handle, slot)

    def status(self, slot) -> int:
        return fd_batch_shot_status(self.handle, slot)

    def size(self):
        return fd_batch_size(self.handle)

    def config(self):
        """(tile_z, tile_y, x-chunk policy, tuned) of the batch's launches."""
        return fd_batch_get_config(self.handle)

    def reset(self):
        fd_batch_reset(self.handle)

    def set_stream(self, stream_ptr):
        fd_batch_set_stream(self.handle, stream_ptr)

    def synchronize(self):
        fd_batch_synchronize(self.handle)

    def close(self):
        if self.handle:
            fd_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Mark:
    def __init__(self, ev):
        self._ev = ev

    def ready(self) -> bool:
        return self._ev.query()

    def wait(self):
        self._ev.synchronize()


class Shot:
    """One single-shot solver handle (owns its device state until close())."""

    def __init__(self, interior, space_order, h, dt, nbl, **opts):
        nx, ny, nz = interior
        self.interior = (int(nx), int(ny), int(nz))
        self.nbl = int(nbl)
        self.space_order = int(space_order)
        self.h = float(h)
        self.dt = float(dt)
        self.handle = fd_acoustic_create_ex(nx, ny, nz, space_order, h, dt, nbl, options(**opts))
        self.shape = fd_get_dims(self.handle)

    def set_model(self, m, eta=None):
        fd_set_model(self.handle, m, eta)

    def set_model_device(self, d_m, d_eta=None):
        fd_set_model_device(self.handle, d_m, d_eta)

    def inject(self, ix, iy, iz, wavelet):
        fd_inject(self.handle, ix, iy, iz, wavelet)

    def forward(self, nt):
        fd_forward(self.handle, nt)

    def forward_two_step(self, nt):
        """nt steps, two per launch (FP32 factored, space order 2 or 4)."""
        fd_forward_two_step(self.handle, nt)

    def forward_flow(self, nt):
        """nt steps in one persistent launch (FP32, TMA kernel): same bits as forward."""
        fd_forward_flow(self.handle, nt)

    def inject_at(self, x, y, z, wavelet):
        """Off-grid source at continuous interior coordinates (trilinear spreading)."""
        fd_inject_at(self.handle, x, y, z, wavelet)

    def set_receivers(self, xyz, nt_max):
        """Receivers at continuous interior coordinates xyz (n, 3), recording up
        to nt_max samples from the current step on."""
        p = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
        fd_set_receivers(self.handle, p, nt_max)
        self._rec = (p.shape[0], int(nt_max))

    def traces(self) -> np.ndarray:
        """Recorded traces, shape (n, recorded samples)."""
        n, nt_max = self._rec
        out = np.empty(n * nt_max, dtype=np.float32)
        done = fd_read_traces(self.handle, out)
        return out.reshape(n, nt_max)[:, :done]

    def fwi_gradient(self, receivers, d_obs, segment=0):
        """(dJ/dm over the domain, synthetic traces [nrec, nt], misfit J) of this
        shot against observed traces d_obs [nrec, nt] at the receivers;
        segment > 0 checkpoints every `segment` steps."""
        d_obs = np.asarray(d_obs, dtype=np.float32)
        grad = np.empty(self.shape, dtype=np.float32)
        syn = np.empty(d_obs.shape, dtype=np.float32)
        J = fd_fwi_gradient(self.handle, receivers, d_obs, grad, syn, segment=segment)
        return grad, syn, J

    def wavefield(self, level=0, out=None) -> np.ndarray:
        if out is None:
            out = np.empty(self.shape, dtype=np.float32)
        return fd_read_wavefield(self.handle, out, level)

    def read_device(self, d_out, level=0):
        fd_read_wavefield_device(self.handle, d_out, level)

    def set_stream(self, stream_ptr):
        fd_set_stream(self.handle, stream_ptr)

    def synchronize(self):
        fd_synchronize(self.handle)

    def reset(self):
        fd_reset(self.handle)

    def load_state(self, u, u_prev, step):
        fd_load_state(self.handle, u, u_prev, step)

    @property
    def step(self) -> int:
        return fd_get_step(self.handle)

    @property
    def config(self):
        return fd_get_config(self.handle)

    @property
    def schedule(self):
        """(rows per thread, schedule 0 per-step / 1 flow / 2 two-step, flow x-chunk)."""
        return fd_get_schedule(self.handle)

    def last_forward_ms(self) -> float:
        return fd_last_forward_ms(self.handle)

    def close(self):
        if self.handle:
            fd_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
