"""ctypes binding of the C-ABI in include/fd_acoustic.h (argument marshalling only).

Every function keeps the C name. Arrays are passed as raw pointers: host
arrays as C-contiguous float32 numpy arrays, device arrays as the integer
address of a CUDA buffer (for example ``tensor.data_ptr()``). Errors come back
as FdError carrying the status code and ``fd_last_error()``. Loading fails
loudly when the compiled library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfdgb.so")

FD_OK = 0
FD_EINVAL = -1
FD_ERANGE = -2
FD_EUNSTABLE = -3
FD_ENOMEM = -4
FD_ECUDA = -5
FD_ENONFINITE = -6
FD_ETIMEOUT = -7
FD_ESTATE = -8
FD_ENOTSUP = -9
FD_EFULL = -10

FD_STORAGE_F32, FD_STORAGE_BF16, FD_STORAGE_F16 = 0, 1, 2
FD_FORM_FACTORED, FD_FORM_EXPANDED = 0, 1
FD_KERNEL_AUTO, FD_KERNEL_STREAM, FD_KERNEL_NAIVE, FD_KERNEL_TMA = 0, 1, 2, 3
FD_BOUNDARY_ZERO, FD_BOUNDARY_PERIODIC = 0, 1
FD_SLAB_BOUNDARY, FD_SLAB_INTERIOR, FD_SLAB_ALL = 1, 2, 3

ERROR_NAMES = {0: "FD_OK", -1: "FD_EINVAL", -2: "FD_ERANGE", -3: "FD_EUNSTABLE", -4: "FD_ENOMEM",
               -5: "FD_ECUDA", -6: "FD_ENONFINITE", -7: "FD_ETIMEOUT", -8: "FD_ESTATE",
               -9: "FD_ENOTSUP", -10: "FD_EFULL"}


class FdError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        self.code = code
        super().__init__(f"{func}: {ERROR_NAMES.get(code, code)}: {msg}")


class fd_options(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("form", ctypes.c_int), ("kernel", ctypes.c_int),
                ("tile_z", ctypes.c_int), ("tile_y", ctypes.c_int), ("x_block", ctypes.c_int),
                ("check_finite", ctypes.c_int), ("boundary", ctypes.c_int), ("rows", ctypes.c_int)]


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_fp = ctypes.POINTER(ctypes.c_float)
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)

# name -> (restype, argtypes); int-returning calls are checked
_SIGNATURES = {
    "fd_options_default": (None, [ctypes.POINTER(fd_options)]),
    "fd_acoustic_create": (_i, [_i, _i, _i, _i, _d, _d, _i, ctypes.POINTER(_vp)]),
    "fd_acoustic_create_ex": (_i, [_i, _i, _i, _i, _d, _d, _i, ctypes.POINTER(fd_options),
                                   ctypes.POINTER(_vp)]),
    "fd_set_model": (_i, [_vp, _vp, _vp]),
    "fd_set_model_device": (_i, [_vp, _vp, _vp]),
    "fd_inject": (_i, [_vp, _i, _i, _i, _vp, _i]),
    "fd_clear_sources": (_i, [_vp]),
    "fd_inject_at": (_i, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _vp, _i]),
    "fd_set_receivers": (_i, [_vp, _i, _vp, _i]),
    "fd_read_traces": (_i, [_vp, _vp, _ip]),
    "fd_fwi_gradient": (_i, [_vp, _i, _vp, _vp, _i, _vp, _vp, ctypes.POINTER(ctypes.c_double)]),
    "fd_fwi_gradient_checkpointed": (_i, [_vp, _i, _vp, _vp, _i, _i, _vp, _vp, ctypes.POINTER(ctypes.c_double)]),
    "fd_forward": (_i, [_vp, _i]),
    "fd_forward_two_step": (_i, [_vp, _i]),
    "fd_forward_flow": (_i, [_vp, _i]),
    "fd_read_wavefield": (_i, [_vp, _vp, _i]),
    "fd_read_wavefield_device": (_i, [_vp, _vp, _i]),
    "fd_set_stream": (_i, [_vp, _vp]),
    "fd_synchronize": (_i, [_vp]),
    "fd_status": (_i, [_vp]),
    "fd_reset": (_i, [_vp]),
    "fd_load_state": (_i, [_vp, _vp, _vp, ctypes.c_longlong]),
    "fd_get_step": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "fd_get_dims": (_i, [_vp, _ip, _ip, _ip]),
    "fd_get_config": (_i, [_vp, _ip, _ip, _ip, _ip]),
    "fd_get_schedule": (_i, [_vp, _ip, _ip, _ip]),
    "fd_last_forward_ms": (_i, [_vp, _fp]),
    "fd_kernel_launches": (_i, [ctypes.POINTER(ctypes.c_longlong)]),
    "fd_selftest_waits": (_i, [ctypes.POINTER(ctypes.c_uint), _dp, _dp]),
    "fd_destroy": (_i, [_vp]),
    "fd_dt_max": (_i, [_i, _d, _d, _dp]),
    "fd_fd_weights": (_i, [_i, _dp]),
    "fd_default_damping": (_i, [_i, _i, _i, _i, _d, _vp, _vp]),
    "fd_forward_noalloc": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _d, _d, _i, _vp, _vp, _i,
                               ctypes.c_longlong, _i, _vp, _fp]),
    "fd_shot_device_bytes": (_i, [_i, _i, _i, _i, _i, ctypes.POINTER(ctypes.c_longlong)]),
    "fd_slab_create": (_i, [_i, _i, _i, _i, _d, _d, _i, _i, _i, ctypes.POINTER(fd_options),
                            ctypes.POINTER(_vp)]),
    "fd_slab_info": (_i, [_vp, _ip, _ip, _ip, _ip]),
    "fd_slab_step": (_i, [_vp, _i]),
    "fd_slab_exchange_ptrs": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                   ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_size_t)]),
    "fd_slab_exchange": (_i, [_vp, _vp, _i, _vp]),
    "fd_batch_create": (_i, [_i, _d, ctypes.POINTER(fd_options), ctypes.POINTER(_vp)]),
    "fd_batch_add": (_i, [_vp, _i, _i, _i, _i, _d, _vp, _vp, _ip]),
    "fd_batch_inject": (_i, [_vp, _i, _i, _i, _i, _vp, _i]),
    "fd_batch_remove": (_i, [_vp, _i]),
    "fd_batch_forward": (_i, [_vp, _i]),
    "fd_batch_forward_flow": (_i, [_vp, _i]),
    "fd_batch_schedule": (_i, [_vp, _ip]),
    "fd_batch_read": (_i, [_vp, _i, _vp, _i]),
    "fd_batch_read_device": (_i, [_vp, _i, _vp, _i]),
    "fd_batch_shot_step": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_longlong)]),
    "fd_batch_shot_status": (_i, [_vp, _i]),
    "fd_batch_size": (_i, [_vp, _ip, _ip]),
    "fd_batch_get_config": (_i, [_vp, _ip, _ip, _ip, _ip]),
    "fd_batch_reset": (_i, [_vp]),
    "fd_batch_set_stream": (_i, [_vp, _vp]),
    "fd_batch_synchronize": (_i, [_vp]),
    "fd_batch_destroy": (_i, [_vp]),
    "fd_last_error": (ctypes.c_char_p, []),
    "fd_version": (ctypes.c_char_p, []),
}


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"CUDA library not built ({LIB_PATH} missing); run "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            h = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                f = getattr(h, name)
                f.restype = res
                f.argtypes = args
            _lib = h
        return _lib


def exported_symbols() -> list[str]:
    return list(_SIGNATURES)


def _check(rc: int, func: str):
    if rc != FD_OK:
        raise FdError(rc, func, lib().fd_last_error().decode())


def _host_f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    """Raw address of a numpy array, an integer address, or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


# ---- thin wrappers with the C names -------------------------------------------

def fd_options_default() -> fd_options:
    o = fd_options()
    lib().fd_options_default(ctypes.byref(o))
    return o


def fd_acoustic_create(nx, ny, nz, space_order, h, dt, nbl) -> int:
    out = _vp()
    _check(lib().fd_acoustic_create(nx, ny, nz, space_order, h, dt, nbl, ctypes.byref(out)),
           "fd_acoustic_create")
    return out.value


def fd_acoustic_create_ex(nx, ny, nz, space_order, h, dt, nbl, opt: fd_options | None) -> int:
    out = _vp()
    _check(lib().fd_acoustic_create_ex(nx, ny, nz, space_order, h, dt, nbl,
                                       ctypes.byref(opt) if opt is not None else None,
                                       ctypes.byref(out)), "fd_acoustic_create_ex")
    return out.value


def fd_set_model(hd, m, eta=None):
    m = _host_f32(m)
    eta = None if eta is None else _host_f32(eta)
    _check(lib().fd_set_model(hd, _ptr(m), _ptr(eta)), "fd_set_model")


def fd_set_model_device(hd, d_m, d_eta=None):
    _check(lib().fd_set_model_device(hd, _ptr(d_m), _ptr(d_eta)), "fd_set_model_device")


def fd_inject(hd, ix, iy, iz, wavelet):
    w = _host_f32(wavelet)
    _check(lib().fd_inject(hd, ix, iy, iz, _ptr(w), int(w.size)), "fd_inject")


def fd_clear_sources(hd):
    _check(lib().fd_clear_sources(hd), "fd_clear_sources")


def fd_inject_at(hd, x, y, z, wavelet):
    w = _host_f32(wavelet)
    _check(lib().fd_inject_at(hd, float(x), float(y), float(z), _ptr(w), int(w.size)), "fd_inject_at")


def fd_set_receivers(hd, xyz, nt_max):
    """xyz: (n, 3) continuous interior coordinates (copied); n = 0 removes them."""
    p = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
    n = int(p.shape[0])
    _check(lib().fd_set_receivers(hd, n, _ptr(p) if n else None, int(nt_max)), "fd_set_receivers")


def fd_fwi_gradient(hd, rec_xyz, d_obs, grad_out: np.ndarray, syn_out=None, segment: int = 0) -> float:
    """Fill grad_out (float32, domain shape) with dJ/dm; optionally syn_out
    (float32 [nrec, nt]); returns the misfit J. segment > 0: checkpointed
    (fd_fwi_gradient_checkpointed)."""
    p = np.ascontiguousarray(np.asarray(rec_xyz, dtype=np.float64).reshape(-1, 3))
    obs = np.ascontiguousarray(np.asarray(d_obs, dtype=np.float32))
    nrec, nt = obs.shape
    assert p.shape[0] == nrec
    assert grad_out.dtype == np.float32 and grad_out.flags.c_contiguous
    if syn_out is not None:
        assert syn_out.dtype == np.float32 and syn_out.flags.c_contiguous and syn_out.shape == obs.shape
    j = ctypes.c_double()
    if segment:
        _check(lib().fd_fwi_gradient_checkpointed(hd, nrec, _ptr(p), _ptr(obs), nt, int(segment), _ptr(grad_out),
                                                  _ptr(syn_out), ctypes.byref(j)), "fd_fwi_gradient_checkpointed")
    else:
        _check(lib().fd_fwi_gradient(hd, nrec, _ptr(p), _ptr(obs), nt, _ptr(grad_out), _ptr(syn_out),
                                     ctypes.byref(j)), "fd_fwi_gradient")
    return j.value


def fd_read_traces(hd, out: np.ndarray) -> int:
    """Fill out (float32, n * nt_max, receiver-major); returns the recorded samples."""
    assert out.dtype == np.float32 and out.flags.c_contiguous
    rec = ctypes.c_int()
    _check(lib().fd_read_traces(hd, _ptr(out), ctypes.byref(rec)), "fd_read_traces")
    return rec.value


def fd_forward(hd, nt):
    _check(lib().fd_forward(hd, nt), "fd_forward")


def fd_forward_two_step(hd, nt):
    _check(lib().fd_forward_two_step(hd, nt), "fd_forward_two_step")


def fd_forward_flow(hd, nt):
    _check(lib().fd_forward_flow(hd, nt), "fd_forward_flow")


def fd_read_wavefield(hd, out: np.ndarray, level: int = 0):
    assert out.dtype == np.float32 and out.flags.c_contiguous
    _check(lib().fd_read_wavefield(hd, _ptr(out), level), "fd_read_wavefield")
    return out


def fd_read_wavefield_device(hd, d_out, level: int = 0):
    _check(lib().fd_read_wavefield_device(hd, _ptr(d_out), level), "fd_read_wavefield_device")


def fd_set_stream(hd, stream_ptr: int | None):
    _check(lib().fd_set_stream(hd, stream_ptr), "fd_set_stream")


def fd_synchronize(hd):
    _check(lib().fd_synchronize(hd), "fd_synchronize")


def fd_status(hd) -> int:
    return lib().fd_status(hd)


def fd_reset(hd):
    _check(lib().fd_reset(hd), "fd_reset")


def fd_load_state(hd, u, u_prev, step: int):
    u = _host_f32(u)
    u_prev = _host_f32(u_prev)
    _check(lib().fd_load_state(hd, _ptr(u), _ptr(u_prev), int(step)), "fd_load_state")


def fd_get_step(hd) -> int:
    v = ctypes.c_longlong()
    _check(lib().fd_get_step(hd, ctypes.byref(v)), "fd_get_step")
    return v.value


def fd_get_dims(hd):
    a, b, c = _i(), _i(), _i()
    _check(lib().fd_get_dims(hd, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "fd_get_dims")
    return a.value, b.value, c.value


def fd_get_config(hd):
    """(kernel, tile_z, tile_y, x_block) of the handle's step kernel."""
    v = [_i() for _ in range(4)]
    _check(lib().fd_get_config(hd, *[ctypes.byref(x) for x in v]), "fd_get_config")
    return tuple(x.value for x in v)


def fd_get_schedule(hd):
    """(rows per thread, schedule: 0 per-step launches / 1 flow / 2 two steps per
    launch, flow x-chunk) that fd_forward runs for the handle."""
    v = [_i() for _ in range(3)]
    _check(lib().fd_get_schedule(hd, *[ctypes.byref(x) for x in v]), "fd_get_schedule")
    return tuple(x.value for x in v)


def fd_last_forward_ms(hd) -> float:
    v = ctypes.c_float()
    _check(lib().fd_last_forward_ms(hd, ctypes.byref(v)), "fd_last_forward_ms")
    return v.value


def fd_selftest_waits():
    """(status bits, seconds of the mbarrier wait, seconds of the flag wait): both
    device-side waits must give up (status 3) after their limits."""
    st = ctypes.c_uint()
    t1, t2 = ctypes.c_double(), ctypes.c_double()
    _check(lib().fd_selftest_waits(ctypes.byref(st), ctypes.byref(t1), ctypes.byref(t2)), "fd_selftest_waits")
    return st.value, t1.value, t2.value


def fd_kernel_launches() -> int:
    """Kernel launches of this library executed or queued since it was loaded."""
    v = ctypes.c_longlong()
    _check(lib().fd_kernel_launches(ctypes.byref(v)), "fd_kernel_launches")
    return v.value


def fd_destroy(hd):
    _check(lib().fd_destroy(hd), "fd_destroy")


def fd_dt_max(space_order, h, vmax) -> float:
    v = _d()
    _check(lib().fd_dt_max(space_order, h, vmax, ctypes.byref(v)), "fd_dt_max")
    return v.value


def fd_fd_weights(space_order) -> np.ndarray:
    out = np.zeros(space_order // 2 + 1 if space_order >= 2 else 1, dtype=np.float64)
    _check(lib().fd_fd_weights(space_order, out.ctypes.data_as(_dp)), "fd_fd_weights")
    return out


def fd_default_damping(m, nbl, h) -> np.ndarray:
    m = _host_f32(m)
    eta = np.empty_like(m)
    nx, ny, nz = m.shape
    _check(lib().fd_default_damping(nx, ny, nz, nbl, h, _ptr(m), _ptr(eta)), "fd_default_damping")
    return eta


def fd_forward_noalloc(d_u, d_u_prev, d_m, d_eta, dims, space_order, h, dt, sources=(),
                       d_wavelet=None, ld=0, step0=0, nt=1, stream=None, want_amax=True):
    """Allocation-free stepping on caller-owned device buffers (see the header).
    sources: domain nodes (x, y, z), at most 4. Returns max |u| when want_amax."""
    nx, ny, nz = dims
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32).reshape(-1))
    amax = ctypes.c_float(0.0)
    rc = lib().fd_forward_noalloc(_ptr(d_u), _ptr(d_u_prev), _ptr(d_m), _ptr(d_eta), nx, ny, nz,
                                  space_order, h, dt, len(sources),
                                  src.ctypes.data if len(sources) else None, _ptr(d_wavelet),
                                  int(ld), int(step0), int(nt), stream,
                                  ctypes.byref(amax) if want_amax else None)
    _check(rc, "fd_forward_noalloc")
    return amax.value if want_amax else None


def fd_shot_device_bytes(nx, ny, nz, nbl, storage) -> int:
    v = ctypes.c_longlong()
    _check(lib().fd_shot_device_bytes(nx, ny, nz, nbl, storage, ctypes.byref(v)),
           "fd_shot_device_bytes")
    return v.value


def fd_slab_create(nx, ny, nz, space_order, h, dt, nbl, x0, x1, opt: fd_options | None = None) -> int:
    out = _vp()
    _check(lib().fd_slab_create(nx, ny, nz, space_order, h, dt, nbl, x0, x1,
                                ctypes.byref(opt) if opt is not None else None, ctypes.byref(out)),
           "fd_slab_create")
    return out.value


def fd_slab_info(hd):
    """(x0, x1, ghost_lo, ghost_hi): own planes [x0, x1) in domain indices, ghost counts."""
    v = [_i() for _ in range(4)]
    _check(lib().fd_slab_info(hd, *[ctypes.byref(x) for x in v]), "fd_slab_info")
    return tuple(x.value for x in v)


def fd_slab_step(hd, part: int = FD_SLAB_ALL):
    _check(lib().fd_slab_step(hd, part), "fd_slab_step")


def fd_slab_exchange_ptrs(hd, level: int):
    """(send_lo, send_hi, recv_lo, recv_hi, bytes): device addresses (None where
    the slab has no neighbour) in the buffer of `level`."""
    v = [_vp() for _ in range(4)]
    n = ctypes.c_size_t()
    _check(lib().fd_slab_exchange_ptrs(hd, level, *[ctypes.byref(x) for x in v], ctypes.byref(n)),
           "fd_slab_exchange_ptrs")
    return tuple(x.value for x in v) + (n.value,)


def fd_slab_exchange(src, dst, level: int, stream_ptr: int | None):
    _check(lib().fd_slab_exchange(src, dst, level, stream_ptr), "fd_slab_exchange")


def fd_batch_create(space_order, h, opt: fd_options | None = None) -> int:
    out = _vp()
    _check(lib().fd_batch_create(space_order, h, ctypes.byref(opt) if opt is not None else None,
                                 ctypes.byref(out)), "fd_batch_create")
    return out.value


def fd_batch_add(b, nx, ny, nz, nbl, dt, m, eta=None) -> int:
    m = _host_f32(m)
    eta = None if eta is None else _host_f32(eta)
    slot = _i()
    _check(lib().fd_batch_add(b, nx, ny, nz, nbl, dt, _ptr(m), _ptr(eta), ctypes.byref(slot)),
           "fd_batch_add")
    return slot.value


def fd_batch_inject(b, slot, ix, iy, iz, wavelet):
    w = _host_f32(wavelet)
    _check(lib().fd_batch_inject(b, slot, ix, iy, iz, _ptr(w), int(w.size)), "fd_batch_inject")


def fd_batch_remove(b, slot):
    _check(lib().fd_batch_remove(b, slot), "fd_batch_remove")


def fd_batch_forward(b, nt):
    _check(lib().fd_batch_forward(b, nt), "fd_batch_forward")


def fd_batch_forward_flow(b, nt):
    _check(lib().fd_batch_forward_flow(b, nt), "fd_batch_forward_flow")


def fd_batch_schedule(b):
    """1 when fd_batch_forward runs one persistent launch per forward, else 0."""
    v = ctypes.c_int(0)
    _check(lib().fd_batch_schedule(b, ctypes.byref(v)), "fd_batch_schedule")
    return v.value


def fd_batch_read(b, slot, out: np.ndarray, level: int = 0):
    assert out.dtype == np.float32 and out.flags.c_contiguous
    _check(lib().fd_batch_read(b, slot, _ptr(out), level), "fd_batch_read")
    return out


def fd_batch_read_device(b, slot, d_out, level: int = 0):
    _check(lib().fd_batch_read_device(b, slot, _ptr(d_out), level), "fd_batch_read_device")


def fd_batch_shot_step(b, slot) -> int:
    v = ctypes.c_longlong()
    _check(lib().fd_batch_shot_step(b, slot, ctypes.byref(v)), "fd_batch_shot_step")
    return v.value


def fd_batch_shot_status(b, slot) -> int:
    return lib().fd_batch_shot_status(b, slot)


def fd_batch_size(b):
    a, w = _i(), _i()
    _check(lib().fd_batch_size(b, ctypes.byref(a), ctypes.byref(w)), "fd_batch_size")
    return a.value, w.value


def fd_batch_get_config(b):
    """(tile_z, tile_y, x-chunk policy, tuned) of the batch."""
    v = [_i() for _ in range(4)]
    _check(lib().fd_batch_get_config(b, *[ctypes.byref(x) for x in v]), "fd_batch_get_config")
    return tuple(x.value for x in v)


def fd_batch_reset(b):
    _check(lib().fd_batch_reset(b), "fd_batch_reset")


def fd_batch_set_stream(b, stream_ptr):
    _check(lib().fd_batch_set_stream(b, stream_ptr), "fd_batch_set_stream")


def fd_batch_synchronize(b):
    _check(lib().fd_batch_synchronize(b), "fd_batch_synchronize")


def fd_batch_destroy(b):
    _check(lib().fd_batch_destroy(b), "fd_batch_destroy")


def fd_last_error() -> str:
    return lib().fd_last_error().decode()


def fd_version() -> str:
    return lib().fd_version().decode()
