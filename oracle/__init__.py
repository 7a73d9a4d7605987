"""FP64 CPU oracle for the damped, source-driven 3D acoustic leapfrog step.

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library never does,
and the two share no code (the only shared module is the seeded input
generator, which holds none of the method's arithmetic).

The arithmetic lives in ``fd_oracle.c`` (plain C, double precision, OpenMP
loops), compiled on first use with gcc into ``oracle/_build/``. This module
only marshals numpy arrays into it. What each function computes, and the paper
passage it follows (arXiv 1912.00695, Sec. 2.1 Eq. 1, Listing 1, Listing 2),
is stated in the C source beside the function.

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, invariants, Listing 2, a library interpolator or a dense brute
force, except the default
damping profile, whose formula is a convention the paper does not give
(parity unpinned as a formula; its invariants are tested).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfdoracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile fd_oracle.c into a shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_fd_weights.argtypes = [ctypes.c_int, _dp]
        lib.oracle_fd_weights.restype = ctypes.c_int
        lib.oracle_laplacian.argtypes = [_dp, _dp, ctypes.c_long, ctypes.c_long, ctypes.c_long,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_int]
        lib.oracle_laplacian.restype = ctypes.c_int
        lib.oracle_step.argtypes = [_dp, _dp, _dp, _dp, _dp, ctypes.c_long, ctypes.c_long,
                                    ctypes.c_long, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int]
        lib.oracle_step.restype = ctypes.c_int
        lib.oracle_forward.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_long, ctypes.c_long,
                                       ctypes.c_long, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, _ip, _ip, _ip,
                                       _dp, ctypes.c_long, ctypes.c_long, ctypes.c_long]
        lib.oracle_forward.restype = ctypes.c_int
        lib.oracle_energy.argtypes = [_dp, _dp, _dp, ctypes.c_long, ctypes.c_long, ctypes.c_long,
                                      ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.oracle_energy.restype = ctypes.c_double
        lib.oracle_dt_max.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        lib.oracle_dt_max.restype = ctypes.c_double
        lib.oracle_default_damping.argtypes = [_dp, _dp, ctypes.c_long, ctypes.c_long,
                                               ctypes.c_long, ctypes.c_int, ctypes.c_double]
        lib.oracle_default_damping.restype = ctypes.c_int
        _lp = ctypes.POINTER(ctypes.c_long)
        lib.oracle_trilinear.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_long, ctypes.c_long, ctypes.c_long, _lp, _dp]
        lib.oracle_trilinear.restype = ctypes.c_int
        lib.oracle_forward_offgrid.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_long, ctypes.c_long,
                                               ctypes.c_long, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                               ctypes.c_long, ctypes.c_int, _dp, _dp, ctypes.c_long,
                                               ctypes.c_long]
        lib.oracle_forward_offgrid.restype = ctypes.c_int
        lib.oracle_fwi_gradient.argtypes = [_dp, _dp, ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp,
                                            ctypes.c_long, ctypes.c_int, _dp, _dp, ctypes.c_long, _dp, _dp, _dp,
                                            _dp]
        lib.oracle_fwi_gradient.restype = ctypes.c_int
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def num_threads() -> int:
    """OpenMP threads the oracle runs on."""
    return int(_load().oracle_num_threads())


def fd_weights(space_order: int) -> np.ndarray:
    """c_0..c_r of the centred 2nd derivative of accuracy order k (closed form)."""
    r = space_order // 2
    c = np.zeros(max(r, 0) + 1, dtype=np.float64)
    if _load().oracle_fd_weights(int(space_order), _ptr(c)) != 0:
        raise ValueError(f"space_order must be even in [2, 24], got {space_order}")
    return c


def laplacian(u, space_order: int, h: float, periodic: bool = False) -> np.ndarray:
    u = _f64(u)
    out = np.empty_like(u)
    nx, ny, nz = u.shape
    rc = _load().oracle_laplacian(_ptr(u), _ptr(out), nx, ny, nz, int(space_order), float(h),
                                  int(periodic))
    if rc != 0:
        raise ValueError("bad arguments to oracle laplacian")
    return out


def step(u, u_prev, m, eta, space_order: int, h: float, dt: float,
         periodic: bool = False) -> np.ndarray:
    """u^{n+1} from u^n and u^{n-1} without sources (eta may be None)."""
    u, u_prev, m = _f64(u), _f64(u_prev), _f64(m)
    eta_a = None if eta is None else _f64(eta)
    out = np.empty_like(u)
    nx, ny, nz = u.shape
    rc = _load().oracle_step(_ptr(u), _ptr(u_prev), _ptr(out), _ptr(m),
                             None if eta_a is None else _ptr(eta_a), nx, ny, nz,
                             int(space_order), float(h), float(dt), int(periodic))
    if rc != 0:
        raise ValueError("bad arguments to oracle step")
    return out


def forward(m, eta, space_order: int, h: float, dt: float, nt: int, sources=(), wavelets=None,
            u0=None, u_prev0=None, step0: int = 0, periodic: bool = False, inplace: bool = False):
    """Advance nt steps; returns (u^{step0+nt}, u^{step0+nt-1}) as float64 arrays.

    sources: sequence of (x, y, z) domain nodes; wavelets: array (ns, ld) of
    source samples indexed by global step (zero beyond ld). inplace: advance
    the given u0 and u_prev0 (contiguous float64 arrays) in place instead of
    copies (marshalling only: the same arithmetic, no per-call copy of large
    fields).
    """
    m = _f64(m)
    shape = m.shape
    if inplace and u0 is not None and u_prev0 is not None:
        u, up = u0, u_prev0
        for a in (u, up):
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.shape != shape:
                raise ValueError("inplace forward needs contiguous float64 levels of the model's shape")
    else:
        u = np.zeros(shape) if u0 is None else _f64(u0).copy()
        up = np.zeros(shape) if u_prev0 is None else _f64(u_prev0).copy()
    eta_a = None if eta is None else _f64(eta)
    ns = len(sources)
    src = np.asarray(sources, dtype=np.int32).reshape(ns, 3)
    sx, sy, sz = (np.ascontiguousarray(src[:, i]) for i in range(3))
    if ns:
        w = _f64(np.asarray(wavelets).reshape(ns, -1))
        ld = w.shape[1]
    else:
        w = np.zeros((1, 1))
        ld = 0
    nx, ny, nz = shape
    rc = _load().oracle_forward(_ptr(u), _ptr(up), _ptr(m),
                                None if eta_a is None else _ptr(eta_a), nx, ny, nz,
                                int(space_order), float(h), float(dt), int(periodic), ns,
                                sx.ctypes.data_as(_ip), sy.ctypes.data_as(_ip),
                                sz.ctypes.data_as(_ip), _ptr(w), ld, int(step0), int(nt))
    if rc != 0:
        raise ValueError(f"oracle forward failed ({rc})")
    return u, up


def trilinear(point, shape):
    """The 8 nodes (8x3 int array) and weights of a continuous domain point."""
    nodes = np.zeros((8, 3), dtype=np.int64)
    w = np.zeros(8)
    rc = _load().oracle_trilinear(float(point[0]), float(point[1]), float(point[2]), *map(int, shape),
                                  nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _ptr(w))
    if rc != 0:
        raise ValueError(f"point {tuple(point)} outside a {tuple(shape)} domain")
    return nodes, w


def forward_offgrid(m, eta, space_order: int, h: float, dt: float, nt: int, sources=(),
                    wavelets=None, receivers=(), u0=None, u_prev0=None, step0: int = 0,
                    periodic: bool = False):
    """Advance nt steps with off-grid sources (continuous domain coordinates,
    trilinear spreading) and receivers (trilinear sampling of each new level).
    Returns (u^{step0+nt}, u^{step0+nt-1}, traces[nr, nt])."""
    m = _f64(m)
    shape = m.shape
    u = np.zeros(shape) if u0 is None else _f64(u0).copy()
    up = np.zeros(shape) if u_prev0 is None else _f64(u_prev0).copy()
    eta_a = None if eta is None else _f64(eta)
    ns, nr = len(sources), len(receivers)
    src = _f64(np.asarray(sources, dtype=np.float64).reshape(ns, 3)) if ns else np.zeros((1, 3))
    rec = _f64(np.asarray(receivers, dtype=np.float64).reshape(nr, 3)) if nr else np.zeros((1, 3))
    if ns:
        w = _f64(np.asarray(wavelets).reshape(ns, -1))
        ld = w.shape[1]
    else:
        w = np.zeros((1, 1))
        ld = 0
    traces = np.zeros((max(nr, 1), max(int(nt), 1)))
    nx, ny, nz = shape
    rc = _load().oracle_forward_offgrid(_ptr(u), _ptr(up), _ptr(m), None if eta_a is None else _ptr(eta_a),
                                        nx, ny, nz, int(space_order), float(h), float(dt), int(periodic),
                                        ns, _ptr(src), _ptr(w), ld, nr, _ptr(rec), _ptr(traces), int(step0),
                                        int(nt))
    if rc != 0:
        raise ValueError(f"oracle forward_offgrid failed ({rc})")
    return u, up, traces[:nr, :nt]


def fwi_gradient(m, eta, space_order: int, h: float, dt: float, nt: int, sources, wavelets, receivers,
                 d_obs, adjoint: bool = False):
    """Misfit J = 1/2 |d - d_obs|^2 of one shot (off-grid sources and receivers,
    traces d^n = R u^{n+1}) and its exact discrete gradient dJ/dm.
    Returns (grad, syn traces [nr, nt], J) and, with adjoint=True, also the
    adjoint of the source-to-traces map applied to d_obs, [ns, nt]."""
    m = _f64(m)
    nx, ny, nz = m.shape
    eta_a = None if eta is None else _f64(eta)
    ns, nr = len(sources), len(receivers)
    src = _f64(np.asarray(sources, dtype=np.float64).reshape(ns, 3)) if ns else np.zeros((1, 3))
    rec = _f64(np.asarray(receivers, dtype=np.float64).reshape(nr, 3))
    w = _f64(np.asarray(wavelets).reshape(ns, -1)) if ns else np.zeros((1, 1))
    ld = w.shape[1] if ns else 0
    obs = _f64(np.asarray(d_obs).reshape(nr, nt))
    grad = np.zeros(m.shape)
    syn = np.zeros((nr, nt))
    J = np.zeros(1)
    adj = np.zeros((max(ns, 1), nt)) if adjoint else None
    rc = _load().oracle_fwi_gradient(_ptr(m), None if eta_a is None else _ptr(eta_a), nx, ny, nz, int(space_order),
                                     float(h), float(dt), ns, _ptr(src), _ptr(w), ld, nr, _ptr(rec), _ptr(obs),
                                     int(nt), _ptr(grad), _ptr(syn), _ptr(J), None if adj is None else _ptr(adj))
    if rc != 0:
        raise ValueError(f"oracle fwi_gradient failed ({rc})")
    if adjoint:
        return grad, syn, float(J[0]), adj[:ns]
    return grad, syn, float(J[0])


def energy(u_new, u_old, m, space_order: int, h: float, dt: float,
           periodic: bool = False) -> float:
    """Discrete energy E^{n+1/2} between two consecutive levels."""
    u_new, u_old, m = _f64(u_new), _f64(u_old), _f64(m)
    nx, ny, nz = m.shape
    return float(_load().oracle_energy(_ptr(u_new), _ptr(u_old), _ptr(m), nx, ny, nz,
                                       int(space_order), float(h), float(dt), int(periodic)))


def dt_max(space_order: int, h: float, vmax: float) -> float:
    v = float(_load().oracle_dt_max(int(space_order), float(h), float(vmax)))
    if v < 0:
        raise ValueError("bad arguments to oracle dt_max")
    return v


def default_damping(m, nbl: int, h: float) -> np.ndarray:
    """The default absorbing-layer eta for model m (convention; see fd_oracle.c)."""
    m = _f64(m)
    out = np.empty_like(m)
    nx, ny, nz = m.shape
    if _load().oracle_default_damping(_ptr(out), _ptr(m), nx, ny, nz, int(nbl), float(h)) != 0:
        raise ValueError("bad arguments to oracle default_damping")
    return out
