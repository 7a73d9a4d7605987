"""CPU-side checks of the C-ABI library: it builds, loads, exports every symbol
include/fd_acoustic.h declares, and its host numerics (Fornberg weights,
stability limit, default damping profile) agree with the independent oracle.
No GPU compute is called here.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1912_00695_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def built_lib():
    from paper_1912_00695_gb300 import build
    build.build()
    return _abi.lib()


def _declared_functions():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(fd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(built_lib):
    declared = _declared_functions()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(built_lib, name), f"{name} declared but not exported"
    # and the binding covers every declared entry point
    assert set(declared) <= set(_abi.exported_symbols())


@pytest.mark.parametrize("k", list(range(2, 25, 2)))
def test_fornberg_weights_match_oracle(built_lib, oracle_mod, k):
    got = _abi.fd_fd_weights(k)
    want = oracle_mod.fd_weights(k)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


def test_weights_reject_odd_orders(built_lib):
    for k in (1, 3, 0, 26):
        with pytest.raises(_abi.FdError) as e:
            _abi.fd_fd_weights(k)
        assert e.value.code == _abi.FD_EINVAL


@pytest.mark.parametrize("k", [2, 4, 8, 12, 16])
def test_dt_max_matches_oracle(built_lib, oracle_mod, k):
    for h, v in ((10.0, 1500.0), (10.0, 4500.0), (3.0, 2000.0)):
        assert _abi.fd_dt_max(k, h, v) == pytest.approx(oracle_mod.dt_max(k, h, v), rel=1e-13)


def test_dt_max_table_values(built_lib):
    """0.9 dt_max at h = 10 m: 3.464 ms (k=2), 3.000 ms (k=4), 2.717 ms (k=8) at
    1.5 km/s; 0.847 ms (k=16) at 4.5 km/s."""
    assert 0.9 * _abi.fd_dt_max(2, 10.0, 1500.0) == pytest.approx(3.4641e-3, rel=1e-4)
    assert 0.9 * _abi.fd_dt_max(4, 10.0, 1500.0) == pytest.approx(3.0000e-3, rel=1e-4)
    assert 0.9 * _abi.fd_dt_max(8, 10.0, 1500.0) == pytest.approx(2.7173e-3, rel=1e-3)
    assert 0.9 * _abi.fd_dt_max(16, 10.0, 4500.0) == pytest.approx(0.8472e-3, rel=1e-3)


def test_default_damping_matches_oracle(built_lib, oracle_mod):
    rng = np.random.default_rng(1)
    shape = (17, 19, 23)
    m = (1.0 / rng.uniform(1500, 4500, shape) ** 2).astype(np.float32)
    for nbl in (0, 3, 6):
        got = _abi.fd_default_damping(m, nbl, 10.0)
        want = oracle_mod.default_damping(m.astype(np.float64), nbl, 10.0)
        np.testing.assert_allclose(got, want, rtol=2e-7, atol=0)


def test_version_and_error_text(built_lib):
    assert "sm_103a" in _abi.fd_version()
    with pytest.raises(_abi.FdError):
        _abi.fd_dt_max(3, 10.0, 1500.0)
    assert "space_order" in _abi.fd_last_error() or _abi.fd_last_error() != ""


def test_options_default(built_lib):
    o = _abi.fd_options_default()
    assert (o.storage, o.form, o.kernel, o.tile_z, o.tile_y, o.x_block, o.check_finite, o.boundary, o.rows) == \
        (0, 0, 0, 0, 0, 0, 1, 0, 0)
    assert ctypes.sizeof(o) == 9 * 4


def test_options_struct_matches_header():
    """The binding's fd_options has the header's fields, in the header's order."""
    import re
    text = open(os.path.join(ROOT, "include", "fd_acoustic.h")).read()
    body = text[text.index("typedef struct fd_options {"):text.index("} fd_options;")]
    fields = re.findall(r"^\s*int (\w+);", body, flags=re.M)
    assert fields == [f for f, _ in _abi.fd_options._fields_]


def test_null_arguments_fail_before_any_device_work(built_lib):
    """Argument errors are reported on the host, with no CUDA call made (these
    run on a machine without a GPU)."""
    lib = built_lib
    assert lib.fd_kernel_launches(None) == _abi.FD_EINVAL
    assert lib.fd_selftest_waits(None, None, None) == _abi.FD_EINVAL
    assert lib.fd_forward(None, 1) == _abi.FD_EINVAL
    assert lib.fd_forward_flow(None, 1) == _abi.FD_EINVAL
    assert lib.fd_forward_two_step(None, 2) == _abi.FD_EINVAL
    assert lib.fd_read_wavefield(None, None, 0) == _abi.FD_EINVAL
    assert lib.fd_destroy(None) == _abi.FD_OK
    assert "NULL" in _abi.fd_last_error() or _abi.fd_last_error() != ""


def test_kernel_launch_counter_reads_on_the_host(built_lib):
    n = _abi.fd_kernel_launches()
    import torch
    if not torch.cuda.is_available():
        assert n == 0  # nothing can have been launched in this process
    else:
        assert n >= 0


def test_shot_device_bytes_counts_the_pitched_fields(built_lib):
    out = ctypes.c_longlong()
    for (nx, ny, nz, nbl, st) in ((64, 64, 64, 10, 0), (100, 37, 250, 20, 1), (1, 1, 1, 0, 2)):
        assert built_lib.fd_shot_device_bytes(nx, ny, nz, nbl, st, ctypes.byref(out)) == _abi.FD_OK
        Nx, Ny, Nz = nx + 2 * nbl, ny + 2 * nbl, nz + 2 * nbl
        n = Nx * Ny * (-(-Nz // 64) * 64)  # rows padded to 64 elements
        levels = 2 * n * 4 if st == 0 else 3 * n * 2  # FP32: two levels; 16-bit: u twice and the increment
        assert out.value == levels + 2 * n * 4 + (1 << 16)  # plus the two coefficient fields and slack
    assert built_lib.fd_shot_device_bytes(0, 1, 1, 0, 0, ctypes.byref(out)) == _abi.FD_EINVAL
    assert built_lib.fd_shot_device_bytes(1, 1, 1, 0, 3, ctypes.byref(out)) == _abi.FD_EINVAL


def test_create_arguments_are_checked_on_the_host(built_lib):
    """Every argument and option check of the create calls runs before any CUDA
    call, so each rejection is reported here without a GPU and leaves the
    output handle NULL."""
    lib = built_lib

    def opts(**kw):
        o = _abi.fd_options_default()
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def create(nx=16, ny=16, nz=16, k=8, h=10.0, dt=1e-3, nbl=2, opt=None):
        out = ctypes.c_void_p(12345)
        rc = lib.fd_acoustic_create_ex(nx, ny, nz, k, h, dt, nbl,
                                       ctypes.byref(opt) if opt is not None else None, ctypes.byref(out))
        assert out.value is None, "a rejected create must leave the handle NULL"
        return rc

    EINVAL, ENOTSUP = _abi.FD_EINVAL, _abi.FD_ENOTSUP
    for k in (-2, 0, 1, 3, 25, 26):
        assert create(k=k) == EINVAL, k
    for dims in ((0, 16, 16), (16, 0, 16), (16, 16, -1)):
        assert create(*dims) == EINVAL, dims
    assert create(nbl=-1) == EINVAL
    for h, dt in ((0.0, 1e-3), (-10.0, 1e-3), (float("nan"), 1e-3), (float("inf"), 1e-3),
                  (10.0, 0.0), (10.0, float("nan")), (10.0, -1e-3)):
        assert create(h=h, dt=dt) == EINVAL, (h, dt)
    # the largest extent is 65535 nodes per axis, layer included
    assert create(nx=65536, nbl=0) == EINVAL
    assert create(ny=65535 - 2 * 99, nbl=100) == EINVAL
    assert create(nz=65534, nbl=1) == EINVAL
    for kw in (dict(storage=3), dict(storage=-1), dict(form=2), dict(kernel=4), dict(boundary=2)):
        assert create(opt=opts(**kw)) == ENOTSUP, kw
    for kw in (dict(boundary=1, storage=1), dict(boundary=1, kernel=3),   # periodic: FP32, naive kernel
               dict(storage=1, form=1), dict(storage=2, kernel=1), dict(storage=2, kernel=2),
               dict(tile_z=48, tile_y=16), dict(kernel=1, tile_z=64, tile_y=8), dict(kernel=2, rows=2)):
        assert create(opt=opts(**kw)) == ENOTSUP, kw
    assert create(opt=opts(rows=3)) == EINVAL
    assert create(opt=opts(rows=-1)) == EINVAL
    assert create(opt=opts(x_block=-1)) == EINVAL
    assert lib.fd_acoustic_create_ex(16, 16, 16, 8, 10.0, 1e-3, 2, None, None) == EINVAL

    def slab(x0, x1, k=8, opt=None):
        out = ctypes.c_void_p(12345)
        rc = lib.fd_slab_create(16, 16, 16, k, 10.0, 1e-3, 2, x0, x1,
                                ctypes.byref(opt) if opt is not None else None, ctypes.byref(out))
        assert out.value is None
        return rc

    assert slab(-1, 4) == EINVAL
    assert slab(5, 5) == EINVAL
    assert slab(0, 21) == EINVAL                 # past the 20 planes of the domain
    assert slab(4, 7) == EINVAL                  # 3 planes, fewer than k/2 = 4
    assert slab(0, 10, opt=opts(storage=1)) == ENOTSUP
    assert slab(0, 10, opt=opts(kernel=2)) == ENOTSUP

    def batch(k=8, h=10.0, opt=None):
        out = ctypes.c_void_p(12345)
        rc = lib.fd_batch_create(k, h, ctypes.byref(opt) if opt is not None else None, ctypes.byref(out))
        assert out.value is None
        return rc

    for k in (0, 3, 18, 24):
        assert batch(k=k) == EINVAL, k
    assert batch(h=0.0) == EINVAL
    assert batch(h=float("nan")) == EINVAL
    for kw in (dict(storage=3), dict(form=2), dict(storage=1, form=1), dict(boundary=1),
               dict(tile_z=128, tile_y=8), dict(rows=2)):
        assert batch(opt=opts(**kw)) == ENOTSUP, kw
