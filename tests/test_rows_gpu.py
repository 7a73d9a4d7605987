"""GPU tests of the two-rows-per-thread launch shapes of the TMA step kernel
(tiles 32x32 and 64x16 in which every thread owns 4 z points of two adjacent
y rows and loads each y-tap row once for both): the same per-point arithmetic
as one row per thread, so the results are bit for bit those of the 32x16 tile
with one row per thread, for every space order up to 16, both stencil forms,
FP32 and 16-bit storage, per-step launches and the flow schedule, on a ragged
grid whose y extent leaves a last tile with one row of a pair outside the
domain, with sources on even and odd rows; and the FP64 oracle within the
FP32 bound."""
import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import inputs
from harness import dt_for, eta_for, rel_l2, run_oracle

pytestmark = pytest.mark.gpu
H = inputs.H


def _spec(k, seed, interior=(41, 43, 57), nbl=5, nt=24):
    rng = np.random.default_rng(seed)
    vel = inputs.smooth_random_velocity(interior, nbl, rng, sigma=4.0)
    return inputs.ShotSpec(interior, nbl, k, vel, (0, 0, 0), 25.0, nt)


# interior nodes on even and odd domain rows (y + nbl), tile edges, the last row
SOURCES = [(3, 0, 5), (20, 27, 31), (40, 42, 56), (11, 26, 0)]


def _run(spec, eta, flow=False, chunks=None, **opts):
    dt = dt_for(spec)
    with fd.Shot(spec.interior, spec.space_order, H, dt, spec.nbl, kernel="tma", **opts) as shot:
        shot.set_model(spec.m, eta)
        for i, s in enumerate(SOURCES):
            shot.inject(*s, inputs.ricker(20.0 + 3 * i, dt, spec.nt))
        for n in (chunks or [spec.nt]):
            (shot.forward_flow if flow else shot.forward)(n)
        assert shot.schedule[0] == opts.get("rows", 1)
        return shot.wavefield(0), shot.wavefield(1)


@pytest.mark.parametrize("form", ["factored", "expanded"])
@pytest.mark.parametrize("k", [2, 4, 6, 8, 10, 12, 14, 16])
def test_two_rows_equal_one_row_fp32(k, form):
    spec = _spec(k, seed=100 + k)
    rng = np.random.default_rng(k)
    eta = (spec.m * rng.uniform(0, 10.0, spec.m.shape) * (rng.uniform(size=spec.m.shape) < 0.3)).astype(np.float32)
    want = _run(spec, eta, form=form, tile_z=32, tile_y=16, rows=1, x_block=11)
    for tz, ty in ((32, 32), (64, 16)):
        got = _run(spec, eta, form=form, tile_z=tz, tile_y=ty, rows=2, x_block=9)
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_array_equal(got[1], want[1])
    # the flow schedule with two rows per thread
    got = _run(spec, eta, flow=True, chunks=[5, spec.nt - 5], form=form, tile_z=32, tile_y=32, rows=2,
               x_block=max(k // 2, 8))
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("k", [2, 8, 16])
def test_two_rows_equal_one_row_16bit(k, storage):
    spec = _spec(k, seed=200 + k)
    eta = eta_for(spec)
    want = _run(spec, eta, storage=storage, tile_z=32, tile_y=16, rows=1, x_block=13)
    for tz, ty in ((32, 32), (64, 16)):
        got = _run(spec, eta, storage=storage, tile_z=tz, tile_y=ty, rows=2, x_block=7)
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_array_equal(got[1], want[1])


def test_two_rows_match_oracle(oracle_mod):
    k = 12
    spec = _spec(k, seed=9)
    dt = dt_for(spec)
    eta = eta_for(spec)
    srcs = [(s, inputs.ricker(20.0 + 3 * i, dt, spec.nt)) for i, s in enumerate(SOURCES)]
    want, want_prev = run_oracle(oracle_mod, spec, spec.nt, dt, eta, sources=srcs)
    got, got_prev = _run(spec, eta, tile_z=32, tile_y=32, rows=2)
    e0, e1 = rel_l2(got, want), rel_l2(got_prev, want_prev)
    print(f"PARITY rows2_so{k} {e0:.3e} {e1:.3e}")
    assert e0 <= 1e-5 and e1 <= 1e-5


def test_two_rows_rejected_where_absent():
    spec = _spec(20, seed=1)
    dt = dt_for(spec)
    with pytest.raises(fd.FdError) as e:
        fd.Shot(spec.interior, 20, H, dt, spec.nbl, kernel="tma", rows=2)
    assert e.value.code == fd.FD_ENOTSUP
    with pytest.raises(fd.FdError) as e:
        fd.Shot(spec.interior, 8, H, dt, spec.nbl, kernel="tma", tile_z=128, tile_y=8, rows=2)
    assert e.value.code == fd.FD_ENOTSUP
