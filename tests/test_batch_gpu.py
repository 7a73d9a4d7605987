"""GPU tests of batches: uneven shots advanced together in one launch per step.

Each shot's result must be the same alone (its own handle, fd_forward) and in
the mix (bit for bit: the per-point arithmetic does not depend on which other
shots share the launch), including shots added and removed between forwards
(continuous batching), and must match the FP64 oracle within the FP32
tolerance.
"""
import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import inputs
from harness import dt_for, eta_for, rel_l2, run_oracle

pytestmark = pytest.mark.gpu

H = inputs.H


def _shots(k, seed, count=5):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        interior = tuple(int(v) for v in rng.integers(20, 60, size=3))
        nbl = int(rng.integers(3, 8))
        vel = inputs.smooth_random_velocity(interior, nbl, rng, sigma=3.0)
        src = tuple(int(rng.integers(0, n)) for n in interior)
        spec = inputs.ShotSpec(interior, nbl, k, vel, src, float(rng.uniform(8, 30)), 200)
        spec.dt = dt_for(spec)
        out.append(spec)
    return out


def _alone(spec, nt, storage="f32", form="factored"):
    with fd.Shot(spec.interior, spec.space_order, H, spec.dt, spec.nbl, storage=storage,
                 form=form, kernel="tma", tile_z=32, tile_y=16) as shot:
        shot.set_model(spec.m)
        shot.inject(*spec.source, inputs.ricker(spec.f0, spec.dt, spec.nt))
        shot.forward(nt)
        return shot.wavefield(0), shot.wavefield(1)


@pytest.mark.parametrize("storage,form", [("f32", "factored"), ("f32", "expanded"),
                                          ("bf16", "factored")])
@pytest.mark.parametrize("k", [4, 8, 16])
def test_batch_equals_alone(k, storage, form):
    specs = _shots(k, seed=k)
    with fd.Batch(k, H, storage=storage, form=form) as b:
        slots = []
        for spec in specs:
            s = b.add(spec.interior, spec.nbl, spec.dt, spec.m)
            b.inject(s, *spec.source, inputs.ricker(spec.f0, spec.dt, spec.nt))
            slots.append(s)
        b.forward(17)
        b.forward(23)
        for spec, s in zip(specs, slots):
            want, want_prev = _alone(spec, 40, storage, form)
            assert b.step(s) == 40
            np.testing.assert_array_equal(b.wavefield(s, 0), want)
            np.testing.assert_array_equal(b.wavefield(s, 1), want_prev)


def test_batch_matches_oracle(oracle_mod):
    specs = _shots(8, seed=3, count=3)
    with fd.Batch(8, H) as b:
        slots = []
        for spec in specs:
            s = b.add(spec.interior, spec.nbl, spec.dt, spec.m)
            b.inject(s, *spec.source, inputs.ricker(spec.f0, spec.dt, spec.nt))
            slots.append(s)
        b.forward(60)
        for spec, s in zip(specs, slots):
            want, _ = run_oracle(oracle_mod, spec, 60, spec.dt, eta_for(spec))
            e = rel_l2(b.wavefield(s, 0), want)
            print(f"PARITY batch_so8_{spec.interior} {e:.3e}")
            assert e <= 1e-5


def test_continuous_batching_add_remove():
    """Shots join and leave between forwards; each still equals its run alone."""
    specs = _shots(8, seed=9, count=4)
    with fd.Batch(8, H) as b:
        def add(spec):
            s = b.add(spec.interior, spec.nbl, spec.dt, spec.m)
            b.inject(s, *spec.source, inputs.ricker(spec.f0, spec.dt, spec.nt))
            return s
        s0 = add(specs[0])
        b.forward(10)
        s1 = add(specs[1])
        s2 = add(specs[2])
        b.forward(15)
        u0 = b.wavefield(s0)
        b.remove(s0)
        s3 = add(specs[3])  # reuses the freed slot
        assert s3 == s0
        b.forward(8)
        b.remove(s2)
        b.forward(5)
        np.testing.assert_array_equal(u0, _alone(specs[0], 25)[0])
        np.testing.assert_array_equal(b.wavefield(s1), _alone(specs[1], 28)[0])
        np.testing.assert_array_equal(b.wavefield(s3), _alone(specs[3], 13)[0])
        assert b.step(s1) == 28 and b.step(s3) == 13
        assert b.size()[0] == 2


def test_batch_errors():
    with pytest.raises(fd.FdError) as e:
        fd.Batch(8, H, storage="bf16", form="expanded")
    assert e.value.code == fd.FD_ENOTSUP
    with fd.Batch(4, H) as b:
        spec = _shots(4, seed=1, count=1)[0]
        s = b.add(spec.interior, spec.nbl, spec.dt, spec.m)
        for _ in range(4):  # a batched shot holds at most 4 sources
            b.inject(s, 0, 0, 0, np.ones(3, np.float32))
        with pytest.raises(fd.FdError) as e:
            b.inject(s, 0, 0, 0, np.ones(3, np.float32))
        assert e.value.code == fd.FD_ENOTSUP
        with pytest.raises(fd.FdError):
            b.remove(s + 5)
        with pytest.raises(fd.FdError) as e:
            b.add(spec.interior, spec.nbl, 10 * spec.dt, spec.m)
        assert e.value.code == fd.FD_EUNSTABLE


@pytest.mark.parametrize("xb", [4, 7, 16])
def test_batch_with_x_chunks(xb):
    """Several x-chunks per shot, shots at different steps: each result still
    equals its run alone, bit for bit, and a forward is one launch per step."""
    specs = _shots(8, seed=20 + xb, count=4)
    with fd.Batch(8, H, x_block=xb) as b:
        slots = []
        for spec in specs[:3]:
            s = b.add(spec.interior, spec.nbl, spec.dt, spec.m)
            b.inject(s, *spec.source, inputs.ricker(spec.f0, spec.dt, spec.nt))
            slots.append(s)
        b.forward(9)
        s3 = b.add(specs[3].interior, specs[3].nbl, specs[3].dt, specs[3].m)
        b.inject(s3, *specs[3].source, inputs.ricker(specs[3].f0, specs[3].dt, specs[3].nt))
        slots.append(s3)
        b.forward(3)  # rebuilds the work list
        b.forward(21)  # first time: direct launches
        n0 = fd.fd_kernel_launches()
        b.forward(21)  # graph replay
        assert fd.fd_kernel_launches() - n0 == 21
        for spec, s, n in zip(specs, slots, (54, 54, 54, 45)):
            want, want_prev = _alone(spec, n)
            assert b.step(s) == n
            np.testing.assert_array_equal(b.wavefield(s, 0), want)
            np.testing.assert_array_equal(b.wavefield(s, 1), want_prev)


def test_batch_launch_per_step_16bit():
    specs = _shots(8, seed=31, count=2)
    with fd.Batch(8, H, storage="bf16") as b:
        for spec in specs:
            s = b.add(spec.interior, spec.nbl, spec.dt, spec.m)
            b.inject(s, *spec.source, inputs.ricker(spec.f0, spec.dt, spec.nt))
        b.forward(5)
        n0 = fd.fd_kernel_launches()
        b.forward(5)
        assert fd.fd_kernel_launches() - n0 == 5


@pytest.mark.parametrize("storage,k", [("f32", 4), ("f32", 16), ("bf16", 8)])
def test_batch_autotune_keeps_results(k, storage):
    """The first forward of at least 39 steps over at least 4 shots times the
    launch shapes (both tiles, six x-chunk policies) on real steps and keeps
    the fastest (FP32 then chooses its schedule on the 30 steps after); every
    shot still equals the same shot alone, bit for bit, and a shot added after
    the choice takes it."""
    specs = _shots(k, seed=50 + k, count=6)
    with fd.Batch(k, H, storage=storage) as b:
        assert b.config()[3] == 0
        slots = []
        for spec in specs[:5]:
            s = b.add(spec.interior, spec.nbl, spec.dt, spec.m)
            b.inject(s, *spec.source, inputs.ricker(spec.f0, spec.dt, spec.nt))
            slots.append(s)
        b.forward(75)
        tz, ty, xb, tuned = b.config()
        assert tuned == 1 and (tz, ty) in ((32, 16), (64, 8)) and xb in (32, 48, 64, 96, 128, 0)
        late = specs[5]
        s_late = b.add(late.interior, late.nbl, late.dt, late.m)
        b.inject(s_late, *late.source, inputs.ricker(late.f0, late.dt, late.nt))
        b.forward(12)
        assert b.config() == (tz, ty, xb, 1)
        for spec, s in zip(specs[:5], slots):
            want, want_prev = _alone(spec, 87, storage)
            assert b.step(s) == 87
            np.testing.assert_array_equal(b.wavefield(s, 0), want)
            np.testing.assert_array_equal(b.wavefield(s, 1), want_prev)
        want, _ = _alone(late, 12, storage)
        np.testing.assert_array_equal(b.wavefield(s_late, 0), want)
