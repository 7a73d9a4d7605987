"""GPU tests of the batch flow schedule: every step of a forward in one
persistent launch over every shot of a batch (FP32).

An item runs the per-step batch kernel's per-point arithmetic, so each shot's
result must equal its run alone bit for bit, for any x-chunk length, with shots
at different steps and shots added between forwards, and must match the FP64
oracle within the FP32 tolerance.
"""
import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import inputs
from harness import dt_for, eta_for, rel_l2, run_oracle
from test_batch_gpu import _alone, _shots

pytestmark = pytest.mark.gpu

H = inputs.H


def _fill(b, specs):
    slots = []
    for spec in specs:
        s = b.add(spec.interior, spec.nbl, spec.dt, spec.m)
        b.inject(s, *spec.source, inputs.ricker(spec.f0, spec.dt, spec.nt))
        slots.append(s)
    return slots


@pytest.mark.parametrize("form", ["factored", "expanded"])
@pytest.mark.parametrize("k,xb", [(2, 0), (2, 3), (8, 4), (8, 13), (16, 8), (16, 0)])
def test_batch_flow_equals_alone(k, xb, form):
    specs = _shots(k, seed=40 + k + xb, count=4)
    with fd.Batch(k, H, form=form, x_block=xb) as b:
        slots = _fill(b, specs)
        b.forward_flow(17)  # first time: direct launch
        b.forward_flow(23)
        n0 = fd.fd_kernel_launches()
        b.forward_flow(23)  # graph replay: one kernel for the 23 steps
        assert fd.fd_kernel_launches() - n0 == 1
        for spec, s in zip(specs, slots):
            want, want_prev = _alone(spec, 63, form=form)
            assert b.step(s) == 63
            assert b.status(s) == 0
            np.testing.assert_array_equal(b.wavefield(s, 0), want)
            np.testing.assert_array_equal(b.wavefield(s, 1), want_prev)


def test_batch_flow_shots_at_different_steps():
    """Shots joining between forwards run behind the others; per-step and flow
    forwards mixed on the same batch give the same bits."""
    specs = _shots(8, seed=77, count=4)
    with fd.Batch(8, H, x_block=7) as b:
        slots = _fill(b, specs[:3])
        b.forward_flow(9)
        slots += _fill(b, specs[3:])
        b.forward(4)
        b.forward_flow(21)
        b.remove(slots[1])
        b.forward_flow(5)
        for i, (spec, n) in enumerate(zip(specs, (39, 30, 39, 30))):
            if i == 1:
                continue
            want, want_prev = _alone(spec, n)
            assert b.step(slots[i]) == n
            np.testing.assert_array_equal(b.wavefield(slots[i], 0), want)
            np.testing.assert_array_equal(b.wavefield(slots[i], 1), want_prev)


def test_batch_flow_matches_oracle(oracle_mod):
    specs = _shots(8, seed=5, count=3)
    with fd.Batch(8, H) as b:
        slots = _fill(b, specs)
        b.forward_flow(60)
        for spec, s in zip(specs, slots):
            want, _ = run_oracle(oracle_mod, spec, 60, spec.dt, eta_for(spec))
            e = rel_l2(b.wavefield(s, 0), want)
            print(f"PARITY batch_flow_so8_{spec.interior} {e:.3e}")
            assert e <= 1e-5


def test_batch_schedule_choice_on_a_later_forward():
    """A forward too short for the schedule choice after the shape tuning (as a
    server's 50-step chunks are) leaves it to the next one; the results do not
    change."""
    specs = _shots(8, seed=93, count=4)
    with fd.Batch(8, H) as b:
        slots = _fill(b, specs)
        b.forward(50)  # shapes: 39 steps; 11 left, too few for the schedule probes
        assert b.config()[3] == 1
        b.forward(40)  # the schedule probes: 30 real steps
        b.forward(7)
        for spec, s in zip(specs, slots):
            want, want_prev = _alone(spec, 97)
            assert b.step(s) == 97
            np.testing.assert_array_equal(b.wavefield(s, 0), want)
            np.testing.assert_array_equal(b.wavefield(s, 1), want_prev)


def test_batch_autotuned_schedule_equals_alone():
    """The autotuner times the per-step shapes, then the flow, and keeps one
    schedule; whichever it keeps, every shot equals its run alone."""
    specs = _shots(4, seed=91, count=5)
    with fd.Batch(4, H) as b:
        slots = _fill(b, specs)
        b.forward(90)  # long enough to tune: the tuning steps are real steps
        assert b.config()[3] == 1
        assert b.schedule() in (0, 1)
        b.forward(11)
        for spec, s in zip(specs, slots):
            want, want_prev = _alone(spec, 101)
            assert b.step(s) == 101
            np.testing.assert_array_equal(b.wavefield(s, 0), want)
            np.testing.assert_array_equal(b.wavefield(s, 1), want_prev)


def test_batch_pinned_per_step_launches():
    """kernel="tma" pins one launch per step: the shape is still tuned, the
    schedule is not probed."""
    specs = _shots(8, seed=95, count=4)
    with fd.Batch(8, H, kernel="tma") as b:
        slots = _fill(b, specs)
        b.forward(80)
        assert b.config()[3] == 1 and b.schedule() == 0
        n0 = fd.fd_kernel_launches()
        b.forward(6)
        assert fd.fd_kernel_launches() - n0 == 6
        for spec, s in zip(specs, slots):
            want, _ = _alone(spec, 86)
            np.testing.assert_array_equal(b.wavefield(s, 0), want)


def test_batch_flow_rejections():
    specs = _shots(8, seed=3, count=1)
    with fd.Batch(8, H, storage="bf16") as b:
        _fill(b, specs)
        with pytest.raises(fd.FdError) as e:
            b.forward_flow(3)
        assert e.value.code == fd.FD_ENOTSUP
    with fd.Batch(8, H, x_block=3) as b:
        _fill(b, specs)
        with pytest.raises(fd.FdError) as e:
            b.forward_flow(3)
        assert e.value.code == fd.FD_ENOTSUP


@pytest.mark.parametrize("schedule", ["auto", "flow"])
def test_batch_full_size_equals_alone(schedule, oracle_mod):
    """The batched workload's shots at their full sizes (the first four of its
    seeded list: each axis 96-256 + 10, space order 8, smooth random velocity),
    through the autotuned batch (shape and schedule timed on real steps) or the
    persistent launch: every shot equals its run alone bit for bit, and the
    first matches the FP64 oracle within the FP32 bound."""
    specs = inputs.batched_shots(count=4, nt=120)
    for spec in specs:
        spec.dt = dt_for(spec)
    with fd.Batch(8, H) as b:
        slots = _fill(b, specs)
        if schedule == "flow":
            b.forward_flow(80)
            b.forward_flow(20)
        else:
            b.forward(80)  # shapes (39 steps) and schedule (30 steps), then 11 more
            assert b.config()[3] == 1 and b.schedule() in (0, 1)
            b.forward(20)
        for spec, s in zip(specs, slots):
            want, want_prev = _alone(spec, 100)
            assert b.step(s) == 100
            np.testing.assert_array_equal(b.wavefield(s, 0), want)
            np.testing.assert_array_equal(b.wavefield(s, 1), want_prev)
        spec = specs[0]
        ref, _ = run_oracle(oracle_mod, spec, 100, spec.dt, eta_for(spec))
        e = rel_l2(b.wavefield(slots[0], 0), ref)
        print(f"PARITY batch_full_{schedule}_{spec.interior} {e:.3e}")
        assert e <= 1e-5
