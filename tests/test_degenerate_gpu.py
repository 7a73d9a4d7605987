"""GPU parity on the degenerate cases of the scheme: domains thinner than the
stencil, a one-node domain, zero-step calls and empty batches.

A domain thinner than the stencil radius along an axis puts every tap beyond
its last node in the zero Dirichlet halo (Eq. 1 with the field zero outside the
computational domain); a one-node domain reduces the Laplacian to its centre
weight. These shapes drive the kernels through one tile, one x-chunk shorter
than the radius, z rows shorter than one 4-point vector, flow items that wait
only on their own region of the previous step, and the two-step kernel on a
chunk narrower than its halo. Every schedule must still match the FP64 oracle,
and a batch holding such shots must give each the bits it gets alone.

Errors are L2 norms of the difference relative to the larger L2 norm of the
oracle's two levels: a level's rounding error scales with the state that formed
it, and on a one-node domain a single level can sit near a sign change (there
its own value is no scale). Bounds: 1e-5 for FP32; for 16-bit storage the
increment form's rounding envelope, 4 half-ulps of the stored format per step
accumulated as a random walk over the steps (bf16 half-ulp 2^-9; fp16 2^-12,
its per-level power-of-two scale keeping values in the normal range).
"""
import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import inputs
from harness import dt_for, eta_for, rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL = 1e-5
NT = 30
STORAGE_TOL = {"bf16": 4 * 2.0 ** -9 * np.sqrt(NT), "f16": 4 * 2.0 ** -12 * np.sqrt(NT)}

# (interior, nbl, space order, source node): each thinner than the radius k/2
# along at least one axis
THIN = [
    ((1, 23, 30), 0, 8, (0, 11, 14)),     # one x plane
    ((1, 20, 26), 2, 16, (0, 9, 12)),     # Nx = 5 < R = 8, with a damping layer
    ((30, 3, 27), 0, 16, (14, 1, 13)),    # Ny = 3 < R
    ((27, 26, 1), 1, 12, (13, 12, 0)),    # Nz = 3: one partial 4-point vector per row
    ((3, 2, 3), 1, 24, (1, 1, 1)),        # every axis thinner than R = 12
    ((1, 1, 1), 0, 4, (0, 0, 0)),         # one node
    ((1, 20, 21), 0, 2, (0, 10, 10)),     # space order 2: the two-step kernel by default
]


def _spec(case, seed):
    interior, nbl, k, src = case
    rng = np.random.default_rng(seed)
    vel = inputs.smooth_random_velocity(interior, nbl, rng, sigma=3.0)
    return inputs.ShotSpec(interior, nbl, k, vel, src, 25.0, NT)


def _state(spec, seed):
    """A smooth random full-field state, so that every node carries signal."""
    rng = np.random.default_rng(seed)
    u0 = inputs._gaussian_smooth(rng.standard_normal(spec.shape), 1.5).astype(np.float32) * 10.0
    return u0, (0.99 * u0).astype(np.float32), 3


def _errs(got, got_prev, want, want_prev):
    """Both levels' errors relative to the larger norm of the oracle's levels."""
    scale = max(np.linalg.norm(want), np.linalg.norm(want_prev))
    return tuple(float(np.linalg.norm(np.asarray(a, np.float64) - b) / scale)
                 for a, b in ((got, want), (got_prev, want_prev)))


def _flow(spec, dt, state, **opts):
    """The same shot through the explicit one-launch flow entry point."""
    shot = fd.Shot(spec.interior, spec.space_order, inputs.H, dt, spec.nbl, **opts)
    shot.set_model(spec.m, None)
    shot.inject(*spec.source, inputs.ricker(spec.f0, dt, spec.nt))
    shot.load_state(*state)
    shot.forward_flow(7)
    shot.forward_flow(NT - 7)
    return shot.wavefield(0), shot.wavefield(1), shot


@pytest.mark.parametrize("form", ["factored", "expanded"])
@pytest.mark.parametrize("case", range(len(THIN)))
def test_thin_domains_match_oracle(oracle_mod, case, form):
    spec = _spec(THIN[case], seed=40 + case)
    dt = dt_for(spec)
    state = _state(spec, seed=50 + case)
    want, want_prev = run_oracle(oracle_mod, spec, NT, dt, eta_for(spec), state=state)
    runs = [("auto", lambda: run_gpu(spec, NT, dt, state=state, chunks=[11, NT - 11], form=form)),
            ("flow", lambda: _flow(spec, dt, state, form=form)),
            ("tma", lambda: run_gpu(spec, NT, dt, state=state, form=form, kernel="tma")),
            ("stream", lambda: run_gpu(spec, NT, dt, state=state, form=form, kernel="stream")),
            ("naive", lambda: run_gpu(spec, NT, dt, state=state, form=form, kernel="naive"))]
    for name, run in runs:
        got, got_prev, shot = run()
        assert shot.step == 3 + NT
        e0, e1 = _errs(got, got_prev, want, want_prev)
        print(f"PARITY thin{THIN[case][0]}_so{spec.space_order}_{form}_{name} {e0:.3e} {e1:.3e}")
        assert e0 <= TOL and e1 <= TOL, (name, e0, e1)
        shot.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("case", [0, 3, 4])
def test_thin_domains_16bit(oracle_mod, case, storage):
    spec = _spec(THIN[case], seed=60 + case)
    dt = dt_for(spec)
    state = _state(spec, seed=70 + case)
    want, want_prev = run_oracle(oracle_mod, spec, NT, dt, eta_for(spec), state=state)
    got, got_prev, shot = run_gpu(spec, NT, dt, state=state, storage=storage)
    e = max(_errs(got, got_prev, want, want_prev))
    print(f"PARITY thin{THIN[case][0]}_so{spec.space_order}_{storage} {e:.3e}")
    assert e <= STORAGE_TOL[storage], e
    shot.close()


def test_zero_steps_change_nothing():
    """nt = 0 is a no-op on every entry point; nt < 0 is an argument error."""
    for k, form in ((8, "expanded"), (2, "factored")):
        spec = _spec(((1, 23, 30), 0, k, (0, 11, 14)), seed=80)
        got, got_prev, shot = run_gpu(spec, 5, dt_for(spec), form=form)
        calls = [shot.forward, shot.forward_flow] + ([shot.forward_two_step] if k <= 4 else [])
        for call in calls:
            call(0)
            assert shot.step == 5
            np.testing.assert_array_equal(shot.wavefield(0), got)
            np.testing.assert_array_equal(shot.wavefield(1), got_prev)
            with pytest.raises(fd.FdError) as e:
                call(-1)
            assert e.value.code == fd.FD_EINVAL
        shot.close()


def test_empty_batch_and_thin_shots_in_a_batch(oracle_mod):
    """An empty batch advances nothing without error, before and after its shots
    are removed; thin shots beside a regular one keep their bits alone in both
    batch schedules."""
    k = 8
    b = fd.Batch(k, inputs.H, kernel="tma")
    b.forward(5)
    b.forward(0)
    assert b.size() == (0, 0)
    cases = [((1, 23, 30), 0, k, (0, 11, 14)), ((27, 26, 1), 1, k, (13, 12, 0)),
             ((3, 2, 3), 1, k, (1, 1, 1)), ((40, 36, 44), 4, k, (20, 18, 22))]
    specs = [_spec(c, seed=90 + i) for i, c in enumerate(cases)]
    dts = [dt_for(s) for s in specs]
    slots = []
    for s, dt in zip(specs, dts):
        slot = b.add(s.interior, s.nbl, dt, s.m)
        b.inject(slot, *s.source, inputs.ricker(s.f0, dt, 60))
        slots.append(slot)
    b.forward(25)
    b.forward_flow(35)
    for s, dt, slot in zip(specs, dts, slots):
        assert b.step(slot) == 60
        with fd.Shot(s.interior, k, inputs.H, dt, s.nbl, kernel="tma") as alone:
            alone.set_model(s.m)
            alone.inject(*s.source, inputs.ricker(s.f0, dt, 60))
            alone.forward(25)
            alone.forward_flow(35)
            u = alone.wavefield(0)
            np.testing.assert_array_equal(b.wavefield(slot, 0), u)
            np.testing.assert_array_equal(b.wavefield(slot, 1), alone.wavefield(1))
        assert np.abs(u).max() > 0
    s, dt = specs[1], dts[1]
    want, _ = run_oracle(oracle_mod, s, 60, dt, eta_for(s),
                         sources=[(s.source, inputs.ricker(s.f0, dt, 60))])
    e = rel_l2(b.wavefield(slots[1], 0), want)
    print(f"PARITY batch_thin{s.interior}_so{k} {e:.3e}")
    assert e <= TOL, e
    for slot in slots:
        b.remove(slot)
    b.forward(5)
    b.forward_flow(5)
    assert b.size() == (0, 0)
    b.close()
