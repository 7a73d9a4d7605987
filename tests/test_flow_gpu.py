"""GPU tests of the flow schedule (one persistent launch for nt steps, work
items started as soon as the items of the previous step around them are done):
bit for bit the per-step launches of the same kernel (every space order, both
forms, several tiles and x-blocks down to x_block = k/2, ragged grids, chunked
calls, sources at tile edges, the benchmark's full-size shot), the FP64 oracle
within the FP32 bound, one kernel launch per call, and the unsupported cases
rejected. Receivers and sources beyond the four fused ones ride on the FP32
flow: traces and fields bit for bit those of the per-step launches."""
import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import inputs
from harness import dt_for, eta_for, rel_l2, run_oracle

pytestmark = pytest.mark.gpu
H = inputs.H


def _spec(k, seed, interior=(53, 41, 70), nbl=7):
    rng = np.random.default_rng(seed)
    vel = inputs.smooth_random_velocity(interior, nbl, rng, sigma=4.0)
    return inputs.ShotSpec(interior, nbl, k, vel, (0, 0, 0), 25.0, 40)


# interior nodes at tile and chunk edges, a corner and inside the layer
SOURCES = [(0, 0, 0), (52, 40, 69), (24, 15, 31), (9, 33, 62)]


def _run(spec, chunks, flow, eta=None, **opts):
    dt = dt_for(spec)
    with fd.Shot(spec.interior, spec.space_order, H, dt, spec.nbl, kernel="tma", **opts) as shot:
        shot.set_model(spec.m, eta)
        for i, src in enumerate(SOURCES):
            shot.inject(*src, inputs.ricker(20.0 + 3 * i, dt, spec.nt))
        for n in chunks:
            (shot.forward_flow if flow else shot.forward)(n)
        return shot.wavefield(0), shot.wavefield(1), shot.step


CASES = [
    (2, "factored", 64, 8, 5), (2, "expanded", 32, 16, 1),
    (4, "factored", 32, 16, 2), (4, "expanded", 128, 8, 9),
    (8, "factored", 32, 32, 4), (8, "expanded", 64, 16, 13),
    (12, "factored", 32, 16, 6), (16, "expanded", 32, 16, 8),
    (16, "factored", 64, 8, 30), (24, "factored", 32, 16, 12), (24, "expanded", 32, 32, 17),
]


@pytest.mark.parametrize("k,form,tz,ty,xb", CASES)
def test_flow_equals_per_step_launches(k, form, tz, ty, xb):
    spec = _spec(k, seed=k + tz)
    rng = np.random.default_rng(k)
    eta = (spec.m * rng.uniform(0, 10.0, spec.m.shape) * (rng.uniform(size=spec.m.shape) < 0.3)).astype(np.float32)
    opts = dict(form=form, tile_z=tz, tile_y=ty, x_block=xb)
    want = _run(spec, [40], False, eta, **opts)
    for chunks in ([40], [1, 16, 23]):
        got = _run(spec, chunks, True, eta, **opts)
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_array_equal(got[1], want[1])
        assert got[2] == want[2] == 40


def test_flow_matches_oracle(oracle_mod):
    k = 8
    spec = _spec(k, seed=5, interior=(40, 35, 44), nbl=6)
    dt = dt_for(spec)
    eta = eta_for(spec)
    srcs = [(s, inputs.ricker(20.0 + 3 * i, dt, spec.nt))
            for i, s in enumerate([(20, 9, 1), (0, 0, 0), (39, 34, 43), (12, 21, 30)])]
    want, want_prev = run_oracle(oracle_mod, spec, spec.nt, dt, eta, sources=srcs)
    with fd.Shot(spec.interior, k, H, dt, spec.nbl) as shot:
        shot.set_model(spec.m, eta)
        for s, w in srcs:
            shot.inject(*s, w)
        shot.forward_flow(spec.nt)
        e0, e1 = rel_l2(shot.wavefield(0), want), rel_l2(shot.wavefield(1), want_prev)
    print(f"PARITY flow_so{k} {e0:.3e} {e1:.3e}")
    assert e0 <= 1e-5 and e1 <= 1e-5


@pytest.mark.parametrize("k", [4, 12])
def test_flow_full_size(k):
    """The 276^3 benchmark shot with the autotuned launch shape: 20 steps in
    one launch equal 20 per-step launches, bit for bit."""
    spec = inputs.sweep_shot(k)
    dt = dt_for(spec)
    wav = inputs.ricker(spec.f0, dt, spec.nt)
    out = []
    for flow in (False, True):
        # the per-step schedule needs the kernel named: the automatic choice is the flow
        with fd.Shot(spec.interior, k, H, dt, spec.nbl, kernel="auto" if flow else "tma") as shot:
            shot.set_model(spec.m)
            shot.inject(*spec.source, wav)
            shot.forward(4)  # tunes the launch shape
            n0 = fd.fd_kernel_launches()
            (shot.forward_flow if flow else shot.forward)(20)
            launches = fd.fd_kernel_launches() - n0
            out.append((shot.wavefield(0), shot.wavefield(1), launches, shot.config))
    (a, ap, na, ca), (b, bp, nb, cb) = out
    assert ca == cb and na == 20 and nb == 1
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ap, bp)


def test_flow_rejections():
    spec = _spec(8, seed=2)
    dt = dt_for(spec)
    for kw in (dict(storage="f16"), dict(kernel="naive"), dict(kernel="stream"), dict(x_block=2)):
        with fd.Shot(spec.interior, 8, H, dt, spec.nbl, **kw) as shot:
            shot.set_model(spec.m)
            with pytest.raises(fd.FdError) as e:
                shot.forward_flow(3)
            assert e.value.code == fd.FD_ENOTSUP, kw
    # BF16 storage: receivers and sources beyond the fused four stay per-step
    with fd.Shot(spec.interior, 8, H, dt, spec.nbl, storage="bf16") as shot:
        shot.set_model(spec.m)
        shot.set_receivers([(1.0, 1.0, 1.0)], 4)
        with pytest.raises(fd.FdError) as e:
            shot.forward_flow(2)
        assert e.value.code == fd.FD_ENOTSUP
    with fd.Shot(spec.interior, 8, H, dt, spec.nbl, storage="bf16") as shot:
        shot.set_model(spec.m)
        for i in range(5):
            shot.inject(3 + i, 4, 5, inputs.ricker(20.0, dt, 10))
        with pytest.raises(fd.FdError) as e:
            shot.forward_flow(2)
        assert e.value.code == fd.FD_ENOTSUP


def _bf16_run(spec, eta, schedule, chunks, **opts):
    dt = dt_for(spec)
    with fd.Shot(spec.interior, spec.space_order, H, dt, spec.nbl, storage="bf16", kernel="tma", **opts) as shot:
        shot.set_model(spec.m, eta)
        for i, src in enumerate(SOURCES):
            shot.inject(*src, inputs.ricker(20.0 + 3 * i, dt, spec.nt))
        for n, how in zip(chunks, schedule):
            (shot.forward_flow if how == "flow" else shot.forward)(n)
        return shot.wavefield(0), shot.wavefield(1)


def _same_values(got, want):
    """The flow stores BF16 levels unscaled, the per-step launches with
    power-of-two scales: the two round identically wherever every intermediate is
    a normal float. Far ahead of the wave front values fall into the FP32
    subnormal range in one and not the other; the tiny difference can flip a
    BF16 rounding there; such a flip is far too small to flip anything 20 orders
    of magnitude larger, so every element above 1e-20 of the field's maximum is
    equal bit for bit and the rest differs by less than that."""
    scale = np.abs(want).max()
    assert scale > 0
    big = np.abs(want) >= 1e-20 * scale
    np.testing.assert_array_equal(got[big], want[big])
    assert np.abs(got[~big] - want[~big]).max(initial=0.0) <= 1e-20 * scale


@pytest.mark.parametrize("k,tz,ty,rows", [(2, 32, 16, 1), (8, 64, 8, 1), (8, 32, 32, 2), (16, 64, 16, 2),
                                          (24, 32, 16, 1)])
def test_bf16_flow_equals_per_step_launches(k, tz, ty, rows):
    """BF16 storage on the flow schedule (unit scales inside the launch) against
    the per-step launches (per-level power-of-two scales): the same values, for
    one launch, chunked launches, and flow and per-step calls interleaved (the
    scale slots handed over in both directions)."""
    spec = _spec(k, seed=300 + k)
    eta = eta_for(spec)
    opts = dict(tile_z=tz, tile_y=ty, rows=rows, x_block=max(k // 2, 9))
    want = _bf16_run(spec, eta, ["step"], [40], **opts)
    for sched, chunks in ((["flow"], [40]), (["flow", "flow", "flow"], [1, 16, 23]),
                          (["step", "flow", "step", "flow"], [5, 11, 7, 17])):
        got = _bf16_run(spec, eta, sched, chunks, **opts)
        _same_values(got[0], want[0])
        _same_values(got[1], want[1])


def test_bf16_flow_matches_oracle(oracle_mod):
    k = 8
    spec = _spec(k, seed=7, interior=(40, 35, 44), nbl=6)
    dt = dt_for(spec)
    eta = eta_for(spec)
    srcs = [(s, inputs.ricker(20.0 + 3 * i, dt, spec.nt)) for i, s in enumerate(SOURCES[:1])]
    want, _ = run_oracle(oracle_mod, spec, spec.nt, dt, eta, sources=srcs)
    with fd.Shot(spec.interior, k, H, dt, spec.nbl, storage="bf16") as shot:
        shot.set_model(spec.m, eta)
        shot.inject(*srcs[0][0], srcs[0][1])
        shot.forward_flow(spec.nt)
        e = rel_l2(shot.wavefield(0), want)
    print(f"PARITY flow_bf16_so{k} {e:.3e}")
    assert e <= 4 * 2.0 ** -9 * spec.nt ** 0.5
