"""GPU tests of the two-steps-per-launch forward (temporal blocking): bit for
bit the single-step result (even and odd step counts, chunked calls, sources
near tile edges and inside the absorbing layer, ragged grids), and the FP64
oracle within the FP32 bound; the unsupported cases are rejected."""
import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import inputs
from harness import dt_for, eta_for, rel_l2, run_oracle

pytestmark = pytest.mark.gpu
H = inputs.H


def _spec(k, seed, interior=(61, 47, 130), nbl=7):
    rng = np.random.default_rng(seed)
    vel = inputs.smooth_random_velocity(interior, nbl, rng, sigma=4.0)
    return inputs.ShotSpec(interior, nbl, k, vel, (0, 0, 0), 25.0, 57)


# interior nodes next to the two-step tile edges (z tiles of 56 from domain z = 0,
# y tiles of 16 - 2R rows), inside the layer and in the middle
SOURCES = [(30, 9, 48), (0, 0, 0), (60, 46, 129), (12, 21, 110)]


def _run(spec, chunks, two_step, eta=None):
    dt = dt_for(spec)
    with fd.Shot(spec.interior, spec.space_order, H, dt, spec.nbl) as shot:
        shot.set_model(spec.m, eta)
        for i, src in enumerate(SOURCES):
            shot.inject(*src, inputs.ricker(20.0 + 3 * i, dt, spec.nt))
        for n in chunks:
            (shot.forward_two_step if two_step else shot.forward)(n)
        return shot.wavefield(0), shot.wavefield(1), shot.step


@pytest.mark.parametrize("k", [2, 4])
def test_two_step_equals_single_step(k):
    spec = _spec(k, seed=k)
    want = _run(spec, [57], False)
    for chunks in ([57], [10, 47], [1, 2, 3, 51]):
        got = _run(spec, chunks, True)
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_array_equal(got[1], want[1])
        assert got[2] == want[2] == 57


@pytest.mark.parametrize("k", [2, 4])
def test_two_step_matches_oracle(oracle_mod, k):
    spec = _spec(k, seed=10 + k, interior=(40, 35, 70), nbl=6)
    dt = dt_for(spec)
    eta = eta_for(spec)
    srcs = [(s, inputs.ricker(20.0 + 3 * i, dt, spec.nt))
            for i, s in enumerate([(20, 9, 1), (0, 0, 0), (39, 34, 69), (12, 21, 50)])]
    want, want_prev = run_oracle(oracle_mod, spec, spec.nt, dt, eta, sources=srcs)
    with fd.Shot(spec.interior, k, H, dt, spec.nbl) as shot:
        shot.set_model(spec.m, eta)
        for s, w in srcs:
            shot.inject(*s, w)
        shot.forward_two_step(spec.nt)
        e0, e1 = rel_l2(shot.wavefield(0), want), rel_l2(shot.wavefield(1), want_prev)
    print(f"PARITY two_step_so{k} {e0:.3e} {e1:.3e}")
    assert e0 <= 1e-5 and e1 <= 1e-5


def test_two_step_rejects_unsupported():
    spec = _spec(8, seed=3)
    dt = dt_for(spec)
    for kw, k in (({}, 8), ({"storage": "bf16"}, 4), ({"form": "expanded"}, 4)):
        with fd.Shot(spec.interior, k, H, dt, spec.nbl, **kw) as shot:
            shot.set_model(spec.m)
            with pytest.raises(fd.FdError) as e:
                shot.forward_two_step(2)
            assert e.value.code == fd.FD_ENOTSUP
    with fd.Shot(spec.interior, 4, H, dt, spec.nbl) as shot:
        shot.set_model(spec.m)
        shot.set_receivers([(1.0, 1.0, 1.0)], 4)
        with pytest.raises(fd.FdError) as e:
            shot.forward_two_step(2)
        assert e.value.code == fd.FD_ENOTSUP


def test_two_step_launch_count_and_timing():
    """A forward of nt steps at space order 2 (automatic kernel choice) runs
    nt // 2 two-step launches plus one single step for odd nt; the library's
    launch counter sees exactly those (no other kernels), and the device time
    of the call covers all of them, the odd step included."""
    spec = _spec(2, seed=7, interior=(120, 120, 120), nbl=8)
    dt = dt_for(spec)
    with fd.Shot(spec.interior, 2, H, dt, spec.nbl) as shot:
        shot.set_model(spec.m)
        shot.inject(60, 60, 60, inputs.ricker(20.0, dt, 200))
        for nt in (10, 41, 1):  # first calls tune and capture; the counts below are of repeats
            shot.forward(nt)
        counts, ms = {}, {}
        for nt in (10, 41, 1):
            n0 = fd.fd_kernel_launches()
            shot.forward(nt)
            counts[nt] = fd.fd_kernel_launches() - n0
            ms[nt] = shot.last_forward_ms()
    assert counts == {10: 5, 41: 21, 1: 1}
    assert ms[41] > 4 * ms[1] and ms[41] > 2 * ms[10]


def test_single_step_launch_count():
    """Per-step schedule: one launch per step through the replayed graph, one
    more per step with more sources than the step kernel fuses (the
    extra-source kernel)."""
    spec = _spec(8, seed=8)
    dt = dt_for(spec)
    with fd.Shot(spec.interior, 8, H, dt, spec.nbl, kernel="tma") as shot:
        shot.set_model(spec.m)
        shot.inject(10, 10, 10, inputs.ricker(20.0, dt, 40))
        shot.forward(6)
        n0 = fd.fd_kernel_launches()
        shot.forward(6)
        assert fd.fd_kernel_launches() - n0 == 6
        for i in range(4):
            shot.inject(12 + i, 10, 10, inputs.ricker(20.0, dt, 40))
        shot.forward(6)
        n0 = fd.fd_kernel_launches()
        shot.forward(6)
        assert fd.fd_kernel_launches() - n0 == 12


def test_flow_launch_count():
    """Automatic kernel choice at space order 8: one flow launch per call, also
    with more sources than the kernel fuses (the items add them) and with
    receivers (the items sample them; one more launch samples the last level);
    with FP16 storage, one launch per step plus the extra-source kernel."""
    spec = _spec(8, seed=8)
    dt = dt_for(spec)
    with fd.Shot(spec.interior, 8, H, dt, spec.nbl) as shot:
        shot.set_model(spec.m)
        shot.inject(10, 10, 10, inputs.ricker(20.0, dt, 40))
        shot.forward(6)
        n0 = fd.fd_kernel_launches()
        shot.forward(6)
        assert fd.fd_kernel_launches() - n0 == 1
        for i in range(4):
            shot.inject(12 + i, 10, 10, inputs.ricker(20.0, dt, 40))
        shot.forward(6)
        n0 = fd.fd_kernel_launches()
        shot.forward(6)
        assert fd.fd_kernel_launches() - n0 == 1
        assert shot.schedule[1] == 1
        shot.set_receivers([(3.5, 4.25, 5.0), (20.0, 1.0, 7.5)], 40)
        shot.forward(6)
        n0 = fd.fd_kernel_launches()
        shot.forward(6)
        assert fd.fd_kernel_launches() - n0 == 2
        assert shot.traces().shape == (2, 12)
    with fd.Shot(spec.interior, 8, H, dt, spec.nbl, storage="f16") as shot:
        shot.set_model(spec.m)
        for i in range(5):
            shot.inject(10 + i, 10, 10, inputs.ricker(20.0, dt, 40))
        shot.forward(6)
        n0 = fd.fd_kernel_launches()
        shot.forward(6)
        assert fd.fd_kernel_launches() - n0 == 12
