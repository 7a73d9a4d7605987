"""Failure detection on the device without a fault: the bounded waits of the
step kernels (ring mbarrier, flow-schedule dependency flag) give up after
their time limits when nothing completes them, the kernel returns, and the
context stays usable for the next shot."""
import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import inputs
from harness import dt_for

pytestmark = pytest.mark.gpu


def test_bounded_waits_give_up_and_the_context_survives():
    status, t_mbar, t_flag = fd.fd_selftest_waits()
    print(f"SELFTEST status {status} mbarrier wait {t_mbar:.3f} s, flag wait {t_flag:.3f} s")
    assert status == 3
    assert 0.9 <= t_mbar <= 5.0
    assert 1.9 <= t_flag <= 6.0
    # the same process goes on computing: a shot advances and reports a finite field
    rng = np.random.default_rng(1)
    vel = inputs.smooth_random_velocity((30, 30, 30), 5, rng, sigma=3.0)
    spec = inputs.ShotSpec((30, 30, 30), 5, 8, vel, (15, 15, 15), 25.0, 40)
    dt = dt_for(spec)
    with fd.Shot(spec.interior, 8, inputs.H, dt, spec.nbl) as shot:
        shot.set_model(spec.m)
        shot.inject(15, 15, 15, inputs.ricker(25.0, dt, 40))
        shot.forward(40)
        u = shot.wavefield(0)
    assert np.isfinite(u).all() and np.abs(u).max() > 0
