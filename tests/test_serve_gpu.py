"""GPU test of the continuous-batching server: requests of different sizes,
space orders and storages arrive over time, are admitted as memory frees up,
share launches with whatever else is resident, and each result equals the same
request run alone (bit for bit: same per-point arithmetic)."""
import numpy as np
import pytest

import paper_1912_00695_gb300 as fd
from paper_1912_00695_gb300 import inputs
from paper_1912_00695_gb300.serve import Request, Server

pytestmark = pytest.mark.gpu
H = inputs.H


def _requests(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        interior = tuple(int(v) for v in rng.integers(20, 49, size=3))
        nbl = 4
        k = int(rng.choice([4, 8]))
        storage = ["f32", "bf16"][i % 2]
        vel = inputs.smooth_random_velocity(interior, nbl, rng, sigma=3.0)
        dt = 0.9 * fd.fd_dt_max(k, H, float(vel.max()))
        nt = int(rng.integers(20, 61))
        src = tuple(int(rng.integers(0, n)) for n in interior)
        wav = inputs.ricker(float(rng.uniform(15, 25)), dt, nt)
        out.append(Request(i, 0.003 * i, interior, nbl, k, storage, dt, inputs.slowness2(vel),
                           src, wav, nt))
    return out


def _alone(r):
    with fd.Shot(r.interior, r.space_order, H, r.dt, r.nbl, storage=r.storage, kernel="tma",
                 tile_z=32, tile_y=16) as shot:
        shot.set_model(r.m)
        shot.inject(*r.source, r.wavelet)
        shot.forward(r.nt)
        return shot.wavefield(0)


@pytest.mark.parametrize("realtime", [False, True])
def test_served_results_equal_alone(realtime):
    """Offline (every request present at once, so the memory budget makes some
    wait) and on the wall clock (arrivals 3 ms apart)."""
    reqs = _requests(0, 10)
    budget = sum(sorted(r.device_bytes for r in reqs)[-3:])  # about three shots at a time
    srv = Server(H, budget, chunk=16)
    stats = srv.run(reqs, realtime=realtime)
    srv.close()
    assert stats["requests"] == len(reqs)
    assert srv.peak_used <= budget
    if not realtime:
        assert sum(r.admitted > 0 for r in reqs) >= 3  # admitted only as memory freed up
    for r in reqs:
        np.testing.assert_array_equal(r.result, _alone(r), err_msg=f"request {r.rid}")
    assert 0 <= stats["p50_s"] <= stats["p99_s"]
